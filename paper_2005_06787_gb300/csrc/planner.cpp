// Contraction-scheme search (Sec. 4, Supp. A.2): branch clusters, stem growth,
// stem-local optimisation and dynamic slicing, scored with the time and space
// complexities of Supp. A.1 (a step costs 2^|E_AB| and holds 2^|E*_AB|; tc
// sums, cw maxes, slicing multiplies tc by 2^|E_s|).
//
// Differences from the paper's search, and why: the paper finds the stem by
// KaHyPar multipartition + recursive bipartition tuned by CMA-ES; neither
// library is available, so the stem is grown here one branch at a time from a
// seed cluster (the same "stem absorbs small branches" shape, Sec. 4), with
// randomised restarts in place of the parameter search. Local optimisation
// brute-forces the order of short windows of consecutive stem steps, the
// branch-switch move of the paper's local-optimisation figure.
#include <algorithm>
#include <atomic>
#include <exception>
#include <mutex>
#include <thread>
#include <array>
#include <cmath>
#include <limits>
#include <map>
#include <numeric>
#include <set>

#include "internal.h"

namespace tn {

double log2_add(double a, double b) {
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    double m = std::max(a, b);
    return m + std::log2(std::exp2(a - m) + std::exp2(b - m));
}

static Bits leaf_bits(const Network &net, int leaf) {
    Bits b(net.n_edges());
    for (int e : net.leaves[(size_t)leaf].edges) b.set(e);
    return b;
}

// Internal cost of a cluster's subtree: sum of 2^|E_u| (log2), with the
// sliced edges removed, and its max |E*_u|.
static void cluster_cost(const Network &net, const Cluster &c, const Bits &sliced, double &log2tc,
                         int &maxw) {
    log2tc = -INFINITY;
    maxw = 0;
    std::vector<Bits> node;
    node.reserve(c.pairs.size());
    auto get = [&](int ref) -> Bits {
        if (ref >= 0) return leaf_bits(net, ref).andnot(sliced);
        return node[(size_t)(-ref - 1)];
    };
    for (auto &p : c.pairs) {
        Bits a = get(p.first), b = get(p.second);
        int eu = count_or(a, b);
        log2tc = log2_add(log2tc, (double)eu);
        Bits o = a ^ b;
        maxw = std::max(maxw, o.count());
        node.push_back(o);
    }
}

// ------------------------------------------------------------------ clusters
// Greedy pairwise merging with a rank cap: repeatedly merge the two adjacent
// clusters whose merged tensor grows least (2^|out| - 2^|a| - 2^|b|), as long
// as the merged rank stays <= cap. Ties: the smallest (min id, max id).
static std::vector<Cluster> make_clusters(const Network &net, int cap, std::mt19937_64 &rng,
                                          double noise) {
    const int L = net.n_leaves();
    std::vector<Cluster> cl((size_t)L);
    std::vector<int> alive((size_t)L, 1);
    std::vector<int> ref((size_t)L);  // cluster id -> ref of its root in its pair list
    for (int i = 0; i < L; ++i) {
        cl[(size_t)i].leaves = {i};
        cl[(size_t)i].out = leaf_bits(net, i);
        ref[(size_t)i] = i;
    }
    // edge -> clusters at its ends
    std::vector<std::array<int, 2>> ends((size_t)net.n_edges());
    for (int e = 0; e < net.n_edges(); ++e) {
        const EdgeInfo &E = net.edges[(size_t)e];
        ends[(size_t)e] = {E.ends[0], E.n_ends > 1 ? E.ends[1] : -1};
    }
    std::uniform_real_distribution<double> U(0.0, 1.0);
    while (true) {
        double best = INFINITY;
        int ba = -1, bb = -1;
        for (int e = 0; e < net.n_edges(); ++e) {
            int a = ends[(size_t)e][0], b = ends[(size_t)e][1];
            if (a < 0 || b < 0 || a == b) continue;
            int ra = cl[(size_t)a].out.count(), rb = cl[(size_t)b].out.count();
            int ro = count_xor(cl[(size_t)a].out, cl[(size_t)b].out);
            if (ro > cap) continue;
            double score = std::exp2(ro) - std::exp2(ra) - std::exp2(rb);
            if (noise > 0) score += noise * U(rng);
            int lo = std::min(a, b), hi = std::max(a, b);
            if (score < best || (score == best && (lo < std::min(ba, bb) ||
                                                  (lo == std::min(ba, bb) && hi < std::max(ba, bb))))) {
                best = score;
                ba = lo;
                bb = hi;
            }
        }
        if (ba < 0) break;
        // merge bb into ba
        Cluster &A = cl[(size_t)ba];
        Cluster &B = cl[(size_t)bb];
        int ra = ref[(size_t)ba], rb = ref[(size_t)bb];
        // re-base B's internal refs
        int base = (int)A.pairs.size();
        for (auto p : B.pairs) {
            auto fix = [&](int r) { return r >= 0 ? r : -((-r - 1) + base + 1); };
            A.pairs.push_back({fix(p.first), fix(p.second)});
        }
        if (rb < 0) rb = -((-rb - 1) + base + 1);
        A.pairs.push_back({ra, rb});
        ref[(size_t)ba] = -(int)A.pairs.size();
        A.leaves.insert(A.leaves.end(), B.leaves.begin(), B.leaves.end());
        A.out ^= B.out;
        alive[(size_t)bb] = 0;
        for (auto &en : ends) {
            if (en[0] == bb) en[0] = ba;
            if (en[1] == bb) en[1] = ba;
        }
        B.pairs.clear();
        B.leaves.clear();
    }
    std::vector<Cluster> out;
    for (int i = 0; i < L; ++i)
        if (alive[(size_t)i]) out.push_back(std::move(cl[(size_t)i]));
    return out;
}

// ------------------------------------------------------------------ stem cost
struct StemEval {
    double log2_stem = -INFINITY;  // log2 sum over stem steps of 2^|E_u|
    int max_rank = 0;               // max stem tensor rank (incl. the seed)
};

static StemEval eval_stem(const std::vector<Bits> &B, int seed, const std::vector<int> &order,
                          const Bits &sliced) {
    StemEval r;
    Bits S = B[(size_t)seed].andnot(sliced);
    r.max_rank = S.count();
    for (int c : order) {
        Bits b = B[(size_t)c].andnot(sliced);
        r.log2_stem = log2_add(r.log2_stem, (double)count_or(S, b));
        S ^= b;
        r.max_rank = std::max(r.max_rank, S.count());
    }
    return r;
}

// Score of a scheme for the search: log2 of the per-slice stem cost times the
// slice count, plus one doubling per bit the width exceeds the limit (each
// such bit will cost about one more sliced edge).
static double scheme_score(const StemEval &e, int n_sliced, int limit) {
    return e.log2_stem + n_sliced + std::max(0, e.max_rank - limit);
}

// Grow a stem from `seed`: absorb, one at a time, the adjacent cluster that
// gives the smallest new stem rank (ties: most shared edges, then noise).
static std::vector<int> grow_stem(const std::vector<Bits> &B, int seed, std::mt19937_64 &rng,
                                  double noise) {
    const int C = (int)B.size();
    std::vector<int> order;
    std::vector<char> used((size_t)C, 0);
    used[(size_t)seed] = 1;
    Bits S = B[(size_t)seed];
    std::uniform_real_distribution<double> U(0.0, 1.0);
    for (int it = 1; it < C; ++it) {
        double best = INFINITY;
        int bc = -1;
        for (int c = 0; c < C; ++c) {
            if (used[(size_t)c]) continue;
            int sh = count_and(S, B[(size_t)c]);
            if (sh == 0) continue;
            int nr = count_xor(S, B[(size_t)c]);
            double score = nr - 0.01 * sh + noise * U(rng);
            if (score < best) {
                best = score;
                bc = c;
            }
        }
        if (bc < 0) {  // disconnected remainder: take the first unused
            for (int c = 0; c < C; ++c)
                if (!used[(size_t)c]) { bc = c; break; }
        }
        used[(size_t)bc] = 1;
        S ^= B[(size_t)bc];
        order.push_back(bc);
    }
    return order;
}

// Supp. A.2 "Local optimization": for each window of w consecutive stem
// steps, try every order of its branches and keep the best. The stem tensor
// after the window does not depend on the order, so the move is local.
static bool local_opt(const std::vector<Bits> &B, int seed, std::vector<int> &order,
                      const Bits &sliced, int limit, int w, int n_sliced) {
    const int L = (int)order.size();
    if (L < 2) return false;
    bool improved_any = false;
    std::vector<Bits> Bs(B.size());
    for (size_t i = 0; i < B.size(); ++i) Bs[i] = B[i].andnot(sliced);
    // prefix stem tensors
    std::vector<Bits> pre((size_t)L + 1);
    std::vector<double> stepc((size_t)L);
    std::vector<int> rank((size_t)L + 1);
    auto rebuild = [&]() {
        pre[0] = Bs[(size_t)seed];
        rank[0] = pre[0].count();
        for (int i = 0; i < L; ++i) {
            const Bits &b = Bs[(size_t)order[(size_t)i]];
            stepc[(size_t)i] = (double)count_or(pre[(size_t)i], b);
            pre[(size_t)i + 1] = pre[(size_t)i] ^ b;
            rank[(size_t)i + 1] = pre[(size_t)i + 1].count();
        }
    };
    rebuild();
    for (int start = 0; start + 1 < L; ++start) {
        int ww = std::min(w, L - start);
        // totals outside the window
        double out_tc = -INFINITY;
        int out_max = rank[0];
        for (int i = 0; i < L; ++i) {
            if (i >= start && i < start + ww) continue;
            out_tc = log2_add(out_tc, stepc[(size_t)i]);
        }
        for (int i = 1; i <= L; ++i)
            if (i <= start || i >= start + ww) out_max = std::max(out_max, rank[(size_t)i]);
        std::vector<int> win(order.begin() + start, order.begin() + start + ww);
        auto eval_win = [&](const std::vector<int> &pw, double &tc, int &mx) {
            Bits S = pre[(size_t)start];
            tc = -INFINITY;
            mx = 0;
            for (size_t j = 0; j < pw.size(); ++j) {
                const Bits &b = Bs[(size_t)pw[j]];
                tc = log2_add(tc, (double)count_or(S, b));
                S ^= b;
                if (j + 1 < pw.size()) mx = std::max(mx, S.count());
            }
        };
        double tc0;
        int mx0;
        eval_win(win, tc0, mx0);
        auto score_of = [&](double tc, int mx) {
            StemEval e;
            e.log2_stem = log2_add(out_tc, tc);
            e.max_rank = std::max(out_max, mx);
            return scheme_score(e, n_sliced, limit);
        };
        double best = score_of(tc0, mx0);
        // never widen the stem beyond max(limit, its current width)
        const int cap = std::max(limit, std::max(out_max, mx0));
        std::vector<int> perm(win), bestp(win);
        std::sort(perm.begin(), perm.end());
        do {
            double tc;
            int mx;
            eval_win(perm, tc, mx);
            if (std::max(out_max, mx) > cap) continue;
            double s = score_of(tc, mx);
            if (s < best - 1e-12) {
                best = s;
                bestp = perm;
            }
        } while (std::next_permutation(perm.begin(), perm.end()));
        if (bestp != win) {
            std::copy(bestp.begin(), bestp.end(), order.begin() + start);
            improved_any = true;
            rebuild();
        }
    }
    return improved_any;
}

static void local_opt_sweeps(const std::vector<Bits> &B, int seed, std::vector<int> &order,
                             const Bits &sliced, int limit, int sweeps, int n_sliced) {
    for (int s = 0; s < sweeps; ++s)
        if (!local_opt(B, seed, order, sliced, limit, 4, n_sliced)) break;
}

// Supp. A.2 "Local optimization", widened: simulated annealing over the
// stem order. A move takes one branch out of the order and puts it back up
// to `window` places away; only the stem tensors between the two places
// change, so a move is scored by recomputing that stretch. Score: log2 of
// the stem cost plus one unit per bit the widest stem tensor exceeds the
// limit (each such bit costs about one more sliced edge), plus area_w times
// the excess width summed over all stem tensors (how long the stem stays
// wide, which decides how many sliced edges it will need). Metropolis
// acceptance at a temperature falling geometrically from t0 to t1.
static void anneal_order(const std::vector<Bits> &B, int seed, std::vector<int> &order,
                         const Bits &sliced, int limit, long iters, std::mt19937_64 &rng,
                         double t0 = 1.0, double t1 = 0.02, int window = 48, int cap_rank = 1 << 30,
                         double area_w = 0.0) {
    const int L = (int)order.size();
    if (L < 3 || iters <= 0) return;
    std::vector<Bits> Bs(B.size());
    for (size_t i = 0; i < B.size(); ++i) Bs[i] = B[i].andnot(sliced);
    std::vector<Bits> pre((size_t)L + 1);
    std::vector<double> cost((size_t)L);  // 2^|E_u| of each stem step
    std::vector<int> rank((size_t)L + 1);
    pre[0] = Bs[(size_t)seed];
    rank[0] = pre[0].count();
    for (int i = 0; i < L; ++i) {
        const Bits &b = Bs[(size_t)order[(size_t)i]];
        cost[(size_t)i] = std::exp2((double)count_or(pre[(size_t)i], b));
        pre[(size_t)i + 1] = pre[(size_t)i] ^ b;
        rank[(size_t)i + 1] = pre[(size_t)i + 1].count();
    }
    double total = 0;
    for (double c : cost) total += c;
    auto max_rank = [&](const std::vector<int> &r) { return *std::max_element(r.begin(), r.end()); };
    auto area = [&](const std::vector<int> &r) {
        double a = 0;
        if (area_w > 0)
            for (int v : r) a += std::max(0, v - limit);
        return area_w * a;
    };
    auto score = [&](double tot, int mr) { return std::log2(tot) + std::max(0, mr - limit); };
    double cur = score(total, max_rank(rank)) + area(rank);
    std::vector<int> best_order = order;
    double best = cur;
    std::uniform_real_distribution<double> U(0.0, 1.0);
    std::uniform_int_distribution<int> pos(0, L - 1);
    std::uniform_int_distribution<int> off(-window, window);
    std::vector<Bits> npre;
    std::vector<double> ncost;
    std::vector<int> nrank(rank);
    std::vector<int> seg;
    for (long it = 0; it < iters; ++it) {
        const double T = t0 * std::pow(t1 / t0, (double)it / (double)iters);
        const int i = pos(rng);
        int j = i + off(rng);
        if (j < 0 || j >= L || j == i) continue;
        const int lo = std::min(i, j), hi = std::max(i, j);
        // new order of positions lo..hi
        seg.assign(order.begin() + lo, order.begin() + hi + 1);
        if (i < j)
            std::rotate(seg.begin(), seg.begin() + 1, seg.end());
        else
            std::rotate(seg.begin(), seg.end() - 1, seg.end());
        npre.resize(seg.size() + 1);
        ncost.resize(seg.size());
        npre[0] = pre[(size_t)lo];
        double old_part = 0, new_part = 0;
        for (size_t t = 0; t < seg.size(); ++t) {
            const Bits &b = Bs[(size_t)seg[t]];
            ncost[t] = std::exp2((double)count_or(npre[t], b));
            npre[t + 1] = npre[t] ^ b;
            new_part += ncost[t];
            old_part += cost[(size_t)lo + t];
        }
        for (size_t t = 1; t < seg.size(); ++t) nrank[(size_t)lo + t] = npre[t].count();
        const double ntotal = total - old_part + new_part;
        const int nmax = max_rank(nrank);
        const double nscore = score(ntotal, nmax) + area(nrank);
        const double d = nscore - cur;
        if (nmax <= cap_rank && (d <= 0 || U(rng) < std::exp(-d / T))) {
            std::copy(seg.begin(), seg.end(), order.begin() + lo);
            for (size_t t = 0; t < seg.size(); ++t) {
                cost[(size_t)lo + t] = ncost[t];
                pre[(size_t)lo + t + 1] = npre[t + 1];
            }
            rank = nrank;
            total = ntotal;
            cur = nscore;
            if (cur < best - 1e-12) {
                best = cur;
                best_order = order;
            }
        } else {
            for (size_t t = 1; t < seg.size(); ++t) nrank[(size_t)lo + t] = rank[(size_t)lo + t];
        }
    }
    order = best_order;
}

// Joint refinement of the stem order and the sliced set once the width is
// within the limit: besides the order moves of anneal_order, a move swaps
// one sliced edge for an unsliced edge of a widest stem tensor, or drops a
// sliced edge (never below min_sliced). The score is the total cost over all
// slices, log2 stem cost + |sliced|, and the width limit is hard, so the
// search keeps slices on edges that live through the expensive part of the
// stem (those slice almost for free, as the paper observes for its stems).
static void anneal_sliced(const Network &net, const std::vector<Bits> &B, int seed,
                          std::vector<int> &order, Bits &sliced, std::vector<int> &sliced_list,
                          int limit, int min_sliced, long iters, std::mt19937_64 &rng) {
    const int L = (int)order.size();
    if (L < 3 || iters <= 0 || sliced_list.empty()) return;
    Bits open(net.n_edges());
    for (int e : net.open_edges) open.set(e);
    auto evaluate = [&](const std::vector<int> &ord, const Bits &sl, int nsl, std::vector<Bits> *wide) {
        Bits S = B[(size_t)seed].andnot(sl);
        double tot = 0;
        int mr = S.count();
        std::vector<Bits> tens;
        if (wide) tens.push_back(S);
        for (int c : ord) {
            const Bits b = B[(size_t)c].andnot(sl);
            tot += std::exp2((double)count_or(S, b));
            S ^= b;
            mr = std::max(mr, S.count());
            if (wide) tens.push_back(S);
        }
        if (wide) {
            wide->clear();
            for (auto &t : tens)
                if (t.count() >= mr) wide->push_back(t);
        }
        if (mr > limit) return (double)INFINITY;  // the width limit is hard once met
        return std::log2(tot) + nsl;
    };
    std::vector<Bits> wide;
    double cur = evaluate(order, sliced, (int)sliced_list.size(), &wide);
    double best = cur;
    std::vector<int> best_order = order, best_list = sliced_list;
    Bits best_sliced = sliced;
    std::uniform_real_distribution<double> U(0.0, 1.0);
    std::uniform_int_distribution<int> pos(0, L - 1), off(-32, 32);
    const double t0 = 0.3, t1 = 0.005;
    for (long it = 0; it < iters; ++it) {
        const double T = t0 * std::pow(t1 / t0, (double)it / (double)iters);
        std::vector<int> ord2 = order;
        Bits sl2 = sliced;
        std::vector<int> list2 = sliced_list;
        const double r = U(rng);
        if (r < 0.7) {
            const int i = pos(rng), j = i + off(rng);
            if (j < 0 || j >= L || j == i) continue;
            const int v = ord2[(size_t)i];
            ord2.erase(ord2.begin() + i);
            ord2.insert(ord2.begin() + j, v);
        } else if (r < 0.95 || list2.size() < 2 || (int)list2.size() <= min_sliced) {
            // swap a sliced edge for an unsliced edge of a widest tensor
            std::vector<int> cand;
            for (auto &t : wide)
                for (int e : t.list())
                    if (!open.test(e)) cand.push_back(e);
            if (cand.empty()) continue;
            const int e_new = cand[(size_t)(U(rng) * (double)cand.size()) % cand.size()];
            const size_t k = (size_t)(U(rng) * (double)list2.size()) % list2.size();
            sl2.reset(list2[k]);
            sl2.set(e_new);
            list2[k] = e_new;
        } else {
            const size_t k = (size_t)(U(rng) * (double)list2.size()) % list2.size();
            sl2.reset(list2[k]);
            list2.erase(list2.begin() + (long)k);
        }
        std::vector<Bits> wide2;
        const double sc = evaluate(ord2, sl2, (int)list2.size(), &wide2);
        const double d = sc - cur;
        if (d <= 0 || U(rng) < std::exp(-d / T)) {
            order.swap(ord2);
            sliced = sl2;
            sliced_list.swap(list2);
            wide.swap(wide2);
            cur = sc;
            if (cur < best - 1e-12) {
                best = cur;
                best_order = order;
                best_sliced = sliced;
                best_list = sliced_list;
            }
        }
    }
    order = best_order;
    sliced = best_sliced;
    sliced_list = best_list;
}

// Supp. A.2 "Dynamic slicing": slice, one edge at a time, the edge of the
// widest stem tensors whose slicing raises the total cost least (ties: the
// lowest edge id), with local optimisation in between.
static bool dynamic_slice(const Network &net, const std::vector<Bits> &B, int seed,
                          std::vector<int> &order, Bits &sliced, std::vector<int> &sliced_list,
                          int limit, int min_sliced, int max_sliced, int lo_iters, long anneal,
                          std::mt19937_64 &rng) {
    Bits open(net.n_edges());
    for (int e : net.open_edges) open.set(e);
    while (true) {
        StemEval ev = eval_stem(B, seed, order, sliced);
        if (ev.max_rank <= limit && (int)sliced_list.size() >= min_sliced) return true;
        if ((int)sliced_list.size() >= max_sliced) return false;
        // widest stem tensors
        std::vector<Bits> wide;
        Bits S = B[(size_t)seed].andnot(sliced);
        std::vector<Bits> tens{S};
        for (int c : order) {
            S ^= B[(size_t)c].andnot(sliced);
            tens.push_back(S);
        }
        for (auto &t : tens)
            if (t.count() == ev.max_rank) wide.push_back(t);
        std::map<int, int> hits;
        for (auto &t : wide)
            for (int e : t.list())
                if (!open.test(e)) hits[e]++;
        if (hits.empty()) return false;
        int maxhit = 0;
        for (auto &h : hits) maxhit = std::max(maxhit, h.second);
        int best_e = -1;
        double best = INFINITY;
        for (auto &h : hits) {
            if (2 * h.second < maxhit) continue;
            Bits s2 = sliced;
            s2.set(h.first);
            StemEval e2 = eval_stem(B, seed, order, s2);
            double sc = e2.log2_stem + (double)(sliced_list.size() + 1) -
                        0.5 * (double)h.second / (double)wide.size();
            if (sc < best) {
                best = sc;
                best_e = h.first;
            }
        }
        sliced.set(best_e);
        sliced_list.push_back(best_e);
        // restructure without widening the stem beyond its current width
        const int cap = eval_stem(B, seed, order, sliced).max_rank;
        anneal_order(B, seed, order, sliced, limit, anneal, rng, 0.3, 0.01, 48, cap);
        local_opt_sweeps(B, seed, order, sliced, limit, lo_iters, (int)sliced_list.size());
    }
}

void evaluate_scheme(const Network &net, Scheme &s) {
    std::vector<Bits> B;
    for (auto &c : s.clusters) B.push_back(c.out);
    StemEval ev = eval_stem(B, s.seed_cluster, s.stem_order, s.sliced);
    double br = -INFINITY;
    int brw = 0;
    Bits none(net.n_edges());
    double br_unsliced = -INFINITY;
    for (auto &c : s.clusters) {
        if (c.pairs.empty()) continue;
        double t;
        int w;
        cluster_cost(net, c, s.sliced, t, w);
        br = log2_add(br, t);
        brw = std::max(brw, w);
        cluster_cost(net, c, none, t, w);
        br_unsliced = log2_add(br_unsliced, t);
    }
    s.stem_tc = std::exp2(ev.log2_stem);
    s.branch_tc = std::exp2(br_unsliced);
    s.log2_tc = log2_add(ev.log2_stem, br) + (double)s.sliced_list.size();
    s.cw = std::max(ev.max_rank, brw);
}

Scheme plan_scheme(const Network &net, const tn_plan_opts &o) {
    const int limit = o.cw_limit > 0 ? o.cw_limit : 30;
    const int restarts = o.restarts > 0 ? o.restarts : 8;
    const int lo_iters = o.local_opt_iters > 0 ? o.local_opt_iters : 4;
    const int cap = o.branch_rank > 0 ? o.branch_rank : 4;
    const int max_sl = o.max_sliced > 0 ? o.max_sliced : 40;
    // annealing moves per restart: explicit, off (< 0), or by default 600 per
    // branch cluster (at most 200000)
    std::mt19937_64 rng(o.seed ? o.seed : 0x5eedull);
    Scheme best;
    double best_score = INFINITY;
    std::vector<Cluster> clusters = make_clusters(net, cap, rng, 0.0);
    std::vector<Bits> B;
    for (auto &c : clusters) B.push_back(c.out);
    const int C = (int)clusters.size();
    const long anneal = o.anneal_iters > 0   ? (long)o.anneal_iters
                        : o.anneal_iters < 0 ? 0L
                                             : std::min(200000L, 600L * (long)C);
    if (C == 1) {
        Scheme s;
        s.clusters = clusters;
        s.seed_cluster = 0;
        s.sliced = Bits(net.n_edges());
        evaluate_scheme(net, s);
        return s;
    }
    // seeds: spread over clusters deterministically, the rest random
    std::uniform_int_distribution<int> pick(0, C - 1);
    struct Candidate {
        double score = INFINITY;
        int seed = -1;
        std::vector<int> order, sl;
        Bits sliced;
    };
    auto take = [&](const Candidate &c) {
        if (c.seed < 0 || !(c.score < best_score)) return;
        best_score = c.score;
        best.clusters = clusters;
        best.seed_cluster = c.seed;
        best.stem_order = c.order;
        best.sliced = c.sliced;
        best.sliced_list = c.sl;
    };
    // slicing and refinement of one annealed order: dynamic slicing with an
    // anneal after every pick, an order anneal that may not widen, the joint
    // order / sliced-set anneal, window optimisation. False when slicing
    // misses the limit. Reads only shared inputs and the given random stream.
    auto slice_refine_into = [&](int seed, std::vector<int> order, long ann, std::mt19937_64 &r,
                                 Candidate &out) {
        Bits sliced(net.n_edges());
        std::vector<int> sl;
        if (!dynamic_slice(net, B, seed, order, sliced, sl, limit, o.min_sliced, max_sl, lo_iters, ann / 10, r))
            return false;
        anneal_order(B, seed, order, sliced, limit, ann / 2, r, 0.3, 0.01, 48, limit);
        anneal_sliced(net, B, seed, order, sliced, sl, limit, o.min_sliced, ann / 4, r);
        local_opt_sweeps(B, seed, order, sliced, limit, lo_iters, (int)sl.size());
        StemEval ev = eval_stem(B, seed, order, sliced);
        if (ev.max_rank > limit) return false;
        out.score = scheme_score(ev, (int)sl.size(), limit);
        out.seed = seed;
        out.order = std::move(order);
        out.sliced = sliced;
        out.sl = std::move(sl);
        return true;
    };
    auto slice_refine = [&](int seed, std::vector<int> order, long ann) {
        Candidate c;
        if (!slice_refine_into(seed, std::move(order), ann, rng, c)) return false;
        take(c);
        return true;
    };
    // unsliced anneal + window optimisation of a grown stem
    auto shape_with = [&](int seed, std::vector<int> order, long ann, std::mt19937_64 &r) {
        Bits none(net.n_edges());
        anneal_order(B, seed, order, none, limit, ann, r, 1.0, 0.02, 48, 1 << 30, o.width_area_weight);
        local_opt_sweeps(B, seed, order, none, limit, lo_iters, 0);
        return order;
    };
    auto shape = [&](int seed, std::vector<int> order, long ann) { return shape_with(seed, std::move(order), ann, rng); };
    const int start0 = ((o.start_cluster % C) + C) % C;
    if (o.stem_starts > 0) {
        // stems grown without noise from stem_starts start clusters spread
        // evenly over all clusters, each annealed, sliced and refined on its
        // own random stream (seeded by the planner seed and its start), on the
        // host's threads; the cheapest wins (ties: the earlier start), so the
        // result does not depend on the thread count
        const int n = std::min(o.stem_starts, C);
        std::vector<int> starts;
        for (int i = 0; i < n; ++i) starts.push_back((int)(((int64_t)i * C) / n));
        std::vector<Candidate> res((size_t)n);
        std::atomic<int> next{0};
        std::exception_ptr err;
        std::mutex err_mu;
        auto worker = [&]() {
            for (int i = next.fetch_add(1); i < n; i = next.fetch_add(1)) {
                try {
                    const int seed = starts[(size_t)i];
                    std::mt19937_64 r((o.seed ? o.seed : 0x5eedull) ^
                                      (0x9e3779b97f4a7c15ull * (uint64_t)(seed + 1)));
                    const std::vector<int> grown = grow_stem(B, seed, r, 0.0);
                    Candidate c;
                    if (!slice_refine_into(seed, shape_with(seed, grown, anneal, r), anneal, r, c) && anneal > 0)
                        slice_refine_into(seed, shape_with(seed, grown, 0, r), 0, r, c);
                    res[(size_t)i] = std::move(c);
                } catch (...) {
                    std::lock_guard<std::mutex> lk(err_mu);
                    if (!err) err = std::current_exception();
                }
            }
        };
        const int nth = std::max(1, std::min(n, (int)std::max(1u, std::thread::hardware_concurrency())));
        std::vector<std::thread> pool;
        for (int t = 1; t < nth; ++t) pool.emplace_back(worker);
        worker();
        for (auto &t : pool) t.join();
        if (err) std::rethrow_exception(err);
        for (const Candidate &c : res) take(c);
    } else if (o.slice_restarts <= 0 || o.slice_restarts >= restarts) {
        // every restart grows, anneals, slices and refines in turn; an annealed
        // stem can need more sliced edges than the budget allows (annealing
        // between picks keeps the width, it does not force it down), and the
        // greedy pipeline is then tried on the same grown stem
        for (int r = 0; r < restarts; ++r) {
            const int seed = (r == 0) ? start0 : pick(rng);
            const double noise = (r == 0) ? 0.0 : 0.9;
            const std::vector<int> grown = grow_stem(B, seed, rng, noise);
            if (!slice_refine(seed, shape(seed, grown, anneal), anneal) && anneal > 0)
                slice_refine(seed, shape(seed, grown, 0), 0);
        }
    } else {
        // Phase 1: every restart grows a stem and anneals its order without
        // slicing (score: log2 stem cost + one unit per bit above the width
        // limit). Phase 2: only the best slice_restarts of them are sliced and
        // refined, which costs more than phase 1, so more restarts widen the
        // search at little extra cost. (The unsliced score predicts the
        // sliced cost well when slicing removes a few bits of width; when it
        // must remove many, slice every restart.)
        struct Start {
            double score;
            int seed;
            std::vector<int> grown, order;
        };
        std::vector<Start> starts;
        for (int r = 0; r < restarts; ++r) {
            Start st;
            st.seed = (r == 0) ? start0 : pick(rng);
            const double noise = (r == 0) ? 0.0 : 0.9;
            st.grown = grow_stem(B, st.seed, rng, noise);
            st.order = shape(st.seed, st.grown, anneal);
            Bits none(net.n_edges());
            st.score = scheme_score(eval_stem(B, st.seed, st.order, none), 0, limit);
            starts.push_back(std::move(st));
        }
        std::stable_sort(starts.begin(), starts.end(),
                         [](const Start &a, const Start &b) { return a.score < b.score; });
        const int keep = std::min<int>((int)starts.size(), o.slice_restarts);
        for (int r = 0; r < keep; ++r) {
            const Start &st = starts[(size_t)r];
            if (!slice_refine(st.seed, st.order, anneal) && anneal > 0)
                slice_refine(st.seed, shape(st.seed, st.grown, 0), 0);
        }
    }
    if (best.seed_cluster < 0)
        fail(TN_ERR_PLAN_INFEASIBLE, "no scheme within the width limit and slice budget");
    evaluate_scheme(net, best);
    return best;
}

// ------------------------------------------------------------------ given order
// Convert an SSA order over the leaves into stem + branches: from the root,
// follow the child whose subtree costs more, until the subtree costs less than
// 1% of the total; the other child of each stem node is a branch.
Scheme scheme_from_order(const Network &net, const std::vector<std::pair<int, int>> &order,
                         const std::vector<int> &sliced_in, const tn_plan_opts &o) {
    const int L = net.n_leaves();
    if ((int)order.size() != L - 1) fail(TN_ERR_INVALID_ARG, "order must have n_leaves - 1 pairs");
    Scheme s;
    s.sliced = Bits(net.n_edges());
    for (int e : sliced_in) {
        if (e < 0 || e >= net.n_edges()) fail(TN_ERR_INVALID_ARG, "sliced edge out of range");
        if (net.edges[(size_t)e].open) fail(TN_ERR_INVALID_ARG, "an open edge cannot be sliced");
        if (s.sliced.test(e)) fail(TN_ERR_INVALID_ARG, "sliced edge listed twice");
        s.sliced.set(e);
        s.sliced_list.push_back(e);
    }
    const int N = 2 * L - 1;
    std::vector<int> lc((size_t)N, -1), rc((size_t)N, -1), used((size_t)N, 0);
    std::vector<Bits> out((size_t)N);
    std::vector<double> sub((size_t)N, -INFINITY);  // log2 subtree cost (sliced)
    for (int i = 0; i < L; ++i) out[(size_t)i] = leaf_bits(net, i);
    for (int k = 0; k < L - 1; ++k) {
        int a = order[(size_t)k].first, b = order[(size_t)k].second;
        int id = L + k;
        if (a < 0 || b < 0 || a >= id || b >= id || a == b || used[(size_t)a] || used[(size_t)b])
            fail(TN_ERR_INVALID_ARG, "order is not a valid SSA pair list");
        used[(size_t)a] = used[(size_t)b] = 1;
        lc[(size_t)id] = a;
        rc[(size_t)id] = b;
        out[(size_t)id] = out[(size_t)a] ^ out[(size_t)b];
        double step = (double)count_or(out[(size_t)a].andnot(s.sliced), out[(size_t)b].andnot(s.sliced));
        sub[(size_t)id] = log2_add(log2_add(sub[(size_t)a], sub[(size_t)b]), step);
    }
    const int root = N - 1;
    // collect a subtree into a cluster
    auto make_cluster = [&](int node) {
        Cluster c;
        c.out = out[(size_t)node];
        std::vector<int> stack{node}, post;
        // iterative post-order
        std::vector<std::pair<int, int>> st{{node, 0}};
        std::map<int, int> refmap;
        while (!st.empty()) {
            auto &[u, state] = st.back();
            if (u < L) {
                c.leaves.push_back(u);
                refmap[u] = u;
                st.pop_back();
                continue;
            }
            if (state == 0) {
                state = 1;
                st.push_back({lc[(size_t)u], 0});
            } else if (state == 1) {
                state = 2;
                st.push_back({rc[(size_t)u], 0});
            } else {
                c.pairs.push_back({refmap[lc[(size_t)u]], refmap[rc[(size_t)u]]});
                refmap[u] = -(int)c.pairs.size();
                st.pop_back();
            }
        }
        return c;
    };
    double total = sub[(size_t)root];
    // storage bits of a subtree kept as a pre-computed branch: its output
    // edges plus every sliced edge touching its leaves (kept as dimensions)
    std::vector<Bits> touch((size_t)N);
    for (int i = 0; i < L; ++i) touch[(size_t)i] = out[(size_t)i] & s.sliced;
    for (int k = 0; k < L - 1; ++k) {
        const int id = L + k;
        touch[(size_t)id] = touch[(size_t)lc[(size_t)id]] | touch[(size_t)rc[(size_t)id]];
    }
    auto storage_bits = [&](int v) { return count_or(out[(size_t)v], touch[(size_t)v]); };
    std::vector<int> path;  // stem nodes root -> bottom
    int u = root;
    while (u >= L) {
        double cl = sub[(size_t)lc[(size_t)u]], cr = sub[(size_t)rc[(size_t)u]];
        // the stem ends where the rest is cheap (< 1% of the cost) and small
        // enough to store as one branch
        if (sub[(size_t)u] < total + std::log2(0.01) && !path.empty() && storage_bits(u) <= 20) break;
        path.push_back(u);
        u = (cl >= cr) ? lc[(size_t)u] : rc[(size_t)u];
    }
    if (path.empty()) {
        s.clusters.push_back(make_cluster(root));
        s.seed_cluster = 0;
    } else {
        // bottom node: seed = its heavy child subtree; its other child = first branch
        std::vector<int> branches_bottom_up;
        int bottom = path.back();
        int heavy = (sub[(size_t)lc[(size_t)bottom]] >= sub[(size_t)rc[(size_t)bottom]])
                        ? lc[(size_t)bottom] : rc[(size_t)bottom];
        int light = heavy == lc[(size_t)bottom] ? rc[(size_t)bottom] : lc[(size_t)bottom];
        s.clusters.push_back(make_cluster(heavy));
        s.seed_cluster = 0;
        s.clusters.push_back(make_cluster(light));
        s.stem_order.push_back(1);
        for (int i = (int)path.size() - 2; i >= 0; --i) {
            int p = path[(size_t)i], child = path[(size_t)i + 1];
            int other = lc[(size_t)p] == child ? rc[(size_t)p] : lc[(size_t)p];
            s.clusters.push_back(make_cluster(other));
            s.stem_order.push_back((int)s.clusters.size() - 1);
        }
    }
    evaluate_scheme(net, s);
    (void)o;
    return s;
}

// Absorb cluster b into the merged branch m (b's pair list after m's, then one
// pair joining the two roots), unless the merged rank (unsliced) would exceed
// rank_cap or the two share a sliced edge (that edge would be summed inside
// the branch instead of being fixed per slice).
static bool absorb_branch(Cluster &m, const Cluster &b, const Bits &sliced, int rank_cap) {
    if ((m.out & b.out & sliced).any()) return false;
    if ((m.out ^ b.out).andnot(sliced).count() > rank_cap) return false;
    // root refs of m and b within the merged pair list
    const int base = (int)m.pairs.size();
    const int ra = m.pairs.empty() ? m.leaves[0] : -(int)m.pairs.size();
    const int rb = b.pairs.empty() ? b.leaves[0] : -((int)b.pairs.size() + base);
    for (auto p : b.pairs) {
        auto fix = [&](int r) { return r >= 0 ? r : -((-r - 1) + base + 1); };
        m.pairs.push_back({fix(p.first), fix(p.second)});
    }
    m.pairs.push_back({ra, rb});
    m.leaves.insert(m.leaves.end(), b.leaves.begin(), b.leaves.end());
    m.out ^= b.out;
    return true;
}

// Supp. A.3 "Branch merging": merge each run of `group` consecutive stem
// branches into one branch, so the stem absorbs one larger tensor at once.
// Runs stop early where absorb_branch refuses the next member.
void merge_branches(const Network &net, Scheme &s, int group, int rank_cap) {
    if (group < 2 || s.stem_order.empty()) return;
    if (rank_cap <= 0) rank_cap = 10;
    std::vector<Cluster> out;
    out.push_back(s.clusters[(size_t)s.seed_cluster]);
    std::vector<int> order;
    size_t i = 0;
    while (i < s.stem_order.size()) {
        Cluster m = s.clusters[(size_t)s.stem_order[i]];
        int members = 1;
        size_t j = i + 1;
        while (j < s.stem_order.size() && members < group &&
               absorb_branch(m, s.clusters[(size_t)s.stem_order[j]], s.sliced, rank_cap)) {
            ++members;
            ++j;
        }
        out.push_back(std::move(m));
        order.push_back((int)out.size() - 1);
        i = j;
    }
    s.clusters = std::move(out);
    s.seed_cluster = 0;
    s.stem_order = std::move(order);
    evaluate_scheme(net, s);
}

// Branch merging chosen branch by branch: join[i] != 0 puts stem branch i + 1
// into the merged branch that holds branch i (where absorb_branch allows it;
// otherwise branch i + 1 starts a new one). Returns the number of joins made.
int merge_branch_runs(const Network &net, Scheme &s, const std::vector<char> &join, int rank_cap) {
    if (s.stem_order.empty()) return 0;
    if (rank_cap <= 0) rank_cap = 10;
    std::vector<Cluster> out;
    out.push_back(s.clusters[(size_t)s.seed_cluster]);
    std::vector<int> order;
    int joined = 0;
    size_t i = 0;
    while (i < s.stem_order.size()) {
        Cluster m = s.clusters[(size_t)s.stem_order[i]];
        size_t j = i + 1;
        while (j < s.stem_order.size() && j - 1 < join.size() && join[j - 1] &&
               absorb_branch(m, s.clusters[(size_t)s.stem_order[j]], s.sliced, rank_cap)) {
            ++joined;
            ++j;
        }
        out.push_back(std::move(m));
        order.push_back((int)out.size() - 1);
        i = j;
    }
    s.clusters = std::move(out);
    s.seed_cluster = 0;
    s.stem_order = std::move(order);
    evaluate_scheme(net, s);
    return joined;
}

// SSA order over the leaves: every cluster's internal pairs, then the stem.
std::vector<std::pair<int, int>> export_order(const Network &net, const Scheme &s) {
    const int L = net.n_leaves();
    std::vector<std::pair<int, int>> order;
    std::vector<int> root_of(s.clusters.size(), -1);
    for (size_t ci = 0; ci < s.clusters.size(); ++ci) {
        const Cluster &c = s.clusters[ci];
        std::vector<int> ids;
        for (auto &p : c.pairs) {
            auto map = [&](int r) { return r >= 0 ? r : ids[(size_t)(-r - 1)]; };
            order.push_back({map(p.first), map(p.second)});
            ids.push_back(L + (int)order.size() - 1);
        }
        root_of[ci] = c.pairs.empty() ? c.leaves[0] : ids.back();
    }
    int cur = root_of[(size_t)s.seed_cluster];
    for (int c : s.stem_order) {
        order.push_back({cur, root_of[(size_t)c]});
        cur = L + (int)order.size() - 1;
    }
    return order;
}

}  // namespace tn
