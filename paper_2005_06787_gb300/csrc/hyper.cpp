// Contraction schemes of hypergraph networks (Supp. A.1 defines a tensor
// network as a multi-hypergraph; Sec. 3 names hyperedges for the diagonal
// parts of gates). A pairwise step over tensors A and B enumerates E_AB, the
// edges of A or B, and keeps E*_AB, those that are open or still held by
// another tensor: an edge that A and B share but a third tensor also holds
// stays an index of the result instead of being summed. The step costs
// 2^|E_AB| and holds 2^|E*_AB| (tc sums, cw maxes).
//
// The order is greedy (the cheapest growth 2^|E*_AB| - 2^|A| - 2^|B| among
// pairs that share an edge) or given by the caller; there is no stem and no
// slicing for these networks: they run on the GPU as a sequence of FP64
// pairwise contractions (executor.cu, hyper_contract).
#include <algorithm>
#include <cmath>
#include <random>

#include "internal.h"

namespace tn {

static HyperScheme one_scheme(const Network &net, const std::vector<std::pair<int, int>> *order,
                              std::mt19937_64 *rng, double noise) {
    const int L = net.n_leaves(), E = net.n_edges();
    if (L < 2) fail(TN_ERR_INVALID_ARG, "a network needs two or more leaves");
    std::vector<Bits> T;
    T.reserve((size_t)(2 * L));
    std::vector<int> cnt((size_t)E, 0);                      // alive tensors holding each edge
    std::vector<std::vector<int>> holders((size_t)E);        // tensors that ever held it
    std::vector<char> alive;
    Bits open(E);
    for (int e : net.open_edges) open.set(e);
    for (int i = 0; i < L; ++i) {
        Bits b(E);
        for (int e : net.leaves[(size_t)i].edges) {
            b.set(e);
            ++cnt[(size_t)e];
            holders[(size_t)e].push_back(i);
        }
        T.push_back(b);
        alive.push_back(1);
    }
    auto out_of = [&](int a, int b) {
        Bits o(E);
        for (int e : (T[(size_t)a] | T[(size_t)b]).list()) {
            const int rest = cnt[(size_t)e] - (int)T[(size_t)a].test(e) - (int)T[(size_t)b].test(e);
            if (open.test(e) || rest > 0) o.set(e);
        }
        return o;
    };
    HyperScheme hs;
    double tc = 0.0;
    auto apply = [&](int a, int b) {
        const Bits o = out_of(a, b);
        tc += std::exp2((double)count_or(T[(size_t)a], T[(size_t)b]));
        hs.cw = std::max(hs.cw, o.count());
        for (int e : (T[(size_t)a] | T[(size_t)b]).list())
            cnt[(size_t)e] -= (int)T[(size_t)a].test(e) + (int)T[(size_t)b].test(e);
        const int id = (int)T.size();
        for (int e : o.list()) {
            ++cnt[(size_t)e];
            holders[(size_t)e].push_back(id);
        }
        T.push_back(o);
        alive[(size_t)a] = alive[(size_t)b] = 0;
        alive.push_back(1);
        hs.pairs.push_back({a, b});
        hs.node_edges.push_back(o.list());
    };
    if (order) {
        if ((int)order->size() != L - 1) fail(TN_ERR_INVALID_ARG, "order must hold n_leaves - 1 pairs");
        for (auto pr : *order) {
            const int a = pr.first, b = pr.second, n = (int)T.size();
            if (a < 0 || b < 0 || a >= n || b >= n || a == b || !alive[(size_t)a] || !alive[(size_t)b])
                fail(TN_ERR_INVALID_ARG, "invalid contraction pair in order");
            apply(a, b);
        }
    } else {
        for (int step = 0; step < L - 1; ++step) {
            double best = INFINITY;
            int ba = -1, bb = -1;
            for (int e = 0; e < E; ++e) {
                if (cnt[(size_t)e] < 2) continue;
                std::vector<int> h;
                for (int x : holders[(size_t)e])
                    if (alive[(size_t)x]) h.push_back(x);
                for (size_t i = 0; i < h.size(); ++i)
                    for (size_t j = i + 1; j < h.size(); ++j) {
                        const int a = std::min(h[i], h[j]), b = std::max(h[i], h[j]);
                        double sc = std::exp2((double)out_of(a, b).count()) -
                                    std::exp2((double)T[(size_t)a].count()) -
                                    std::exp2((double)T[(size_t)b].count());
                        // restarts other than the first: noise of up to `noise`
                        // times the larger input's size
                        if (rng && noise > 0)
                            sc += noise * std::uniform_real_distribution<double>(0.0, 1.0)(*rng) *
                                  std::exp2((double)std::max(T[(size_t)a].count(), T[(size_t)b].count()));
                        if (sc < best || (sc == best && (a < ba || (a == ba && b < bb)))) {
                            best = sc;
                            ba = a;
                            bb = b;
                        }
                    }
            }
            if (ba < 0) {  // no two tensors share an edge: outer product of the first two
                for (int i = 0; i < (int)alive.size(); ++i)
                    if (alive[(size_t)i]) {
                        if (ba < 0) ba = i;
                        else if (bb < 0) bb = i;
                    }
            }
            apply(ba, bb);
        }
    }
    // the last node keeps the open edges; bit j of a layout is its j-th edge,
    // and the amplitude index has the first open qubit as its most
    // significant bit, so the open edges go in reverse
    Bits fin = T.back();
    if (!(fin == open)) fail(TN_ERR_INVALID_ARG, "the order does not leave exactly the open edges");
    hs.node_edges.back().assign(net.open_edges.rbegin(), net.open_edges.rend());
    hs.log2_tc = std::log2(tc);
    return hs;
}

HyperScheme hyper_scheme(const Network &net, const std::vector<std::pair<int, int>> *order, int restarts,
                         uint64_t seed, int cw_limit) {
    if (order) return one_scheme(net, order, nullptr, 0.0);
    // restart 0 is the plain greedy order; the others add noise to the scores;
    // the cheapest scheme within the width limit wins (else the narrowest)
    std::mt19937_64 rng(seed);
    HyperScheme best = one_scheme(net, nullptr, nullptr, 0.0);
    for (int r = 1; r < std::max(restarts, 1); ++r) {
        HyperScheme h = one_scheme(net, nullptr, &rng, 0.5);
        const bool fits = h.cw <= cw_limit, best_fits = best.cw <= cw_limit;
        if ((fits && (!best_fits || h.log2_tc < best.log2_tc)) || (!fits && !best_fits && h.cw < best.cw))
            best = std::move(h);
    }
    return best;
}

}  // namespace tn
