// Step-time cost models and the plan search that uses them.
//
// Each kernel launch of a stem batch (a fused pass, a permute, a GEMM step)
// is described by features (kind, ranks, steps fused, contracted/new bits,
// tile bits, items, log bytes, log flops, precision). Two models estimate
// its time: the plain FLOP-and-memory model (max of bytes over HBM bandwidth
// and flops over the arithmetic rate, plus launch overhead) and the learned
// MLP trained on measured launch times (mlp.cu). The search enumerates
// candidate plans (stem-growth seeds x tile size x steps per pass x branch
// merging), scores every launch of every candidate with the MLP in one
// batched GPU inference, and keeps the MLP's pick unless the FLOP-and-memory
// model rates it much worse than its own pick (then it falls back).
#include <algorithm>
#include <cmath>
#include <memory>

#include "plan.h"

namespace tn {

struct Mlp;
void mlp_predict(Mlp &m, const float *X, int rows, float *y);

// Nominal rates of this GPU for the plain model (GB300: HBM copy 6.78 TB/s as
// measured, FP32 SIMT 152 SMs x 128 lanes x 2 flops x 1.9 GHz, tensor rates
// per precision in algorithmic flops).
constexpr double HBM_BPS = 6.78e12;
constexpr double SIMT_FPS = 7.4e13;
constexpr double LAUNCH_S = 4e-6;

static double tensor_fps(tn_precision p) {
    switch (p) {
        case TN_PREC_TF32x3: return 1.1e15 / 3.0;
        case TN_PREC_BF16x3: return 2.25e15 / 3.0;
        case TN_PREC_BF16x1: return 2.25e15;
        default: return SIMT_FPS;
    }
}

int choose_batch(int max_rank, int n_sliced, int n_prefixes, int slice_batch) {
    int64_t SB = slice_batch > 0 ? slice_batch : 0;
    if (SB == 0) {
        const int64_t budget = (int64_t)1 << 27;  // entries per stem buffer (1 GiB)
        SB = std::max<int64_t>(1, budget / (((int64_t)1 << max_rank) * std::max(1, n_prefixes)));
    }
    if (n_sliced < 62) SB = std::min<int64_t>(SB, (int64_t)1 << n_sliced);
    SB = std::min<int64_t>(SB, 65535 / std::max(1, n_prefixes));
    return (int)std::max<int64_t>(SB, 1);
}

std::vector<LaunchDesc> launch_list(const StemPlan &sp, tn_exec_mode mode, int items) {
    std::vector<LaunchDesc> out;
    auto step_flops = [&](int s) {
        const ExecStep &es = sp.plain_steps[(size_t)s];
        return 8.0 * std::exp2((double)(es.r_in + es.n));
    };
    if (mode == TN_EXEC_FUSED) {
        for (const FusedItem &it : sp.fused_items) {
            LaunchDesc d{};
            d.items = items;
            if (it.kind == 0) {
                const DevPass &P = sp.fused_passes[(size_t)it.pass];
                d.kind = 0;
                d.r_in = P.r_in;
                d.r_out = P.r_out;
                d.t_in = P.t_in;
                d.t_out = P.t_out;
                double fl = 0;
                for (size_t s = 0; s < sp.step_pass.size(); ++s)
                    if (sp.step_pass[s] == it.pass) {
                        ++d.n_steps;
                        d.sum_k += sp.plain_steps[s].k;
                        d.sum_n += sp.plain_steps[s].n;
                        fl += step_flops((int)s);
                    }
                d.flops = fl * items;
                d.bytes = 8.0 * (std::exp2(P.r_in) + std::exp2(P.r_out)) * items;
            } else {
                d.kind = 1;
                d.r_in = it.r_in;
                d.r_out = it.r_out;
                d.n_steps = 1;
                d.sum_k = it.k;
                d.sum_n = it.n;
                d.flops = 8.0 * std::exp2((double)(it.r_in + it.n)) * items;
                d.bytes = 8.0 * (std::exp2(it.r_in) + std::exp2(it.r_out)) * items;
            }
            out.push_back(d);
        }
    } else {
        for (size_t i = 0; i < sp.plain_steps.size(); ++i) {
            const ExecStep &es = sp.plain_steps[i];
            const DevPass &P = sp.plain_passes[(size_t)es.permute_pass];
            LaunchDesc perm{};
            perm.kind = 2;
            perm.items = 1;
            perm.r_in = perm.r_out = P.r_in;
            perm.t_in = P.t_in;
            perm.t_out = P.t_out;
            perm.bytes = 16.0 * std::exp2(P.r_in);
            out.push_back(perm);
            LaunchDesc g{};
            g.kind = 1;
            g.items = 1;
            g.r_in = es.r_in;
            g.r_out = es.r_out;
            g.n_steps = 1;
            g.sum_k = es.k;
            g.sum_n = es.n;
            g.flops = step_flops((int)i);
            g.bytes = 8.0 * (std::exp2(es.r_in) + std::exp2(es.r_out));
            out.push_back(g);
        }
    }
    return out;
}

void launch_features(const LaunchDesc &d, tn_precision prec, float *f) {
    for (int i = 0; i < N_FEATURES; ++i) f[i] = 0.f;
    f[d.kind] = 1.f;  // 0 pass, 1 GEMM, 2 permute
    f[3] = (float)(std::log2((double)std::max(d.items, 1)) / 16.0);
    f[4] = (float)(d.r_in / 32.0);
    f[5] = (float)(d.r_out / 32.0);
    f[6] = (float)(d.n_steps / 8.0);
    f[7] = (float)(d.sum_k / 16.0);
    f[8] = (float)(d.sum_n / 16.0);
    f[9] = (float)(d.t_in / 16.0);
    f[10] = (float)(d.t_out / 16.0);
    f[11] = (float)(std::log2(std::max(d.bytes, 1.0)) / 40.0);
    f[12] = (float)(std::log2(d.flops + 1.0) / 50.0);
    if (d.kind == 1) {
        if (prec == TN_PREC_TF32x3) f[13] = 1.f;
        if (prec == TN_PREC_BF16x3) f[14] = 1.f;
        if (prec == TN_PREC_BF16x1) f[15] = 1.f;
    }
}

double flop_model_ms(const LaunchDesc &d, tn_precision prec) {
    const double rate = (d.kind == 1) ? tensor_fps(prec) : SIMT_FPS;
    return 1e3 * (std::max(d.bytes / HBM_BPS, d.flops / rate) + LAUNCH_S);
}

// ------------------------------------------------------------------ merges
// Predicted time of a whole plan: the model's time per batch of SB slices,
// times the number of batches (the MLP when given, else the plain model).
static double predicted_total_ms(const Network &net, const Scheme &s, const tn_plan_opts &o, Mlp *mlp,
                                 tn_precision prec, bool &ok) {
    ok = false;
    if (s.cw > o.cw_limit) return INFINITY;
    BuiltStem st;
    try {
        st = build_stem_plan(net, s, o);
    } catch (const Error &) {
        return INFINITY;
    }
    const int nsl = (int)s.sliced_list.size();
    const int SB = choose_batch(st.sp.max_rank, nsl, 1, o.slice_batch);
    const std::vector<LaunchDesc> ls = launch_list(st.sp, TN_EXEC_FUSED, SB);
    double ms = 0;
    if (mlp) {
        std::vector<float> X(ls.size() * N_FEATURES), y(ls.size());
        for (size_t i = 0; i < ls.size(); ++i) launch_features(ls[i], prec, &X[i * N_FEATURES]);
        mlp_predict(*mlp, X.data(), (int)ls.size(), y.data());
        for (float v : y) ms += std::exp((double)v);
    } else {
        for (const LaunchDesc &d : ls) ms += flop_model_ms(d, prec);
    }
    ok = true;
    return ms / SB * std::exp2((double)nsl);
}

// Supp. A.3 branch merging chosen branch by branch (merge_group < 0): going
// along the stem, stem branch i + 1 joins the merged branch that holds branch
// i when the model predicts the whole plan faster by more than 0.1 % (the
// merged branch is contracted once in pre-computation; the stem absorbs it
// in one step, fused into a pass when it stays small, else as a GEMM step).
Scheme choose_merges(const Network &net, const Scheme &base, const tn_plan_opts &o, Mlp *mlp,
                     tn_precision prec, int *n_joins) {
    const size_t L = base.stem_order.size();
    std::vector<char> join(L > 0 ? L - 1 : 0, 0);
    bool ok = false;
    Scheme cur = base;
    double best = predicted_total_ms(net, cur, o, mlp, prec, ok);
    int joins = 0;
    for (size_t i = 0; i + 1 < L; ++i) {
        join[i] = 1;
        Scheme trial = base;
        merge_branch_runs(net, trial, join, o.merge_rank_cap);
        const double t = predicted_total_ms(net, trial, o, mlp, prec, ok);
        if (ok && t < best * (1.0 - 1e-3)) {
            best = t;
            cur = std::move(trial);
            ++joins;
        } else {
            join[i] = 0;
        }
    }
    if (n_joins) *n_joins = joins;
    return cur;
}

// ------------------------------------------------------------------ search

struct Candidate {
    tn_plan_opts opts;
    Scheme scheme;
    BuiltStem stem;
    int items = 1;
    double slices_per_batch = 1;
    double n_slices = 1;
    std::vector<LaunchDesc> launches;
};

SearchResult plan_search(const Network &net, const tn_plan_opts &base, const tn_search_opts &so,
                         Mlp *mlp, tn_precision prec) {
    const int n_seeds = so.n_seeds > 0 ? so.n_seeds : 3;
    const std::vector<int> tiles{10, 11, 12};
    const std::vector<int> steps{2, 3, 4, 6, 8};
    const std::vector<int> merges{0, 2, 3};
    std::vector<Candidate> cands;
    for (int sd = 0; sd < n_seeds; ++sd) {
        tn_plan_opts o = base;
        o.seed = base.seed + 7919ull * (uint64_t)sd;
        Scheme sch;
        try {
            sch = plan_scheme(net, o);
        } catch (const Error &) {
            continue;  // this stem-growth seed finds no scheme within the limits
        }
        for (int mg : merges) {
            Scheme s2 = sch;
            if (mg >= 2) merge_branches(net, s2, mg, base.merge_rank_cap);
            if (s2.cw > 31) continue;
            for (int tb : tiles)
                for (int ms : steps) {
                    Candidate c;
                    c.opts = o;
                    c.opts.tile_bits = tb;
                    c.opts.max_pass_steps = ms;
                    c.opts.merge_group = mg;
                    c.scheme = s2;
                    try {
                        c.stem = build_stem_plan(net, c.scheme, c.opts);
                    } catch (const Error &) {
                        continue;
                    }
                    const int nsl = (int)c.scheme.sliced_list.size();
                    const int SB = choose_batch(c.stem.sp.max_rank, nsl, 1, base.slice_batch);
                    c.items = SB;
                    c.slices_per_batch = SB;
                    c.n_slices = std::exp2((double)nsl);
                    c.launches = launch_list(c.stem.sp, TN_EXEC_FUSED, SB);
                    cands.push_back(std::move(c));
                }
        }
    }
    if (cands.empty()) fail(TN_ERR_PLAN_INFEASIBLE, "no candidate plan");
    // FLOP-and-memory model: time per slice x slices
    std::vector<double> flop_total(cands.size()), mlp_total(cands.size(), 0.0);
    size_t rows = 0;
    for (size_t i = 0; i < cands.size(); ++i) {
        double ms = 0;
        for (auto &d : cands[i].launches) ms += flop_model_ms(d, prec);
        flop_total[i] = ms / cands[i].slices_per_batch * cands[i].n_slices;
        rows += cands[i].launches.size();
    }
    size_t flop_pick = (size_t)(std::min_element(flop_total.begin(), flop_total.end()) - flop_total.begin());
    size_t mlp_pick = flop_pick;
    if (mlp) {
        std::vector<float> X(rows * N_FEATURES), y(rows);
        size_t r = 0;
        for (auto &c : cands)
            for (auto &d : c.launches) launch_features(d, prec, &X[(r++) * N_FEATURES]);
        mlp_predict(*mlp, X.data(), (int)rows, y.data());
        r = 0;
        for (size_t i = 0; i < cands.size(); ++i) {
            double ms = 0;
            for (size_t j = 0; j < cands[i].launches.size(); ++j) ms += std::exp((double)y[r++]);
            mlp_total[i] = ms / cands[i].slices_per_batch * cands[i].n_slices;
        }
    }
    // per-branch merge choice (merge_group -1): for every stem-growth seed,
    // from its unmerged candidate the primary model (the MLP when given, else
    // the plain model) rates fastest, joins chosen one by one by that model;
    // each result joins the candidates, scored by both models
    {
        const std::vector<double> &prim = mlp ? mlp_total : flop_total;
        std::vector<size_t> best_of_seed;
        for (size_t i = 0; i < cands.size(); ++i) {
            if (cands[i].opts.merge_group != 0) continue;
            size_t k = 0;
            while (k < best_of_seed.size() && cands[best_of_seed[k]].opts.seed != cands[i].opts.seed) ++k;
            if (k == best_of_seed.size())
                best_of_seed.push_back(i);
            else if (prim[i] < prim[best_of_seed[k]])
                best_of_seed[k] = i;
        }
        for (size_t b : best_of_seed) {
            Candidate c;
            c.opts = cands[b].opts;
            c.opts.merge_group = -1;
            int joins = 0;
            c.scheme = choose_merges(net, cands[b].scheme, c.opts, mlp, prec, &joins);
            if (joins == 0) continue;  // the same plan as its unmerged candidate
            try {
                c.stem = build_stem_plan(net, c.scheme, c.opts);
            } catch (const Error &) {
                continue;
            }
            const int nsl = (int)c.scheme.sliced_list.size();
            const int SB = choose_batch(c.stem.sp.max_rank, nsl, 1, base.slice_batch);
            c.items = SB;
            c.slices_per_batch = SB;
            c.n_slices = std::exp2((double)nsl);
            c.launches = launch_list(c.stem.sp, TN_EXEC_FUSED, SB);
            double fms = 0;
            for (auto &d : c.launches) fms += flop_model_ms(d, prec);
            flop_total.push_back(fms / c.slices_per_batch * c.n_slices);
            double mms = 0;
            if (mlp) {
                std::vector<float> X(c.launches.size() * N_FEATURES), y(c.launches.size());
                for (size_t j = 0; j < c.launches.size(); ++j)
                    launch_features(c.launches[j], prec, &X[j * N_FEATURES]);
                mlp_predict(*mlp, X.data(), (int)c.launches.size(), y.data());
                for (float v : y) mms += std::exp((double)v);
            }
            mlp_total.push_back(mms / c.slices_per_batch * c.n_slices);
            rows += c.launches.size();
            cands.push_back(std::move(c));
        }
    }
    flop_pick = (size_t)(std::min_element(flop_total.begin(), flop_total.end()) - flop_total.begin());
    mlp_pick = flop_pick;
    if (mlp) mlp_pick = (size_t)(std::min_element(mlp_total.begin(), mlp_total.end()) - mlp_total.begin());
    SearchResult res;
    res.n_candidates = (int)cands.size();
    res.n_launch_rows = (int)rows;
    res.flop_opts = cands[flop_pick].opts;
    res.mlp_opts = cands[mlp_pick].opts;
    res.flop_pick_flop_ms = flop_total[flop_pick];
    res.mlp_pick_flop_ms = flop_total[mlp_pick];
    res.flop_pick_mlp_ms = mlp ? mlp_total[flop_pick] : 0;
    res.mlp_pick_mlp_ms = mlp ? mlp_total[mlp_pick] : 0;
    // the plain model checks the learned pick: beyond the allowed factor the
    // search falls back to the plain model's own pick
    const double allow = so.fallback_factor > 0 ? so.fallback_factor : 4.0;
    res.used_mlp = mlp && flop_total[mlp_pick] <= allow * flop_total[flop_pick];
    const size_t pick = res.used_mlp ? mlp_pick : flop_pick;
    res.opts = cands[pick].opts;
    res.scheme = std::move(cands[pick].scheme);
    res.stem = std::move(cands[pick].stem);
    return res;
}

}  // namespace tn
