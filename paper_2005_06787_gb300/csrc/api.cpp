// extern "C" entry points of libtnstem (declared in include/tnstem.h). Every
// call catches all exceptions and turns them into a tn_status plus a
// thread-local message.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>

#include "plan.h"

struct tn_network {
    tn::Network net;
};
struct tn_plan {
    std::unique_ptr<tn::Plan> p;
};
struct tn_mlp {
    tn::Mlp *m = nullptr;
    ~tn_mlp() { tn::mlp_destroy(m); }
};

namespace tn {
static thread_local std::string g_last_error;
void set_last_error(const std::string &m) { g_last_error = m; }
void fail(tn_status code, const std::string &msg) { throw Error{code, msg}; }
}  // namespace tn

template <class F>
static tn_status guard(F &&f) {
    try {
        f();
        tn::set_last_error("");
        return TN_OK;
    } catch (const tn::Error &e) {
        tn::set_last_error(e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        tn::set_last_error("host allocation failed");
        return TN_ERR_OOM;
    } catch (const std::exception &e) {
        tn::set_last_error(e.what());
        return TN_ERR_INVALID_ARG;
    } catch (...) {
        tn::set_last_error("unknown error");
        return TN_ERR_INVALID_ARG;
    }
}

static tn_plan_opts default_opts() {
    tn_plan_opts o{};
    o.cw_limit = 30;
    o.max_sliced = 40;
    o.restarts = 8;
    o.local_opt_iters = 4;
    o.branch_rank = 4;
    o.seed = 0x5eed;
    return o;
}

extern "C" {

const char *tn_last_error(void) { return tn::g_last_error.c_str(); }
const char *tn_version(void) { return "tnstem 0.1 (sm_103a)"; }

tn_status tn_build_network(const tn_circuit *c, const int32_t *open_qubits, int32_t n_open,
                           const uint8_t *closed_bits, tn_network **out) {
    return guard([&] {
        if (!c || !out) tn::fail(TN_ERR_INVALID_ARG, "null argument");
        auto *n = new tn_network;
        try {
            n->net = tn::build_network(*c, open_qubits, n_open, closed_bits);
        } catch (...) {
            delete n;
            throw;
        }
        *out = n;
    });
}

tn_status tn_build_hypernetwork(const tn_circuit *c, const int32_t *open_qubits, int32_t n_open,
                                const uint8_t *closed_bits, tn_network **out) {
    return guard([&] {
        if (!c || !out) tn::fail(TN_ERR_INVALID_ARG, "null argument");
        auto *n = new tn_network;
        try {
            n->net = tn::build_network(*c, open_qubits, n_open, closed_bits, true);
        } catch (...) {
            delete n;
            throw;
        }
        *out = n;
    });
}

// Calls that only the stem path offers.
static void require_stem_plan(const tn::Plan &p) {
    if (p.hyper) tn::fail(TN_ERR_UNSUPPORTED, "not available for a hypergraph plan (no stem)");
}

tn_status tn_network_info(const tn_network *net, int32_t *n_leaves, int32_t *n_edges,
                          int32_t *qubit, int32_t *segment) {
    return guard([&] {
        if (!net) tn::fail(TN_ERR_INVALID_ARG, "null network");
        if (n_leaves) *n_leaves = net->net.n_leaves();
        if (n_edges) *n_edges = net->net.n_edges();
        for (int e = 0; e < net->net.n_edges(); ++e) {
            if (qubit) qubit[e] = net->net.edges[(size_t)e].qubit;
            if (segment) segment[e] = net->net.edges[(size_t)e].segment;
        }
    });
}

tn_status tn_plan_create(tn_network *net, const int32_t *order, int32_t n_pairs,
                         const int32_t *sliced_edges, int32_t n_sliced, const tn_plan_opts *opts,
                         tn_plan **out) {
    return guard([&] {
        if (!net || !out) tn::fail(TN_ERR_INVALID_ARG, "null argument");
        tn_plan_opts o = opts ? *opts : default_opts();
        if (o.cw_limit <= 0) o.cw_limit = 30;
        if (o.cw_limit > 31) tn::fail(TN_ERR_INVALID_ARG, "cw_limit above 31");
        if (n_sliced < 0 || (n_sliced > 0 && !sliced_edges))
            tn::fail(TN_ERR_INVALID_ARG, "bad sliced-edge list");
        auto p = std::make_unique<tn::Plan>();
        p->net = net->net;
        p->opts = o;
        if (p->net.hyper) {
            if (n_sliced > 0) tn::fail(TN_ERR_UNSUPPORTED, "hypergraph plans are not sliced");
            std::vector<std::pair<int, int>> ord((size_t)std::max(n_pairs, 0));
            for (int i = 0; order && i < n_pairs; ++i) ord[(size_t)i] = {order[2 * i], order[2 * i + 1]};
            p->hs = tn::hyper_scheme(p->net, order ? &ord : nullptr, o.restarts, o.seed, o.cw_limit);
            p->hyper = true;
            if (p->hs.cw > o.cw_limit)
                tn::fail(TN_ERR_PLAN_INFEASIBLE, "hypergraph scheme wider than cw_limit (" +
                                                     std::to_string(p->hs.cw) + ")");
            auto *h = new tn_plan;
            h->p = std::move(p);
            *out = h;
            return;
        }
        if (order) {
            std::vector<std::pair<int, int>> ord((size_t)std::max(n_pairs, 0));
            for (int i = 0; i < n_pairs; ++i) ord[(size_t)i] = {order[2 * i], order[2 * i + 1]};
            std::vector<int> sl(sliced_edges, sliced_edges + n_sliced);
            p->scheme = tn::scheme_from_order(p->net, ord, sl, o);
        } else {
            if (n_sliced > 0) {
                // fixed slicing with a searched order is not offered: pass an order too
                tn::fail(TN_ERR_UNSUPPORTED, "sliced_edges without an order");
            }
            p->scheme = tn::plan_scheme(p->net, o);
        }
        if (o.merge_group >= 2) tn::merge_branches(p->net, p->scheme, o.merge_group, o.merge_rank_cap);
        if (o.merge_group < 0)
            p->scheme = tn::choose_merges(p->net, p->scheme, o, nullptr, TN_PREC_FP32_SIMT, nullptr);
        if (p->scheme.cw > 31) tn::fail(TN_ERR_PLAN_INFEASIBLE, "contraction width above 31");
        tn::BuiltStem bs = tn::build_stem_plan(p->net, p->scheme, o);
        p->sp = std::move(bs.sp);
        p->layouts = std::move(bs.layouts);
        auto *h = new tn_plan;
        h->p = std::move(p);
        *out = h;
    });
}

tn_status tn_plan_prepare(tn_plan *plan, const uint8_t *prefixes, int32_t n_prefixes,
                          void *cuda_stream) {
    return guard([&] {
        if (!plan) tn::fail(TN_ERR_INVALID_ARG, "null plan");
        if (n_prefixes < 0 || n_prefixes > 4096) tn::fail(TN_ERR_INVALID_ARG, "bad n_prefixes");
        if (n_prefixes > 0 && !prefixes) tn::fail(TN_ERR_INVALID_ARG, "null prefixes");
        if (plan->p->hyper)
            tn::hyper_prepare(*plan->p, prefixes, n_prefixes, (cudaStream_t)cuda_stream);
        else
            tn::plan_prepare(*plan->p, prefixes, n_prefixes, (cudaStream_t)cuda_stream);
    });
}

tn_status tn_plan_info(const tn_plan *plan, tn_plan_stats *out) {
    return guard([&] {
        if (!plan || !out) tn::fail(TN_ERR_INVALID_ARG, "null argument");
        const tn::Plan &p = *plan->p;
        std::memset(out, 0, sizeof(*out));
        if (p.hyper) {
            out->log2_tc = p.hs.log2_tc;
            out->stem_tc_per_slice = std::exp2(p.hs.log2_tc);
            out->cw = p.hs.cw;
            out->n_open = (int)p.net.open_edges.size();
            out->n_prefixes = p.n_prefix;
            out->batch_items = std::max(p.n_prefix, 1);
            out->device_bytes = p.device_bytes;
            return;
        }
        out->log2_tc = p.scheme.log2_tc;
        out->stem_tc_per_slice = p.scheme.stem_tc;
        out->branch_tc = p.scheme.branch_tc;
        out->cw = p.scheme.cw;
        out->n_sliced = (int)p.scheme.sliced_list.size();
        out->n_stem_steps = (int)p.scheme.stem_order.size();
        out->n_branches = (int)p.scheme.clusters.size();
        out->n_passes_fused = 0;
        for (auto &it : p.sp.fused_items) out->n_passes_fused += it.kind == 0;
        out->n_gemm_steps = 0;
        for (auto &it : p.sp.fused_items) out->n_gemm_steps += it.kind == 1;
        out->n_open = (int)p.net.open_edges.size();
        out->n_prefixes = p.n_prefix;
        out->batch_items = p.SB * std::max(p.n_prefix, 1);
        out->stem_bytes_plain = p.sp.bytes_plain;
        out->stem_bytes_fused = p.sp.bytes_fused;
        out->max_stem_elems = std::exp2((double)p.sp.max_rank);
        out->device_bytes = p.device_bytes;
        out->n_passes_cbank = 0;
        if (out->batch_items == 1)
            for (auto &it : p.sp.fused_items)
                if (it.kind == 0 && tn::pass_has_const_steps(p.sp.fused_passes[(size_t)it.pass]))
                    ++out->n_passes_cbank;
    });
}

tn_status tn_plan_export(const tn_plan *plan, int32_t *order, int32_t *sliced_edges) {
    return guard([&] {
        if (!plan) tn::fail(TN_ERR_INVALID_ARG, "null plan");
        const tn::Plan &p = *plan->p;
        if (p.hyper) {
            for (size_t i = 0; order && i < p.hs.pairs.size(); ++i) {
                order[2 * i] = p.hs.pairs[i].first;
                order[2 * i + 1] = p.hs.pairs[i].second;
            }
            return;
        }
        if (order) {
            auto ord = tn::export_order(p.net, p.scheme);
            for (size_t i = 0; i < ord.size(); ++i) {
                order[2 * i] = ord[i].first;
                order[2 * i + 1] = ord[i].second;
            }
        }
        if (sliced_edges)
            for (size_t i = 0; i < p.scheme.sliced_list.size(); ++i) sliced_edges[i] = p.scheme.sliced_list[i];
    });
}

tn_status tn_plan_steps(const tn_plan *plan, tn_step_info *out, int32_t max_steps,
                        int32_t *n_written) {
    return guard([&] {
        if (!plan) tn::fail(TN_ERR_INVALID_ARG, "null plan");
        const tn::Plan &p = *plan->p;
        require_stem_plan(p);
        const int L = (int)p.sp.plain_steps.size();
        int w = 0;
        for (int i = 0; i < L && (out && i < max_steps); ++i) {
            const tn::ExecStep &es = p.sp.plain_steps[(size_t)i];
            out[i].r_in = es.r_in;
            out[i].r_out = es.r_out;
            out[i].k = es.k;
            out[i].n = es.n;
            out[i].pass = p.sp.step_pass.empty() ? -1 : p.sp.step_pass[(size_t)i];
            out[i].gemm = p.sp.step_gemm.empty() ? 0 : p.sp.step_gemm[(size_t)i];
            out[i].pair = 0;
            if (out[i].pass >= 0 && !out[i].gemm) {
                // a pass holds a run of consecutive steps, in slot order
                int slot = 0;
                while (i - slot - 1 >= 0 && p.sp.step_pass[(size_t)(i - slot - 1)] == out[i].pass) ++slot;
                const tn::DevPass &P = p.sp.fused_passes[(size_t)out[i].pass];
                if (slot < P.n_steps) out[i].pair = P.steps[slot].pair;
            }
            ++w;
        }
        if (n_written) *n_written = out ? w : L;
    });
}

tn_status tn_contract_stem(tn_plan *plan, uint64_t slice_begin, uint64_t slice_end,
                           tn_precision prec, tn_exec_mode mode, void *cuda_stream,
                           double *amps_out, int32_t accumulate) {
    return guard([&] {
        if (!plan) tn::fail(TN_ERR_INVALID_ARG, "null plan");
        if (plan->p->hyper) {
            if ((int)prec < 0 || (int)prec > 3) tn::fail(TN_ERR_INVALID_ARG, "bad precision");
            tn::hyper_contract(*plan->p, slice_begin, slice_end, (cudaStream_t)cuda_stream, amps_out,
                               accumulate);
            return;
        }
        tn::plan_contract(*plan->p, slice_begin, slice_end, prec, mode, (cudaStream_t)cuda_stream,
                          amps_out, accumulate);
    });
}

tn_status tn_plan_profile(tn_plan *plan, uint64_t slice_begin, tn_precision prec,
                          tn_exec_mode mode, void *cuda_stream, tn_launch_record *out,
                          int32_t max_records, int32_t *n_records) {
    return guard([&] {
        if (!plan || !n_records || (max_records > 0 && !out))
            tn::fail(TN_ERR_INVALID_ARG, "null argument");
        require_stem_plan(*plan->p);
        auto recs = tn::plan_profile(*plan->p, slice_begin, prec, mode, (cudaStream_t)cuda_stream);
        int w = 0;
        for (size_t i = 0; i < recs.size() && w < max_records; ++i) out[w++] = recs[i];
        *n_records = max_records > 0 ? w : (int32_t)recs.size();
    });
}

tn_status tn_contract_stem_noalloc(tn_plan *plan, uint64_t slice_begin, uint64_t slice_end,
                                   void *cuda_stream, double *amps_out, int32_t accumulate) {
    return guard([&] {
        if (!plan) tn::fail(TN_ERR_INVALID_ARG, "null plan");
        require_stem_plan(*plan->p);
        tn::plan_contract_noalloc(*plan->p, slice_begin, slice_end, (cudaStream_t)cuda_stream,
                                  amps_out, accumulate);
    });
}

tn_status tn_plan_features(const tn_plan *plan, tn_precision prec, tn_exec_mode mode, float *X,
                           double *flop_ms, int32_t max_rows, int32_t *n_rows) {
    return guard([&] {
        if (!plan || !n_rows) tn::fail(TN_ERR_INVALID_ARG, "null argument");
        const tn::Plan &p = *plan->p;
        require_stem_plan(p);
        const int nsl = (int)p.scheme.sliced_list.size();
        const int npre = std::max(p.n_prefix, 1);
        const int items = mode == TN_EXEC_FUSED
                              ? (p.prepared ? p.SB : tn::choose_batch(p.sp.max_rank, nsl, npre, p.opts.slice_batch)) * npre
                              : 1;
        auto L = tn::launch_list(p.sp, mode, items);
        int w = 0;
        for (size_t i = 0; i < L.size() && w < max_rows; ++i, ++w) {
            if (X) tn::launch_features(L[i], prec, X + (size_t)w * tn::N_FEATURES);
            if (flop_ms) flop_ms[w] = tn::flop_model_ms(L[i], prec);
        }
        *n_rows = max_rows > 0 ? w : (int32_t)L.size();
    });
}

tn_status tn_mlp_create(int32_t n_in, int32_t h1, int32_t h2, uint64_t seed, tn_mlp **out) {
    return guard([&] {
        if (!out) tn::fail(TN_ERR_INVALID_ARG, "null argument");
        auto *h = new tn_mlp;
        try {
            h->m = tn::mlp_create(n_in, h1, h2, seed);
        } catch (...) {
            delete h;
            throw;
        }
        *out = h;
    });
}
tn_status tn_mlp_n_params(const tn_mlp *m, int64_t *n) {
    return guard([&] {
        if (!m || !n) tn::fail(TN_ERR_INVALID_ARG, "null argument");
        *n = tn::mlp_n_params(*m->m);
    });
}
tn_status tn_mlp_set_params(tn_mlp *m, const float *params, int64_t n) {
    return guard([&] {
        if (!m || !params) tn::fail(TN_ERR_INVALID_ARG, "null argument");
        tn::mlp_set_params(*m->m, params, n);
    });
}
tn_status tn_mlp_get_params(const tn_mlp *m, float *params, int64_t n) {
    return guard([&] {
        if (!m || !params) tn::fail(TN_ERR_INVALID_ARG, "null argument");
        tn::mlp_get_params(*m->m, params, n);
    });
}
tn_status tn_mlp_loss_grad(tn_mlp *m, const float *X, const float *t, int32_t rows, double *loss,
                           float *grad) {
    return guard([&] {
        if (!m || !X || !t || !loss) tn::fail(TN_ERR_INVALID_ARG, "null argument");
        tn::mlp_loss_grad_host(*m->m, X, t, rows, loss, grad);
    });
}
tn_status tn_mlp_train(tn_mlp *m, const float *X, const float *t, int32_t rows, int32_t epochs,
                       int32_t batch, float lr, uint64_t seed, double *final_loss) {
    return guard([&] {
        if (!m || !X || !t) tn::fail(TN_ERR_INVALID_ARG, "null argument");
        const double l = tn::mlp_train(*m->m, X, t, rows, epochs, batch, lr, seed);
        if (final_loss) *final_loss = l;
    });
}
tn_status tn_mlp_predict(tn_mlp *m, const float *X, int32_t rows, float *y) {
    return guard([&] {
        if (!m || !X || !y || rows < 0) tn::fail(TN_ERR_INVALID_ARG, "bad argument");
        tn::mlp_predict(*m->m, X, rows, y);
    });
}
void tn_mlp_destroy(tn_mlp *m) { delete m; }

tn_status tn_plan_search(tn_network *net, const tn_plan_opts *base, const tn_search_opts *so,
                         tn_mlp *mlp, tn_precision prec, tn_plan **out, tn_search_report *report) {
    return guard([&] {
        if (!net || !out) tn::fail(TN_ERR_INVALID_ARG, "null argument");
        if (net->net.hyper) tn::fail(TN_ERR_UNSUPPORTED, "plan search needs a graph network (stem plans)");
        tn_plan_opts o = base ? *base : default_opts();
        if (o.cw_limit <= 0) o.cw_limit = 30;
        tn_search_opts s{};
        if (so) s = *so;
        tn::SearchResult r = tn::plan_search(net->net, o, s, mlp ? mlp->m : nullptr, prec);
        auto p = std::make_unique<tn::Plan>();
        p->net = net->net;
        p->opts = r.opts;
        p->scheme = std::move(r.scheme);
        p->sp = std::move(r.stem.sp);
        p->layouts = std::move(r.stem.layouts);
        if (report) {
            report->n_candidates = r.n_candidates;
            report->n_launch_rows = r.n_launch_rows;
            report->used_mlp = r.used_mlp ? 1 : 0;
            report->chosen = r.opts;
            report->mlp_pick = r.mlp_opts;
            report->flop_pick = r.flop_opts;
            report->mlp_pick_mlp_ms = r.mlp_pick_mlp_ms;
            report->mlp_pick_flop_ms = r.mlp_pick_flop_ms;
            report->flop_pick_mlp_ms = r.flop_pick_mlp_ms;
            report->flop_pick_flop_ms = r.flop_pick_flop_ms;
        }
        auto *h = new tn_plan;
        h->p = std::move(p);
        *out = h;
    });
}

void tn_plan_destroy(tn_plan *plan) { delete plan; }
void tn_network_destroy(tn_network *net) { delete net; }
void tn_destroy_plan(tn_plan *plan) { delete plan; }
void tn_destroy_network(tn_network *net) { delete net; }

tn_status tn_set_prefix(tn_network *net, const uint8_t *closed_bits) {
    return guard([&] {
        if (!net) tn::fail(TN_ERR_INVALID_ARG, "null network");
        tn::set_prefix(net->net, closed_bits);
    });
}

tn_status tn_device_status(void) {
    return guard([&] {
        TN_CUDA(cudaDeviceSynchronize());
        int tc_flag = 0;
        TN_CUDA(tn::tc_error_flag(&tc_flag));
        if (tc_flag) tn::fail(TN_ERR_TIMEOUT, "a tensor-core GEMM wait timed out");
    });
}

tn_status tn_fp32_fma_peak(void *cuda_stream, double *tflops, int32_t *sm_count) {
    return guard([&] {
        if (!tflops || !sm_count) tn::fail(TN_ERR_INVALID_ARG, "null output");
        int sms = 0;
        TN_CUDA(tn::measure_fma_peak((cudaStream_t)cuda_stream, tflops, &sms));
        *sm_count = sms;
    });
}

tn_status tn_frugal_sample(const double *amps_dev, const double *u_dev, const double *key_dev,
                           int64_t n_batches, int32_t batch_size, int32_t n_qubits, double M,
                           void *cuda_stream, int32_t *index_dev, int32_t *accepted_dev,
                           double *picked_dev) {
    return guard([&] {
        if (n_batches < 0 || batch_size < 1 || batch_size > (1 << 20) || n_qubits < 1 ||
            n_qubits > 1000 || !(M > 0.0) || !std::isfinite(M))
            tn::fail(TN_ERR_INVALID_ARG, "bad sampling size or threshold");
        if (n_batches == 0) return;
        const void *ptrs[] = {amps_dev, u_dev, key_dev, index_dev, accepted_dev, picked_dev};
        for (const void *q : ptrs) {
            cudaPointerAttributes a{};
            if (!q || cudaPointerGetAttributes(&a, q) != cudaSuccess ||
                (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
                cudaGetLastError();
                tn::fail(TN_ERR_INVALID_ARG, "sampling buffers must be device memory");
            }
        }
        TN_CUDA(tn::launch_frugal_sample(reinterpret_cast<const double2 *>(amps_dev), u_dev, key_dev,
                                         n_batches, batch_size, n_qubits, M, index_dev, accepted_dev,
                                         reinterpret_cast<double2 *>(picked_dev),
                                         (cudaStream_t)cuda_stream));
    });
}

tn_status tn_linear_xeb(const double *amps_dev, int64_t count, int32_t n_qubits,
                        void *cuda_stream, double *out) {
    return guard([&] {
        if (!amps_dev || !out || count <= 0 || n_qubits <= 0 || n_qubits > 1000)
            tn::fail(TN_ERR_INVALID_ARG, "bad argument");
        cudaStream_t st = (cudaStream_t)cuda_stream;
        double *tmp = nullptr;
        TN_CUDA(cudaMallocAsync((void **)&tmp, 257 * sizeof(double), st));
        cudaError_t e = tn::launch_xeb_sum(reinterpret_cast<const double2 *>(amps_dev), count, tmp, st);
        double sum = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&sum, tmp, sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaFreeAsync(tmp, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        TN_CUDA(e);
        *out = std::exp2((double)n_qubits) * sum / (double)count - 1.0;
    });
}

tn_status tn_permute(const float *in, float *out, int32_t rank, const int32_t *perm,
                     void *cuda_stream) {
    return guard([&] {
        if (!in || !out || !perm || rank < 0 || rank > 31) tn::fail(TN_ERR_INVALID_ARG, "bad argument");
        std::vector<int> seen((size_t)std::max(rank, 1), 0);
        for (int j = 0; j < rank; ++j) {
            if (perm[j] < 0 || perm[j] >= rank || seen[(size_t)perm[j]]++)
                tn::fail(TN_ERR_INVALID_ARG, "perm is not a permutation");
        }
        cudaStream_t st = (cudaStream_t)cuda_stream;
        if (rank >= 4 && !(((uintptr_t)in | (uintptr_t)out) & 15)) {
            // tiles of 128-byte chunks through shared memory (the fused pass
            // kernel with no stem step): coalesced 16-byte reads and writes,
            // which need 16-byte aligned tensors
            std::vector<int> chunks;
            const tn::DevPass P = tn::make_permute_pass(rank, std::vector<int>(perm, perm + rank), chunks);
            TN_CUDA(tn::init_kernels());
            unsigned char *d = nullptr;
            const size_t cb = (chunks.size() * sizeof(int) + 255) & ~(size_t)255;
            TN_CUDA(cudaMallocAsync((void **)&d, sizeof(tn::DevPass) + cb + sizeof(tn::DevState), st));
            auto *d_pass = reinterpret_cast<tn::DevPass *>(d);
            auto *d_chunks = reinterpret_cast<int *>(d + sizeof(tn::DevPass));
            auto *d_state = reinterpret_cast<tn::DevState *>(d + sizeof(tn::DevPass) + cb);
            const tn::DevState h_state{0, 1, 0, 0};
            cudaError_t e = cudaMemcpyAsync(d_pass, &P, sizeof(P), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d_chunks, chunks.data(), chunks.size() * sizeof(int), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d_state, &h_state, sizeof(h_state), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = tn::launch_pass(d_pass, P, d_chunks, nullptr, nullptr, nullptr,
                                    reinterpret_cast<const float2 *>(in), reinterpret_cast<float2 *>(out),
                                    tn::BatchArgs{d_state, 1, 1, 0}, st);
            cudaFreeAsync(d, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            TN_CUDA(e);
            return;
        }
        std::vector<int> tab(4 * 256, 0);
        for (int b = 0; b < 4; ++b)
            for (int v = 0; v < 256; ++v) {
                uint32_t o = 0;
                for (int t = 0; t < 8; ++t) {
                    int j = 8 * b + t;
                    if (j < rank && ((v >> t) & 1)) o |= 1u << perm[j];
                }
                tab[(size_t)(b * 256 + v)] = (int)o;
            }
        int *d_tab = nullptr;
        TN_CUDA(cudaMallocAsync((void **)&d_tab, tab.size() * sizeof(int), st));
        cudaError_t e = cudaMemcpyAsync(d_tab, tab.data(), tab.size() * sizeof(int),
                                        cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = tn::launch_permute(reinterpret_cast<const float2 *>(in), reinterpret_cast<float2 *>(out),
                                   rank, d_tab, st);
        cudaFreeAsync(d_tab, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        TN_CUDA(e);
    });
}

tn_status tn_cgemm(const float *A, const float *B, float *C, int64_t M, int64_t K, int64_t N,
                   int64_t batch, int64_t strideA, int64_t strideB, int64_t strideC,
                   tn_precision prec, void *cuda_stream) {
    return guard([&] {
        if (!A || !B || !C || M < 0 || K <= 0 || N <= 0 || batch < 0)
            tn::fail(TN_ERR_INVALID_ARG, "bad argument");
        if ((int)prec < 0 || (int)prec > 3) tn::fail(TN_ERR_INVALID_ARG, "bad precision");
        TN_CUDA(tn::init_kernels());
        TN_CUDA(tn::launch_cgemm(reinterpret_cast<const float2 *>(A), reinterpret_cast<const float2 *>(B),
                                 reinterpret_cast<float2 *>(C), M, K, N, batch, strideA, strideB,
                                 strideC, prec, (cudaStream_t)cuda_stream));
    });
}

}  // extern "C"
