// Executor: device resources of a plan, branch pre-computation (Supp. A.3)
// and the slice loop (Supp. A.1 "Slicing": subtasks share one structure and
// their values are summed).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>

#include "plan.h"

namespace tn {

Plan::~Plan() { release(); }

void Plan::release() {
    for (auto &g : graphs) cudaGraphExecDestroy(g.second);
    graphs.clear();
    if (graph_stream) cudaStreamDestroy(graph_stream);
    graph_stream = nullptr;
    void *ptrs[] = {d_pool, d_branches, d_plain, d_fused, d_chunks, d_buf[0], d_buf[1],
                    d_state, d_sum, d_comp, d_out, d_pos_plain, d_pos_fused, d_hleaf};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    d_pool = nullptr;
    d_branches = nullptr;
    d_plain = d_fused = nullptr;
    d_chunks = nullptr;
    d_buf[0] = d_buf[1] = nullptr;
    d_state = nullptr;
    d_sum = d_comp = d_out = nullptr;
    d_pos_plain = d_pos_fused = nullptr;
    d_hleaf = nullptr;
    device_bytes = 0;
    prepared = false;
}

template <class T>
static T *dev_alloc(Plan &p, size_t count) {
    void *ptr = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    TN_CUDA(cudaMalloc(&ptr, bytes));
    p.device_bytes += (int64_t)bytes;
    return reinterpret_cast<T *>(ptr);
}

// Descriptor of one pairwise step out[lay_c] = sum A[lay_a] * B[lay_b].
static SmallContract make_contract(const std::vector<int> &la, const std::vector<int> &lb,
                                   const std::vector<int> &lc) {
    SmallContract d{};
    d.ra = (int)la.size();
    d.rb = (int)lb.size();
    d.rc = (int)lc.size();
    if (d.ra > 40 || d.rb > 40 || d.rc > 40) fail(TN_ERR_UNSUPPORTED, "branch tensor too large");
    auto pos = [](const std::vector<int> &l, int e) {
        for (size_t i = 0; i < l.size(); ++i)
            if (l[i] == e) return (int)i;
        return -1;
    };
    // an output edge comes from A, from B, or from both (a batch edge: a
    // sliced edge shared by the two, indexed in both and not summed)
    int batch = 0;
    for (int j = 0; j < d.rc; ++j) {
        d.a_out[j] = pos(la, lc[(size_t)j]);
        d.b_out[j] = pos(lb, lc[(size_t)j]);
        if (d.a_out[j] < 0 && d.b_out[j] < 0)
            fail(TN_ERR_INVALID_ARG, "internal: output edge in neither input");
        if (d.a_out[j] >= 0 && d.b_out[j] >= 0) ++batch;
    }
    d.k = 0;
    for (int i = 0; i < d.ra; ++i) {
        int pb = pos(lb, la[(size_t)i]);
        if (pb >= 0 && pos(lc, la[(size_t)i]) < 0) {
            d.a_k[d.k] = i;
            d.b_k[d.k] = pb;
            d.k++;
        }
    }
    if (d.ra + d.rb - 2 * d.k - batch != d.rc)
        fail(TN_ERR_INVALID_ARG, "internal: edge count mismatch");
    return d;
}

void plan_prepare(Plan &p, const uint8_t *prefixes, int n_prefixes, cudaStream_t st) {
    const Network &net = p.net;
    const int n_closed = (int)net.closed_qubits.size();
    if (n_prefixes <= 0) {
        prefixes = nullptr;
        n_prefixes = 1;
    }
    std::vector<uint8_t> pre((size_t)n_prefixes * n_closed);
    for (int i = 0; i < n_prefixes; ++i)
        for (int j = 0; j < n_closed; ++j) {
            uint8_t b = prefixes ? prefixes[(size_t)i * n_closed + j] : net.closed_bits[(size_t)j];
            if (b > 1) fail(TN_ERR_INVALID_ARG, "prefix bits must be 0 or 1");
            pre[(size_t)i * n_closed + j] = b;
        }
    p.release();
    TN_CUDA(init_kernels());
    TN_CUDA(cudaGetDevice(&p.device));
    p.n_prefix = n_prefixes;

    // ---- leaf values per prefix (complex64), offsets per leaf
    const int L = net.n_leaves();
    std::vector<int64_t> leaf_off((size_t)L);
    int64_t leaf_total = 0;
    for (int i = 0; i < L; ++i) {
        leaf_off[(size_t)i] = leaf_total;
        leaf_total += (int64_t)net.leaves[(size_t)i].vals.size();
        leaf_total = (leaf_total + 1) & ~1ll;
    }
    // leaves and branch intermediates stay in FP64; each branch is rounded to
    // FP32 once, when it is stored (rounding every gate separately would bias
    // the result: 1/sqrt(2) rounds the same way in every single-qubit gate)
    std::vector<double2> h_leaf((size_t)(leaf_total * n_prefixes));
    for (int pp = 0; pp < n_prefixes; ++pp)
        for (int i = 0; i < L; ++i) {
            const Leaf &lf = net.leaves[(size_t)i];
            for (size_t v = 0; v < lf.vals.size(); ++v) {
                cd x = lf.vals[v];
                if (lf.kind == LEAF_PROJ) {
                    int b = pre[(size_t)pp * n_closed + lf.gate];
                    x = (v == (size_t)b) ? 1.0 : 0.0;
                }
                h_leaf[(size_t)(pp * leaf_total + leaf_off[(size_t)i] + (int64_t)v)] =
                    make_double2(x.real(), x.imag());
            }
        }
    double2 *d_leaf = nullptr;
    TN_CUDA(cudaMalloc(&d_leaf, h_leaf.size() * sizeof(double2)));
    TN_CUDA(cudaMemcpyAsync(d_leaf, h_leaf.data(), h_leaf.size() * sizeof(double2),
                            cudaMemcpyHostToDevice, st));

    // ---- branch pool layout
    const int C = (int)p.scheme.clusters.size();
    p.h_branches.assign((size_t)C, DevBranch{});
    int64_t pool = 0;
    for (int c = 0; c < C; ++c) {
        const BranchLayout &bl = p.layouts[(size_t)c];
        DevBranch &d = p.h_branches[(size_t)c];
        const int64_t sz = (int64_t)1 << bl.bits.size();
        d.base = pool;
        d.prefix_stride = bl.prefix_dependent ? sz : 0;
        d.k = bl.k;
        d.n = bl.n;
        d.n_sl = (int)bl.sliced_edges.size();
        for (int i = 0; i < d.n_sl; ++i) {
            int e = bl.sliced_edges[(size_t)i];
            d.sl_bit[i] = (int)(std::find(p.scheme.sliced_list.begin(), p.scheme.sliced_list.end(), e) -
                                p.scheme.sliced_list.begin());
            d.sl_pos[i] = (int)bl.bits.size() - d.n_sl + i;
        }
        const int64_t copies = bl.prefix_dependent ? n_prefixes : 1;
        pool += ((sz * copies) + 63) & ~63ll;
    }
    p.pool_elems = pool;
    if (pool > ((int64_t)1 << 33))
        fail(TN_ERR_UNSUPPORTED, "pre-computed branches would exceed 64 GiB (a branch keeps too many "
                                 "sliced edges as dimensions)");
    // every branch read stays inside the pool: last prefix copy, all sliced
    // bits set, a full 2^(k+n) matrix (or the whole seed tensor)
    for (int c = 0; c < C; ++c) {
        const DevBranch &d = p.h_branches[(size_t)c];
        const BranchLayout &bl = p.layouts[(size_t)c];
        int64_t last = d.base + (bl.prefix_dependent ? (int64_t)(n_prefixes - 1) * d.prefix_stride : 0);
        for (int i = 0; i < d.n_sl; ++i) last += (int64_t)1 << d.sl_pos[i];
        last += ((int64_t)1 << (bl.bits.size() - (size_t)d.n_sl)) - 1;
        if (last >= pool || d.k + d.n + d.n_sl != (int)bl.bits.size() && c != p.scheme.seed_cluster)
            fail(TN_ERR_UNSUPPORTED, "internal: branch storage bounds");
        for (int i = 0; i < d.n_sl; ++i)
            if (d.sl_bit[i] < 0 || d.sl_bit[i] >= (int)p.scheme.sliced_list.size())
                fail(TN_ERR_UNSUPPORTED, "internal: branch slice bit");
    }
    p.d_pool = dev_alloc<float2>(p, (size_t)pool);

    // ---- pre-compute each cluster (per prefix when it holds a projector)
    // scratch: the largest sum of intermediate sizes of one cluster
    auto leaf_layout = [&](int leaf) { return net.leaves[(size_t)leaf].edges; };
    const Bits &sliced = p.scheme.sliced;
    int64_t scratch_need = 0;
    std::vector<std::vector<std::vector<int>>> node_layouts((size_t)C);
    for (int c = 0; c < C; ++c) {
        const Cluster &cl = p.scheme.clusters[(size_t)c];
        std::vector<std::vector<int>> lays;
        int64_t need = 0;
        auto lay_of = [&](int ref) -> std::vector<int> {
            return ref >= 0 ? leaf_layout(ref) : lays[(size_t)(-ref - 1)];
        };
        for (size_t k = 0; k < cl.pairs.size(); ++k) {
            std::vector<int> la = lay_of(cl.pairs[k].first), lb = lay_of(cl.pairs[k].second);
            std::vector<int> lc;
            if (k + 1 == cl.pairs.size()) {
                lc = p.layouts[(size_t)c].bits;
            } else {
                // shared edges are summed, except sliced ones (kept as batch dims)
                for (int e : la)
                    if (std::find(lb.begin(), lb.end(), e) == lb.end() || sliced.test(e))
                        lc.push_back(e);
                for (int e : lb)
                    if (std::find(la.begin(), la.end(), e) == la.end()) lc.push_back(e);
            }
            if (lc.size() > 34) fail(TN_ERR_UNSUPPORTED, "branch intermediate above 2^34 entries");
            lays.push_back(lc);
            if (k + 1 < cl.pairs.size()) need += (((int64_t)1 << lc.size()) + 63) & ~63ll;
        }
        node_layouts[(size_t)c] = lays;
        scratch_need = std::max(scratch_need, need);
    }
    double2 *d_scratch = nullptr;
    TN_CUDA(cudaMalloc(&d_scratch, (size_t)std::max<int64_t>(scratch_need, 64) * sizeof(double2)));
    for (int c = 0; c < C; ++c) {
        const Cluster &cl = p.scheme.clusters[(size_t)c];
        const BranchLayout &bl = p.layouts[(size_t)c];
        const int copies = bl.prefix_dependent ? n_prefixes : 1;
        const auto &lays = node_layouts[(size_t)c];
        for (int pp = 0; pp < copies; ++pp) {
            float2 *dst = p.d_pool + p.h_branches[(size_t)c].base +
                          (int64_t)pp * p.h_branches[(size_t)c].prefix_stride;
            const double2 *leafbase = d_leaf + (int64_t)pp * leaf_total;
            if (cl.pairs.empty()) {
                int leaf = cl.leaves[0];
                SmallContract d = make_contract(leaf_layout(leaf), {}, bl.bits);
                TN_CUDA(launch_small_contract(leafbase + leaf_off[(size_t)leaf], nullptr, nullptr, dst,
                                              d, st));
                continue;
            }
            std::vector<const double2 *> node_ptr;
            int64_t off = 0;
            for (size_t k = 0; k < cl.pairs.size(); ++k) {
                auto ptr_of = [&](int ref) -> const double2 * {
                    return ref >= 0 ? leafbase + leaf_off[(size_t)ref] : node_ptr[(size_t)(-ref - 1)];
                };
                auto lay_of = [&](int ref) -> std::vector<int> {
                    return ref >= 0 ? leaf_layout(ref) : lays[(size_t)(-ref - 1)];
                };
                const auto &pr = cl.pairs[k];
                const bool last = k + 1 == cl.pairs.size();
                double2 *out = nullptr;
                if (!last) {
                    out = d_scratch + off;
                    off += (((int64_t)1 << lays[k].size()) + 63) & ~63ll;
                }
                SmallContract d = make_contract(lay_of(pr.first), lay_of(pr.second), lays[k]);
                TN_CUDA(launch_small_contract(ptr_of(pr.first), ptr_of(pr.second), out,
                                              last ? dst : nullptr, d, st));
                node_ptr.push_back(out);
            }
        }
    }
    TN_CUDA(cudaStreamSynchronize(st));
    cudaFree(d_scratch);
    cudaFree(d_leaf);

    // ---- descriptors
    p.d_branches = dev_alloc<DevBranch>(p, (size_t)C);
    TN_CUDA(cudaMemcpy(p.d_branches, p.h_branches.data(), sizeof(DevBranch) * (size_t)C,
                       cudaMemcpyHostToDevice));
    p.d_plain = dev_alloc<DevPass>(p, p.sp.plain_passes.size());
    TN_CUDA(cudaMemcpy(p.d_plain, p.sp.plain_passes.data(),
                       sizeof(DevPass) * p.sp.plain_passes.size(), cudaMemcpyHostToDevice));
    p.d_fused = dev_alloc<DevPass>(p, p.sp.fused_passes.size());
    TN_CUDA(cudaMemcpy(p.d_fused, p.sp.fused_passes.data(),
                       sizeof(DevPass) * p.sp.fused_passes.size(), cudaMemcpyHostToDevice));
    p.d_chunks = dev_alloc<int>(p, p.sp.chunk_table.size());
    TN_CUDA(cudaMemcpy(p.d_chunks, p.sp.chunk_table.data(), sizeof(int) * p.sp.chunk_table.size(),
                       cudaMemcpyHostToDevice));

    // ---- stem buffers: fused batches hold n_prefix * SB items
    const int maxr = p.sp.max_rank;
    const int nsl = (int)p.scheme.sliced_list.size();
    const int64_t SB = choose_batch(maxr, nsl, n_prefixes, p.opts.slice_batch);
    p.SB = (int)SB;
    const int64_t items = SB * n_prefixes;
    p.buf_elems = std::max<int64_t>(items << maxr, (int64_t)1 << maxr);
    p.d_buf[0] = dev_alloc<float2>(p, (size_t)p.buf_elems);
    p.d_buf[1] = dev_alloc<float2>(p, (size_t)p.buf_elems);

    const int nb = 1 << (int)net.open_edges.size();
    p.d_state = dev_alloc<DevState>(p, 1);
    p.d_sum = dev_alloc<double2>(p, (size_t)n_prefixes * nb);
    p.d_comp = dev_alloc<double2>(p, (size_t)n_prefixes * nb);
    p.d_out = dev_alloc<double2>(p, (size_t)n_prefixes * nb);
    auto positions = [&](const std::vector<int> &lay) {
        std::vector<int> pos;
        for (int e : net.open_edges)
            pos.push_back((int)(std::find(lay.begin(), lay.end(), e) - lay.begin()));
        if (pos.empty()) pos.push_back(0);
        return pos;
    };
    std::vector<int> pp = positions(p.sp.final_layout_plain), pf = positions(p.sp.final_layout_fused);
    p.d_pos_plain = dev_alloc<int>(p, pp.size());
    p.d_pos_fused = dev_alloc<int>(p, pf.size());
    TN_CUDA(cudaMemcpy(p.d_pos_plain, pp.data(), sizeof(int) * pp.size(), cudaMemcpyHostToDevice));
    TN_CUDA(cudaMemcpy(p.d_pos_fused, pf.data(), sizeof(int) * pf.size(), cudaMemcpyHostToDevice));
    TN_CUDA(cudaStreamCreateWithFlags(&p.graph_stream, cudaStreamNonBlocking));
    p.prepared = true;
}

// Enqueue one fused batch: passes / GEMM steps, accumulation, advance.
static void enqueue_fused_batch(Plan &p, tn_precision prec, cudaStream_t st) {
    const int items = p.SB * p.n_prefix;
    BatchArgs ba{p.d_state, p.SB, items, 0};
    int cur = -1;  // -1: seed branch storage
    for (const FusedItem &it : p.sp.fused_items) {
        const float2 *in = cur < 0 ? nullptr : p.d_buf[cur];
        const int nxt = cur < 0 ? 0 : 1 - cur;
        if (it.kind == 0) {
            TN_CUDA(launch_pass(p.d_fused + it.pass, p.sp.fused_passes[(size_t)it.pass], p.d_chunks,
                                p.d_branches, p.h_branches.data(), p.d_pool, in, p.d_buf[nxt], ba, st));
        } else {
            TN_CUDA(launch_stem_gemm(p.d_buf[cur], p.d_buf[nxt], it.M, it.k, it.n,
                                     (int64_t)1 << it.r_in, (int64_t)1 << it.r_out,
                                     p.d_branches + it.branch, p.d_pool, ba, prec, st));
        }
        cur = nxt;
    }
    TN_CUDA(launch_accumulate(p.d_buf[cur], (int)p.net.open_edges.size(), p.d_pos_fused, p.d_sum,
                              p.d_comp, ba, p.n_prefix, st));
    TN_CUDA(launch_advance(p.d_state, p.SB, st));
}

// Enqueue one plain slice for prefix pp: per step a permute then a GEMM.
static void enqueue_plain_item(Plan &p, int pp, cudaStream_t st) {
    BatchArgs ba{p.d_state, 1, 1, pp};
    int cur = -1;
    if (p.sp.plain_steps.empty()) {
        TN_CUDA(launch_pass(p.d_plain, p.sp.plain_passes[0], p.d_chunks, p.d_branches,
                            p.h_branches.data(), p.d_pool, nullptr, p.d_buf[0], ba, st));
        cur = 0;
    }
    for (const ExecStep &es : p.sp.plain_steps) {
        const float2 *in = cur < 0 ? nullptr : p.d_buf[cur];
        const int mid = cur < 0 ? 0 : 1 - cur;
        TN_CUDA(launch_pass(p.d_plain + es.permute_pass, p.sp.plain_passes[(size_t)es.permute_pass],
                            p.d_chunks, p.d_branches, p.h_branches.data(), p.d_pool, in, p.d_buf[mid],
                            ba, st));
        const int out = 1 - mid;
        TN_CUDA(launch_stem_gemm(p.d_buf[mid], p.d_buf[out], es.M, es.k, es.n, (int64_t)1 << es.r_in,
                                 (int64_t)1 << es.r_out, p.d_branches + es.branch, p.d_pool, ba,
                                 TN_PREC_FP32_SIMT, st));
        cur = out;
    }
    TN_CUDA(launch_accumulate(p.d_buf[cur], (int)p.net.open_edges.size(), p.d_pos_plain, p.d_sum,
                              p.d_comp, ba, 1, st));
}

void require_plan_device(const Plan &p) {
    if (!p.prepared) fail(TN_ERR_INVALID_ARG, "plan not prepared (call tn_plan_prepare)");
    int dev = -1;
    TN_CUDA(cudaGetDevice(&dev));
    if (dev != p.device)
        fail(TN_ERR_INVALID_ARG, "the current CUDA device is " + std::to_string(dev) +
                                     ", but the plan was prepared on device " + std::to_string(p.device));
}

static bool is_device_pointer(const void *ptr) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void plan_contract(Plan &p, uint64_t s0, uint64_t s1, tn_precision prec, tn_exec_mode mode,
                   cudaStream_t st, double *amps_out, int accumulate) {
    require_plan_device(p);
    const int nsl = (int)p.scheme.sliced_list.size();
    const uint64_t total = nsl >= 63 ? ~0ull : (1ull << nsl);
    if (s0 > s1 || s1 > total) fail(TN_ERR_INVALID_ARG, "slice range outside [0, 2^n_sliced]");
    if (!amps_out) fail(TN_ERR_INVALID_ARG, "amps_out is null");
    if ((int)prec < 0 || (int)prec > 3) fail(TN_ERR_INVALID_ARG, "bad precision");
    if (mode != TN_EXEC_PLAIN && mode != TN_EXEC_FUSED) fail(TN_ERR_INVALID_ARG, "bad mode");
    const int nb = 1 << (int)p.net.open_edges.size();
    const int64_t nout = (int64_t)p.n_prefix * nb;
    TN_CUDA(cudaMemsetAsync(p.d_sum, 0, sizeof(double2) * (size_t)nout, st));
    TN_CUDA(cudaMemsetAsync(p.d_comp, 0, sizeof(double2) * (size_t)nout, st));
    DevState h{(int64_t)s0, (int64_t)s1, 0, 0};
    TN_CUDA(cudaMemcpyAsync(p.d_state, &h, sizeof(h), cudaMemcpyHostToDevice, st));
    if (s1 > s0) {
        if (mode == TN_EXEC_PLAIN) {
            for (uint64_t s = s0; s < s1; ++s) {
                for (int pp = 0; pp < p.n_prefix; ++pp) enqueue_plain_item(p, pp, st);
                TN_CUDA(launch_advance(p.d_state, 1, st));
            }
        } else {
            const uint64_t nbatch = (s1 - s0 + (uint64_t)p.SB - 1) / (uint64_t)p.SB;
            auto it = p.graphs.find((int)prec);
            if (it == p.graphs.end()) {
                cudaGraph_t g;
                TN_CUDA(cudaStreamBeginCapture(p.graph_stream, cudaStreamCaptureModeThreadLocal));
                try {
                    enqueue_fused_batch(p, prec, p.graph_stream);
                } catch (...) {
                    cudaGraph_t junk;
                    cudaStreamEndCapture(p.graph_stream, &junk);
                    if (junk) cudaGraphDestroy(junk);
                    throw;
                }
                TN_CUDA(cudaStreamEndCapture(p.graph_stream, &g));
                cudaGraphExec_t ge;
                cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
                cudaGraphDestroy(g);
                TN_CUDA(e);
                it = p.graphs.emplace((int)prec, ge).first;
            }
            ConstBankOrder order(st);
            for (uint64_t b = 0; b < nbatch; ++b) TN_CUDA(cudaGraphLaunch(it->second, st));
        }
    }
    if (is_device_pointer(amps_out)) {
        TN_CUDA(launch_finalize(p.d_sum, p.d_comp, reinterpret_cast<double2 *>(amps_out), nout,
                                accumulate, st));
    } else {
        TN_CUDA(launch_finalize(p.d_sum, p.d_comp, p.d_out, nout, 0, st));
        std::vector<double> h_out((size_t)nout * 2);
        TN_CUDA(cudaMemcpyAsync(h_out.data(), p.d_out, sizeof(double2) * (size_t)nout,
                                cudaMemcpyDeviceToHost, st));
        TN_CUDA(cudaStreamSynchronize(st));
        for (int64_t i = 0; i < nout * 2; ++i)
            amps_out[i] = accumulate ? amps_out[i] + h_out[(size_t)i] : h_out[(size_t)i];
    }
}

// ------------------------------------------------------------------------
// Hypergraph plans: every pairwise step of the scheme runs as one FP64
// contraction on the GPU (small_contract_kernel with the kept shared edges as
// batch indices), per prefix; intermediates are stream-ordered allocations
// freed as soon as they are consumed.
void hyper_prepare(Plan &p, const uint8_t *prefixes, int n_prefixes, cudaStream_t st) {
    const Network &net = p.net;
    const int n_closed = (int)net.closed_qubits.size();
    if (n_prefixes <= 0) {
        prefixes = nullptr;
        n_prefixes = 1;
    }
    p.release();
    TN_CUDA(init_kernels());
    TN_CUDA(cudaGetDevice(&p.device));
    p.n_prefix = n_prefixes;
    const int L = net.n_leaves();
    p.h_leaf_off.assign((size_t)L, 0);
    int64_t total = 0;
    for (int i = 0; i < L; ++i) {
        p.h_leaf_off[(size_t)i] = total;
        total += (int64_t)net.leaves[(size_t)i].vals.size();
    }
    p.h_leaf_total = total;
    std::vector<double2> h((size_t)(total * n_prefixes));
    for (int pp = 0; pp < n_prefixes; ++pp)
        for (int i = 0; i < L; ++i) {
            const Leaf &lf = net.leaves[(size_t)i];
            for (size_t v = 0; v < lf.vals.size(); ++v) {
                cd x = lf.vals[v];
                if (lf.kind == LEAF_PROJ) {
                    const uint8_t b = prefixes ? prefixes[(size_t)pp * n_closed + lf.gate]
                                               : net.closed_bits[(size_t)lf.gate];
                    if (b > 1) fail(TN_ERR_INVALID_ARG, "prefix bits must be 0 or 1");
                    x = (v == (size_t)b) ? 1.0 : 0.0;
                }
                h[(size_t)(pp * total + p.h_leaf_off[(size_t)i] + (int64_t)v)] = make_double2(x.real(), x.imag());
            }
        }
    p.d_hleaf = dev_alloc<double2>(p, h.size());
    TN_CUDA(cudaMemcpy(p.d_hleaf, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice));
    const int nb = 1 << (int)net.open_edges.size();
    p.d_sum = dev_alloc<double2>(p, (size_t)n_prefixes * nb);
    p.d_comp = dev_alloc<double2>(p, (size_t)n_prefixes * nb);
    p.d_out = dev_alloc<double2>(p, (size_t)n_prefixes * nb);
    TN_CUDA(cudaMemset(p.d_comp, 0, sizeof(double2) * (size_t)n_prefixes * nb));
    p.prepared = true;
}

void hyper_contract(Plan &p, uint64_t s0, uint64_t s1, cudaStream_t st, double *amps_out,
                    int accumulate) {
    require_plan_device(p);
    if (s0 > s1 || s1 > 1) fail(TN_ERR_INVALID_ARG, "a hypergraph plan has one slice: range within [0, 1]");
    if (!amps_out) fail(TN_ERR_INVALID_ARG, "amps_out is null");
    const Network &net = p.net;
    const int L = net.n_leaves();
    const int nb = 1 << (int)net.open_edges.size();
    const int64_t nout = (int64_t)p.n_prefix * nb;
    TN_CUDA(cudaMemsetAsync(p.d_sum, 0, sizeof(double2) * (size_t)nout, st));
    const HyperScheme &hs = p.hs;
    const size_t np = hs.pairs.size();
    auto layout = [&](int ref) -> const std::vector<int> & {
        return ref < L ? net.leaves[(size_t)ref].edges : hs.node_edges[(size_t)(ref - L)];
    };
    // all prefixes in each launch: a tensor that depends on a projector has
    // one copy per prefix (stride = its size), the others one shared copy
    if (s1 > s0) {
        std::vector<double2 *> node(np, nullptr);
        std::vector<char> per_prefix(np, 0);
        auto dep = [&](int ref) {
            return ref < L ? net.leaves[(size_t)ref].kind == LEAF_PROJ && p.n_prefix > 1
                           : (bool)per_prefix[(size_t)(ref - L)];
        };
        auto base = [&](int ref) -> const double2 * {
            return ref < L ? p.d_hleaf + p.h_leaf_off[(size_t)ref] : node[(size_t)(ref - L)];
        };
        auto stride = [&](int ref) -> int64_t {
            if (!dep(ref)) return 0;
            return ref < L ? p.h_leaf_total : (int64_t)1 << hs.node_edges[(size_t)(ref - L)].size();
        };
        for (size_t k = 0; k < np; ++k) {
            const int a = hs.pairs[k].first, b = hs.pairs[k].second;
            const std::vector<int> &lc = hs.node_edges[k];
            const bool last = k + 1 == np;
            per_prefix[k] = last || dep(a) || dep(b);
            const int items = per_prefix[k] ? p.n_prefix : 1;
            double2 *out = p.d_sum;  // last node: prefix-major, 2^n_open each
            if (!last) {
                void *q = nullptr;
                TN_CUDA(cudaMallocAsync(&q, (sizeof(double2) << lc.size()) * (size_t)items, st));
                out = static_cast<double2 *>(q);
            }
            SmallContract d = make_contract(layout(a), layout(b), lc);
            TN_CUDA(launch_small_contract_batched(base(a), stride(a), base(b), stride(b), out, nullptr,
                                                  items > 1 ? (int64_t)1 << lc.size() : 0, items, d, st));
            node[k] = out;
            for (int r : {a, b})
                if (r >= L) {
                    TN_CUDA(cudaFreeAsync(node[(size_t)(r - L)], st));
                    node[(size_t)(r - L)] = nullptr;
                }
        }
    }
    if (is_device_pointer(amps_out)) {
        TN_CUDA(launch_finalize(p.d_sum, p.d_comp, reinterpret_cast<double2 *>(amps_out), nout, accumulate, st));
    } else {
        TN_CUDA(launch_finalize(p.d_sum, p.d_comp, p.d_out, nout, 0, st));
        std::vector<double> h_out((size_t)nout * 2);
        TN_CUDA(cudaMemcpyAsync(h_out.data(), p.d_out, sizeof(double2) * (size_t)nout,
                                cudaMemcpyDeviceToHost, st));
        TN_CUDA(cudaStreamSynchronize(st));
        for (int64_t i = 0; i < nout * 2; ++i)
            amps_out[i] = accumulate ? amps_out[i] + h_out[(size_t)i] : h_out[(size_t)i];
    }
}

// Flops of the stem steps applied by each fused pass / plain step.
static double step_flops(const Plan &p, int step) {
    const ExecStep &es = p.sp.plain_steps[(size_t)step];
    return 8.0 * std::exp2((double)(es.r_in + es.n));
}

std::vector<tn_launch_record> plan_profile(Plan &p, uint64_t s0, tn_precision prec,
                                          tn_exec_mode mode, cudaStream_t st) {
    require_plan_device(p);
    const int nsl = (int)p.scheme.sliced_list.size();
    const uint64_t total = nsl >= 63 ? ~0ull : (1ull << nsl);
    if (s0 >= total) fail(TN_ERR_INVALID_ARG, "slice_begin out of range");
    const uint64_t sb = mode == TN_EXEC_FUSED ? (uint64_t)p.SB : 1ull;
    const uint64_t s1 = std::min<uint64_t>(total, s0 + sb);
    const int nb = 1 << (int)p.net.open_edges.size();
    TN_CUDA(cudaMemsetAsync(p.d_sum, 0, sizeof(double2) * (size_t)p.n_prefix * nb, st));
    TN_CUDA(cudaMemsetAsync(p.d_comp, 0, sizeof(double2) * (size_t)p.n_prefix * nb, st));
    DevState h{(int64_t)s0, (int64_t)s1, 0, 0};
    TN_CUDA(cudaMemcpyAsync(p.d_state, &h, sizeof(h), cudaMemcpyHostToDevice, st));
    std::vector<tn_launch_record> recs;
    std::vector<cudaEvent_t> ev;
    auto mark = [&]() {
        cudaEvent_t e;
        TN_CUDA(cudaEventCreate(&e));
        TN_CUDA(cudaEventRecord(e, st));
        ev.push_back(e);
    };
    const int items_fused = p.SB * p.n_prefix;
    const int items = mode == TN_EXEC_FUSED ? (int)std::min<uint64_t>(s1 - s0, sb) * p.n_prefix
                                            : 1;
    std::unique_ptr<ConstBankOrder> order;
    if (mode == TN_EXEC_FUSED) order.reset(new ConstBankOrder(st));
    mark();
    if (mode == TN_EXEC_FUSED) {
        BatchArgs ba{p.d_state, p.SB, items_fused, 0};
        int cur = -1;
        for (size_t i = 0; i < p.sp.fused_items.size(); ++i) {
            const FusedItem &it = p.sp.fused_items[i];
            const float2 *in = cur < 0 ? nullptr : p.d_buf[cur];
            const int nxt = cur < 0 ? 0 : 1 - cur;
            tn_launch_record r{};
            r.index = (int)i;
            r.items = items;
            if (it.kind == 0) {
                const DevPass &P = p.sp.fused_passes[(size_t)it.pass];
                TN_CUDA(launch_pass(p.d_fused + it.pass, P, p.d_chunks, p.d_branches,
                                    p.h_branches.data(), p.d_pool, in, p.d_buf[nxt], ba, st));
                r.kind = 0;
                r.r_in = P.r_in;
                r.r_out = P.r_out;
                int ns = 0;
                double fl = 0;
                for (size_t s = 0; s < p.sp.step_pass.size(); ++s)
                    if (p.sp.step_pass[s] == it.pass) {
                        ++ns;
                        fl += step_flops(p, (int)s);
                    }
                r.n_steps = ns;
                r.flops = fl * items;
                r.bytes = 8.0 * (std::exp2(P.r_in) + std::exp2(P.r_out)) * items;
            } else {
                TN_CUDA(launch_stem_gemm(p.d_buf[cur], p.d_buf[nxt], it.M, it.k, it.n,
                                         (int64_t)1 << it.r_in, (int64_t)1 << it.r_out,
                                         p.d_branches + it.branch, p.d_pool, ba, prec, st));
                r.kind = 1;
                r.r_in = it.r_in;
                r.r_out = it.r_out;
                r.n_steps = 1;
                r.k = it.k;
                r.n = it.n;
                r.flops = 8.0 * std::exp2((double)(it.r_in + it.n)) * items;
                r.bytes = 8.0 * (std::exp2(it.r_in) + std::exp2(it.r_out)) * items;
            }
            recs.push_back(r);
            mark();
            cur = nxt;
        }
        TN_CUDA(launch_accumulate(p.d_buf[cur], (int)p.net.open_edges.size(), p.d_pos_fused,
                                  p.d_sum, p.d_comp, ba, p.n_prefix, st));
        tn_launch_record r{};
        r.kind = 3;
        r.index = (int)recs.size();
        r.items = items;
        r.bytes = 8.0 * nb * items;
        recs.push_back(r);
        mark();
    } else {
        BatchArgs ba{p.d_state, 1, 1, 0};
        int cur = -1;
        for (size_t i = 0; i < p.sp.plain_steps.size(); ++i) {
            const ExecStep &es = p.sp.plain_steps[i];
            const float2 *in = cur < 0 ? nullptr : p.d_buf[cur];
            const int mid = cur < 0 ? 0 : 1 - cur;
            const DevPass &P = p.sp.plain_passes[(size_t)es.permute_pass];
            TN_CUDA(launch_pass(p.d_plain + es.permute_pass, P, p.d_chunks, p.d_branches,
                                p.h_branches.data(), p.d_pool, in, p.d_buf[mid], ba, st));
            tn_launch_record r{};
            r.kind = 2;
            r.index = (int)recs.size();
            r.items = 1;
            r.r_in = r.r_out = P.r_in;
            r.bytes = 16.0 * std::exp2(P.r_in);
            recs.push_back(r);
            mark();
            const int out = 1 - mid;
            TN_CUDA(launch_stem_gemm(p.d_buf[mid], p.d_buf[out], es.M, es.k, es.n,
                                     (int64_t)1 << es.r_in, (int64_t)1 << es.r_out,
                                     p.d_branches + es.branch, p.d_pool, ba, TN_PREC_FP32_SIMT, st));
            tn_launch_record g{};
            g.kind = 1;
            g.index = (int)recs.size();
            g.items = 1;
            g.r_in = es.r_in;
            g.r_out = es.r_out;
            g.n_steps = 1;
            g.k = es.k;
            g.n = es.n;
            g.flops = step_flops(p, (int)i);
            g.bytes = 8.0 * (std::exp2(es.r_in) + std::exp2(es.r_out));
            recs.push_back(g);
            mark();
            cur = out;
        }
    }
    order.reset();
    TN_CUDA(cudaStreamSynchronize(st));
    for (size_t i = 0; i < recs.size(); ++i) {
        float ms = 0;
        TN_CUDA(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
        recs[i].ms = ms;
    }
    for (auto e : ev) cudaEventDestroy(e);
    return recs;
}

}  // namespace tn
