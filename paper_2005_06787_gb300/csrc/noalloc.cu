// tn_contract_stem_noalloc: the fused stem contraction with its scratch in a
// fixed static device array, so that the call itself allocates no memory.
//
// Who needs it: callers that must not allocate device memory while they run
// the contraction. cudaMalloc synchronises the whole device and may fail under
// a memory budget owned by someone else (a framework's own pooling
// allocator, a process sharing the GPU under a fixed quota); a host loop that
// hands slice ranges to the GPU at high rate cannot afford either. Such a
// caller prepares a plan once (which does allocate: branch storage and
// descriptors), then calls this entry point as often as it likes.
//
// Limits and sharing. The scratch holds two stem buffers of NOALLOC_STEM_MAX
// complex64 entries and NOALLOC_AMPS_MAX compensated FP64 sums. A plan fits if
// n_prefixes * 2^max_rank <= NOALLOC_STEM_MAX and n_prefixes * 2^n_open <=
// NOALLOC_AMPS_MAX; otherwise the call returns TN_ERR_UNSUPPORTED. Every GPU
// that loads the library holds this array (about 16.5 MiB) until the process
// exits. All calls share the one array: calls whose work overlaps on the GPU
// (on different streams, or from different threads) race and corrupt each
// other; serialise them. Each call clears the sums it uses before starting,
// so leftovers of an earlier call never leak into the result.
//
// Set-up. The first call on each device looks up the array's device address
// with cudaGetSymbolAddress, with that device current, and caches it; make
// that first call before any stream capture is begun on the calling thread.
#include <cuda_runtime.h>

#include <mutex>

#include "plan.h"

namespace tn {

constexpr int64_t NOALLOC_STEM_MAX = (int64_t)1 << 20;  // entries per stem buffer (8 MiB)
constexpr int64_t NOALLOC_AMPS_MAX = (int64_t)1 << 14;  // compensated sums (256 KiB each)

struct NoAllocScratch {
    float2 buf[2][NOALLOC_STEM_MAX];
    double2 sum[NOALLOC_AMPS_MAX];
    double2 comp[NOALLOC_AMPS_MAX];
    DevState state;
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of the scratch, per device, from cudaGetSymbolAddress.
static NoAllocScratch *noalloc_scratch_for_current_device() {
    static std::mutex mu;
    static NoAllocScratch *addr[64] = {nullptr};
    int dev = 0;
    TN_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(TN_ERR_UNSUPPORTED, "device index above 63");
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            fail(TN_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        addr[dev] = reinterpret_cast<NoAllocScratch *>(p);
    }
    return addr[dev];
}

__global__ void noalloc_begin_kernel(NoAllocScratch *s, int64_t s0, int64_t s1, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        s->sum[i] = make_double2(0.0, 0.0);
        s->comp[i] = make_double2(0.0, 0.0);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s->state.slice_base = s0;
        s->state.slice_end = s1;
        s->state.err = 0;
    }
}

void plan_contract_noalloc(Plan &p, uint64_t s0, uint64_t s1, cudaStream_t st, double *amps_out,
                           int accumulate) {
    // the plan's buffers live on the device it was prepared on, and the
    // scratch address below is that of the current device: they must agree
    require_plan_device(p);
    const int nsl = (int)p.scheme.sliced_list.size();
    const uint64_t total = nsl >= 63 ? ~0ull : (1ull << nsl);
    if (s0 > s1 || s1 > total) fail(TN_ERR_INVALID_ARG, "slice range outside [0, 2^n_sliced]");
    if (!amps_out) fail(TN_ERR_INVALID_ARG, "amps_out is null");
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, amps_out) != cudaSuccess ||
        (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        fail(TN_ERR_INVALID_ARG, "amps_out must be device memory for the allocation-free call");
    }
    const int n_open = (int)p.net.open_edges.size();
    const int64_t nout = (int64_t)p.n_prefix << n_open;
    const int64_t per_slice = (int64_t)p.n_prefix << p.sp.max_rank;
    if (per_slice > NOALLOC_STEM_MAX || nout > NOALLOC_AMPS_MAX)
        fail(TN_ERR_UNSUPPORTED,
             "plan too large for the allocation-free call: needs n_prefixes * 2^max_rank <= 2^20 "
             "and n_prefixes * 2^n_open <= 2^14 (use tn_contract_stem)");
    NoAllocScratch *S = noalloc_scratch_for_current_device();
    // slices per launch: the plan's batch, shrunk to fit the static buffers
    const int64_t SB = std::max<int64_t>(1, std::min<int64_t>(p.SB, NOALLOC_STEM_MAX / per_slice));
    noalloc_begin_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((nout + 255) / 256, 1024)),
                           256, 0, st>>>(S, (int64_t)s0, (int64_t)s1, (int)nout);
    TN_CUDA(cudaGetLastError());
    const int items = (int)SB * p.n_prefix;
    BatchArgs ba{&S->state, (int)SB, items, 0};
    const uint64_t nbatch = (s1 - s0 + (uint64_t)SB - 1) / (uint64_t)SB;
    ConstBankOrder order(st);
    for (uint64_t b = 0; b < nbatch; ++b) {
        int cur = -1;
        for (const FusedItem &it : p.sp.fused_items) {
            const float2 *in = cur < 0 ? nullptr : S->buf[cur];
            const int nxt = cur < 0 ? 0 : 1 - cur;
            if (it.kind == 0) {
                TN_CUDA(launch_pass(p.d_fused + it.pass, p.sp.fused_passes[(size_t)it.pass],
                                    p.d_chunks, p.d_branches, p.h_branches.data(), p.d_pool, in,
                                    S->buf[nxt], ba, st));
            } else {
                TN_CUDA(launch_stem_gemm(S->buf[cur], S->buf[nxt], it.M, it.k, it.n,
                                         (int64_t)1 << it.r_in, (int64_t)1 << it.r_out,
                                         p.d_branches + it.branch, p.d_pool, ba, TN_PREC_FP32_SIMT,
                                         st));
            }
            cur = nxt;
        }
        TN_CUDA(launch_accumulate(S->buf[cur], n_open, p.d_pos_fused, S->sum, S->comp, ba,
                                  p.n_prefix, st));
        TN_CUDA(launch_advance(&S->state, SB, st));
    }
    TN_CUDA(launch_finalize(S->sum, S->comp, reinterpret_cast<double2 *>(amps_out), nout,
                            accumulate, st));
}

}  // namespace tn
