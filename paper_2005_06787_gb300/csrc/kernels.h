// Host-side launchers of the CUDA kernels (kernels.cu, gemm_tc.cu).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace tn {

// Per-launch batch bookkeeping kept in device memory, so that a captured
// graph can be replayed for successive slice batches.
struct DevState {
    int64_t slice_base;  // slice of batch item 0
    int64_t slice_end;   // end of the requested slice range
    int32_t err;         // nonzero: a kernel met an out-of-range descriptor
    int32_t pad;
};

// Batch items: item = p_local * SB + j -> prefix p0 + p_local, slice base + j.
struct BatchArgs {
    const DevState *state;
    int SB;          // slices per batch
    int n_items;     // items in this launch
    int p0;          // first prefix of this launch
};

struct SmallContract {
    int ra, rb, rc, k;
    int a_out[40], b_out[40];  // per output bit: position in A / B, -1 if absent
    int a_k[40], b_k[40];      // per contracted bit: position in A / B
};

cudaError_t init_kernels();

// A fused pass launched with one batch item reads the branch matrices of its
// (2,2) steps and paired (2,1), (1,3), (1,2) steps from a per-device
// constant-bank copy that launch_pass stages on the launch's stream (one
// gather kernel and one device-to-device copy); other shapes keep them in
// shared memory.
bool pass_uses_const_bank(const DevPass &h_pass, const BatchArgs &ba);
inline bool step_on_const_bank(const DevStep &S) {
    if (S.branch < 0) return false;
    if (S.k == 2 && S.n == 2) return true;
    return S.pair && ((S.k == 2 && S.n == 1) || (S.k == 1 && S.n == 3) || (S.k == 1 && S.n == 2));
}
inline bool pass_has_const_steps(const DevPass &h_pass) {
    for (int t = 0; t < h_pass.n_steps; ++t)
        if (step_on_const_bank(h_pass.steps[t])) return true;
    return false;
}


// Orders the calls that enqueue such passes: the constructor takes a
// process-wide lock and makes `st` wait for the last call enqueued on this
// device; the destructor records this call's end on `st` and unlocks. A
// stream under capture is left alone (the graph is ordered where it is
// launched).
class ConstBankOrder {
  public:
    explicit ConstBankOrder(cudaStream_t st);
    ~ConstBankOrder();
    ConstBankOrder(const ConstBankOrder &) = delete;
    ConstBankOrder &operator=(const ConstBankOrder &) = delete;

  private:
    cudaStream_t st_;
    cudaEvent_t ev_ = nullptr;
};
cudaError_t launch_pass(const DevPass *d_pass, const DevPass &h_pass, const int *d_chunks,
                        const DevBranch *d_branches, const DevBranch *h_branches,
                        const float2 *pool, const float2 *in, float2 *out, BatchArgs ba,
                        cudaStream_t st);

// FP64 pairwise contraction for branch pre-computation; writes FP64 to Cd, or
// rounds to FP32 into Cf when Cf is given.
cudaError_t launch_small_contract(const double2 *A, const double2 *B, double2 *Cd, float2 *Cf,
                                  const SmallContract &d, cudaStream_t st);
// The same over `items` batch items: item i reads A + i sA, B + i sB and
// writes Cd / Cf + i sC (stride 0: one copy shared by every item).
cudaError_t launch_small_contract_batched(const double2 *A, int64_t sA, const double2 *B, int64_t sB,
                                          double2 *Cd, float2 *Cf, int64_t sC, int items,
                                          const SmallContract &d, cudaStream_t st);

// Stem GEMM step over batch items: C_item[m][nu] = sum_kappa A_item[m][kappa] *
// Branch_item[kappa][nu]; A item stride 2^r_in, C item stride 2^r_out.
cudaError_t launch_stem_gemm(const float2 *A, float2 *C, int64_t M, int k, int n, int64_t strideA,
                             int64_t strideC, const DevBranch *d_branch_entry, const float2 *pool,
                             BatchArgs ba, tn_precision prec, cudaStream_t st);

// Plain batched complex GEMM (tn_cgemm).
cudaError_t launch_cgemm(const float2 *A, const float2 *B, float2 *C, int64_t M, int64_t K,
                         int64_t N, int64_t batch, int64_t sA, int64_t sB, int64_t sC,
                         tn_precision prec, cudaStream_t st);

// FP64 Neumaier accumulation of final open tensors into sum / comp.
cudaError_t launch_accumulate(const float2 *fin, int n_open, const int *d_pos, double2 *sum,
                              double2 *comp, BatchArgs ba, int n_prefix_total, cudaStream_t st);
cudaError_t launch_advance(DevState *state, int64_t by, cudaStream_t st);
cudaError_t launch_finalize(const double2 *sum, const double2 *comp, double2 *out, int64_t n,
                            int accumulate, cudaStream_t st);
cudaError_t launch_xeb_sum(const double2 *amps, int64_t n, double *out_sum, cudaStream_t st);
cudaError_t launch_permute(const float2 *in, float2 *out, int rank, const int *perm,
                           cudaStream_t st);
cudaError_t launch_frugal_sample(const double2 *amps, const double *u, const double *key, int64_t B,
                                 int K, int n_qubits, double M, int32_t *idx, int32_t *cnt,
                                 double2 *picked, cudaStream_t st);

// FP32 FMA rate of this GPU (TFLOP/s) from independent FMA chains on every
// SM, best of three timed launches; synchronises st.
cudaError_t measure_fma_peak(cudaStream_t st, double *tflops, int *sm_count);

// Large complex GEMMs on tcgen05 (gemm_large.cu): TMA-fed, warp-specialised,
// for K >= 32, 2K % 64 == 0, 2N a multiple of the tile width (128 for the x3
// precisions, 256 for BF16 x1), M >= 128 and 16-byte aligned A and C.
bool tc_large_supported(int64_t M, int64_t K, int64_t N, tn_precision prec, const void *A, const void *C);
cudaError_t launch_tc_cgemm_large(const float2 *A, const float2 *B, float2 *C, int64_t M, int64_t K,
                                  int64_t N, tn_precision prec, int *err, cudaStream_t st);
// A stem GEMM step of one batch item (2^k x 2^n branch of the launch's slice)
// on the same TMA-fed kernels: 2^k, 2^n >= 16, M >= 128.
bool tc_large_stem_supported(int64_t M, int k, int n, tn_precision prec, const void *A, const void *C);
cudaError_t launch_tc_stem_gemm_large(const float2 *A, float2 *C, int64_t M, int k, int n,
                                      const DevBranch *d_branch_entry, const float2 *pool, BatchArgs ba,
                                      tn_precision prec, int *err, cudaStream_t st);

bool tc_gemm_supported(int k, int n);
cudaError_t tc_gemm_init();
cudaError_t tc_error_flag(int *out);
cudaError_t launch_tc_cgemm(const float2 *A, const float2 *B, float2 *C, int64_t M, int64_t K,
                            int64_t N, int64_t batch, int64_t sA, int64_t sB, int64_t sC,
                            tn_precision prec, cudaStream_t st);
cudaError_t launch_tc_stem_gemm(const float2 *A, float2 *C, int64_t M, int k, int n,
                                int64_t strideA, int64_t strideC, const DevBranch *d_branch_entry,
                                const float2 *pool, BatchArgs ba, tn_precision prec,
                                cudaStream_t st);

}  // namespace tn
