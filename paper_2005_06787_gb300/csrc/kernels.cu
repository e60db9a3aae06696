// CUDA kernels of the stem (sm_103a): fused multi-step pass, branch
// pre-computation contraction, SIMT complex GEMM, FP64 compensated slice sum,
// XEB reduction.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <mutex>

#include "kernels.h"

namespace tn {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ void cfma(float2 &acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

// Offset (in complex entries) of branch storage for prefix p and slice s.
__device__ __forceinline__ int64_t branch_offset(const DevBranch &b, int p, int64_t s) {
    int64_t o = b.base + (int64_t)p * b.prefix_stride;
    for (int i = 0; i < b.n_sl; ++i)
        if ((s >> b.sl_bit[i]) & 1) o += (int64_t)1 << b.sl_pos[i];
    return o;
}

// ---------------------------------------------------------------- fused pass
// Tile bank swizzle (same map as tile_swizzle on the host).
__device__ __forceinline__ int dev_swizzle(int p) {
    const int x = (p >> 4) & 255;
    return p ^ (((x ^ (x >> 3) ^ (x >> 6)) & 7) << 1);
}

// One stem step on the tile, in place: for each rest index rho (one per
// thread and iteration), y[nu] = sum_kappa x[kappa] * B[kappa][nu], reading
// x at t(rho) ^ koff[kappa] and writing y at t(rho) ^ noff[nu]. A thread
// reads all of its x before writing, and different rest indices touch
// disjoint entries. Branch clusters have rank <= 4, so B (2^(K+N) <= 16
// entries) and both offset lists live in registers for the whole step. The
// thread count is a power of two >= 64, so rest-index bits 0-5 are fixed per
// thread and only the high table is read per iteration.
template <int K, int N>
__device__ __forceinline__ void step_body(float2 *tile, const DevStep &S, const float2 *__restrict__ Bm,
                                          int nt) {
    constexpr int NK = 1 << K, NN = 1 << N;
    float2 bv[NK * NN];
#pragma unroll
    for (int i = 0; i < NK * NN; ++i) bv[i] = Bm[i];
    int koff[NK], noff[NN];
#pragma unroll
    for (int kk = 0; kk < NK; ++kk) koff[kk] = S.koff[kk];
    // k == n: the nu bits took the kappa positions in order, so results go
    // where their inputs were (the host checks noff == koff for such steps)
#pragma unroll
    for (int nn = 0; nn < NN; ++nn) noff[nn] = (K == N) ? koff[nn % NK] : S.noff[nn];
    const int nrest = 1 << S.rest;
    const int t_lo = S.lo[threadIdx.x & 63];
    for (int r = threadIdx.x; r < nrest; r += nt) {
        const int t = t_lo ^ S.hi[r >> 6];
        float2 x[NK];
#pragma unroll
        for (int kk = 0; kk < NK; ++kk) x[kk] = tile[t ^ koff[kk]];
#pragma unroll
        for (int nn = 0; nn < NN; ++nn) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int kk = 0; kk < NK; ++kk) cfma(acc, x[kk], bv[kk * NN + nn]);
            tile[t ^ noff[nn]] = acc;
        }
    }
}

// The same step with rest indices taken in adjacent pairs: rest-index bit 0
// is tile position 0 (offset bit 0), so the entries of rest indices 2i and
// 2i+1 sit side by side and move with one 16-byte access per kappa / nu.
template <int K, int N>
__device__ __forceinline__ void step_body_pair(float2 *tile, const DevStep &S,
                                               const float2 *__restrict__ Bm, int nt) {
    constexpr int NK = 1 << K, NN = 1 << N;
    float2 bv[NK * NN];
#pragma unroll
    for (int i = 0; i < NK * NN; ++i) bv[i] = Bm[i];
    int koff[NK], noff[NN];
#pragma unroll
    for (int kk = 0; kk < NK; ++kk) koff[kk] = S.koff[kk];
    // k == n: the nu bits took the kappa positions in order, so results go
    // where their inputs were (the host checks noff == koff for such steps)
#pragma unroll
    for (int nn = 0; nn < NN; ++nn) noff[nn] = (K == N) ? koff[nn % NK] : S.noff[nn];
    const int npair = 1 << (S.rest - 1);
    const int t_lo = S.lo[(2 * threadIdx.x) & 63];
    for (int r2 = threadIdx.x; r2 < npair; r2 += nt) {
        const int t = t_lo ^ S.hi[r2 >> 5];
        float4 x[NK];
#pragma unroll
        for (int kk = 0; kk < NK; ++kk) x[kk] = *reinterpret_cast<const float4 *>(tile + (t ^ koff[kk]));
#pragma unroll
        for (int nn = 0; nn < NN; ++nn) {
            float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
            for (int kk = 0; kk < NK; ++kk) {
                const float2 b = bv[kk * NN + nn];
                cfma(a0, make_float2(x[kk].x, x[kk].y), b);
                cfma(a1, make_float2(x[kk].z, x[kk].w), b);
            }
            *reinterpret_cast<float4 *>(tile + (t ^ noff[nn])) = make_float4(a0.x, a0.y, a1.x, a1.y);
        }
    }
}

__device__ void run_step(float2 *tile, const DevStep &S, const float2 *Bm, int nt) {
    if (S.pair) {
        switch (S.k * 8 + S.n) {
#define TN_CASE(K, N) \
    case K * 8 + N: step_body_pair<K, N>(tile, S, Bm, nt); return;
            TN_CASE(1, 0) TN_CASE(1, 1) TN_CASE(1, 2) TN_CASE(1, 3)
            TN_CASE(2, 0) TN_CASE(2, 1) TN_CASE(2, 2)
            TN_CASE(3, 0)
#undef TN_CASE
            default: break;
        }
    }
    switch (S.k * 8 + S.n) {
#define TN_CASE(K, N) \
    case K * 8 + N: step_body<K, N>(tile, S, Bm, nt); break;
        TN_CASE(1, 0) TN_CASE(1, 1) TN_CASE(1, 2) TN_CASE(1, 3)
        TN_CASE(2, 0) TN_CASE(2, 1) TN_CASE(2, 2)
        TN_CASE(3, 0) TN_CASE(3, 1)
        TN_CASE(4, 0)
#undef TN_CASE
        default: break;
    }
}

// Asynchronous global -> shared copies (cp.async): 16 bytes = one entry
// pair (bypassing L1), or 8 bytes = one entry for rank-0 tensors.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() {
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

constexpr int PASS_THREADS = 256;
constexpr size_t PASS_HEAD_BYTES = (offsetof(DevPass, steps) + 15) / 16 * 16;

// Branch matrices in the constant bank. All units of a launch with one batch
// item (one prefix, one slice) use the same branch matrices, so the pass can
// take them as constant-bank operands of its FMAs at fixed offsets: for a
// (2,2) step this frees the 32 registers a 4 x 4 complex matrix would hold
// and the shared-memory loads that fill them at every step. stage_bm_kernel
// gathers the matrices of the launch's slice into g_bm_stage, and a
// device-to-device copy on the same stream moves them into c_bm right before
// the pass; ConstBankOrder keeps calls on different streams from overlapping.
constexpr int CB_ENTRIES = MAX_PASS_STEPS * 16;
__constant__ float2 c_bm[CB_ENTRIES];
__device__ float2 g_bm_stage[CB_ENTRIES];
// the same entries as (Br, Bi, -Bi, Br) for the packed FP32 FMAs of paired
// (2,2) steps
__constant__ float4 c_bm2[CB_ENTRIES];
__device__ float4 g_bm2_stage[CB_ENTRIES];

// Packed FP32 pairs (fma.rn.f32x2): one instruction does two FP32 FMAs at
// the same lane rate as two FFMA, which halves the issue slots of the
// arithmetic in an issue-bound loop.
__device__ __forceinline__ unsigned long long pk2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1,%2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long x) {
    float lo, hi;
    asm("mov.b64 {%0,%1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x));
    return make_float2(lo, hi);
}
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

constexpr int CB_MAX_DEV = 64;
static float2 *g_bm_stage_dev[CB_MAX_DEV];
static float4 *g_bm2_stage_dev[CB_MAX_DEV];
static cudaEvent_t g_cb_event[CB_MAX_DEV];
static std::recursive_mutex g_cb_mutex;

// one block: entries of every step's branch matrix (at most 16) for batch
// item 0, at 16 * (step slot) in the stage, and each entry's expansion for
// the packed FMAs
__global__ void stage_bm_kernel(const DevPass *__restrict__ gpass, const DevBranch *__restrict__ branches,
                                const float2 *__restrict__ pool, BatchArgs ba) {
    const int p = ba.p0;
    const int64_t s = ba.state->slice_base;
    const int n = gpass->n_steps;
    for (int t = 0; t < n; ++t) {
        const DevStep &S = gpass->steps[t];
        if (S.branch < 0) continue;
        const float2 *src = pool + branch_offset(branches[S.branch], p, s);
        const int cnt = 1 << (S.k + S.n);
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const float2 b = src[i];
            g_bm_stage[t * 16 + i] = b;
            g_bm2_stage[t * 16 + i] = make_float4(b.x, b.y, -b.y, b.x);
        }
    }
}

// A (2,2) step in step slot T with its branch matrix in c_bm (c_bm2 for the
// packed FMAs of the paired form; k == n, so the results go back to the kappa
// offsets); PAIR as in step_body_pair. S is the
// step's descriptor in the kernel's parameter bank: its offsets and counts
// are constant-bank operands, and its hi table is read at warp-uniform
// indices. The lo table, which every lane reads at its own index, comes from
// the shared-memory copy (divergent constant-bank reads serialise).
template <int T, bool PAIR>
__device__ __forceinline__ void step22_const(float2 *tile, const DevStep &S, const int *lo_sm, int nt) {
    int koff[4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) koff[kk] = S.koff[kk];
    if (PAIR) {
        const int npair = 1 << (S.rest - 1);
        const int t_lo = lo_sm[(2 * threadIdx.x) & 63];
        for (int r2 = threadIdx.x; r2 < npair; r2 += nt) {
            const int t = t_lo ^ S.hi[r2 >> 5];
            float4 x[4];
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) x[kk] = *reinterpret_cast<const float4 *>(tile + (t ^ koff[kk]));
            // (acc.re, acc.im) += (x.re, x.re) * (Br, Bi) + (x.im, x.im) * (-Bi, Br):
            // the FMAs of cfma in the same order, two per instruction
            unsigned long long X0[4], S0[4], X1[4], S1[4];
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                X0[kk] = pk2(x[kk].x, x[kk].x);
                S0[kk] = pk2(x[kk].y, x[kk].y);
                X1[kk] = pk2(x[kk].z, x[kk].z);
                S1[kk] = pk2(x[kk].w, x[kk].w);
            }
#pragma unroll
            for (int nn = 0; nn < 4; ++nn) {
                unsigned long long a0 = 0ull, a1 = 0ull;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const float4 b = c_bm2[T * 16 + kk * 4 + nn];
                    const unsigned long long b1 = pk2(b.x, b.y), b2 = pk2(b.z, b.w);
                    a0 = ffma2(X0[kk], b1, a0);
                    a0 = ffma2(S0[kk], b2, a0);
                    a1 = ffma2(X1[kk], b1, a1);
                    a1 = ffma2(S1[kk], b2, a1);
                }
                const float2 y0 = upk2(a0), y1 = upk2(a1);
                *reinterpret_cast<float4 *>(tile + (t ^ koff[nn])) = make_float4(y0.x, y0.y, y1.x, y1.y);
            }
        }
    } else {
        const int nrest = 1 << S.rest;
        const int t_lo = lo_sm[threadIdx.x & 63];
        for (int r = threadIdx.x; r < nrest; r += nt) {
            const int t = t_lo ^ S.hi[r >> 6];
            float2 x[4];
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) x[kk] = tile[t ^ koff[kk]];
#pragma unroll
            for (int nn = 0; nn < 4; ++nn) {
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) cfma(acc, x[kk], c_bm[T * 16 + kk * 4 + nn]);
                tile[t ^ koff[nn]] = acc;
            }
        }
    }
}

// a paired step of shape (K, N) in slot T with its branch matrix in c_bm:
// (2,1), (1,3) and (1,2), the other shapes the 53-qubit stems use most
template <int T, int K, int N>
__device__ __forceinline__ void stepkn_const_pair(float2 *tile, const DevStep &S, const int *lo_sm, int nt) {
    constexpr int NK = 1 << K, NN = 1 << N;
    int koff[NK], noff[NN];
#pragma unroll
    for (int kk = 0; kk < NK; ++kk) koff[kk] = S.koff[kk];
#pragma unroll
    for (int nn = 0; nn < NN; ++nn) noff[nn] = (K == N) ? koff[nn % NK] : S.noff[nn];
    const int npair = 1 << (S.rest - 1);
    const int t_lo = lo_sm[(2 * threadIdx.x) & 63];
    for (int r2 = threadIdx.x; r2 < npair; r2 += nt) {
        const int t = t_lo ^ S.hi[r2 >> 5];
        float4 x[NK];
#pragma unroll
        for (int kk = 0; kk < NK; ++kk) x[kk] = *reinterpret_cast<const float4 *>(tile + (t ^ koff[kk]));
#pragma unroll
        for (int nn = 0; nn < NN; ++nn) {
            float2 a0 = make_float2(0.f, 0.f), a1 = a0;
#pragma unroll
            for (int kk = 0; kk < NK; ++kk) {
                const float2 b = c_bm[T * 16 + kk * NN + nn];
                cfma(a0, make_float2(x[kk].x, x[kk].y), b);
                cfma(a1, make_float2(x[kk].z, x[kk].w), b);
            }
            *reinterpret_cast<float4 *>(tile + (t ^ noff[nn])) = make_float4(a0.x, a0.y, a1.x, a1.y);
        }
    }
}

// other step shapes on the constant-bank path: one out-of-line copy of the
// generic dispatch instead of one per step slot
__device__ __noinline__ void run_step_outline(float2 *tile, const DevStep &S, const float2 *Bm, int nt) {
    run_step(tile, S, Bm, nt);
}

// the steps of a pass, slot by slot from T (slots known at compile time); P is
// the descriptor's shared-memory copy, CP the same descriptor passed by value
// in the kernel's parameter bank
template <int T>
__device__ __forceinline__ void run_steps_const(float2 *tile, const DevPass &P, const DevPass &CP,
                                                const float2 *bm, const int *bm_off, int nt) {
    if constexpr (T < MAX_PASS_STEPS) {
        if (T >= CP.n_steps) return;
        const DevStep &S = CP.steps[T];
        if (S.branch >= 0) {
            if (S.k == 2 && S.n == 2) {
                if (S.pair)
                    step22_const<T, true>(tile, S, P.steps[T].lo, nt);
                else
                    step22_const<T, false>(tile, S, P.steps[T].lo, nt);
            } else if (S.pair && S.k == 2 && S.n == 1) {
                stepkn_const_pair<T, 2, 1>(tile, S, P.steps[T].lo, nt);
            } else if (S.pair && S.k == 1 && S.n == 3) {
                stepkn_const_pair<T, 1, 3>(tile, S, P.steps[T].lo, nt);
            } else if (S.pair && S.k == 1 && S.n == 2) {
                stepkn_const_pair<T, 1, 2>(tile, S, P.steps[T].lo, nt);
            } else {
                run_step_outline(tile, P.steps[T], bm + bm_off[T], nt);
            }
            __syncthreads();
        }
        run_steps_const<T + 1>(tile, P, CP, bm, bm_off, nt);
    }
}

// A fused pass over batch items x tiles. Each block walks its tiles with two
// tile buffers: while the steps run in place on one tile, the next tile's
// entries stream into the other buffer with cp.async, so the HBM read of
// tile i+1 overlaps the arithmetic of tile i. A tile's load puts input tile
// edge i at tile position i; the store reads the final positions through the
// st_lo / st_hi tables and writes the next layout.
// Shared memory: pass header and used step tables | chunk tables | two tiles
// | branch matrices of the current batch item. The CBANK instantiation (one
// batch item per launch) reads the branch matrices of its (2,2) and paired
// (2,1), (1,3), (1,2) steps from the constant bank and their descriptors from
// cpass, the pass descriptor passed by value; the two instantiations get
// their registers allocated separately.
template <int MINB, bool CBANK>
__global__ void __launch_bounds__(PASS_THREADS, MINB)
pass_kernel(const DevPass *__restrict__ gpass, const int *__restrict__ chunks,
            const DevBranch *__restrict__ branches, const float2 *__restrict__ pool,
            const float2 *__restrict__ in, float2 *__restrict__ out, BatchArgs ba,
            const __grid_constant__ DevPass cpass) {
    extern __shared__ __align__(16) unsigned char smem[];
    DevPass &P = *reinterpret_cast<DevPass *>(smem);
    const int n_steps_g = gpass->n_steps;
    {
        const int4 *src = reinterpret_cast<const int4 *>(gpass);
        int4 *dst = reinterpret_cast<int4 *>(smem);
        const int n16 = (int)((PASS_HEAD_BYTES + (size_t)n_steps_g * sizeof(DevStep)) / 16);
        for (int i = threadIdx.x; i < n16; i += PASS_THREADS) dst[i] = src[i];
    }
    __syncthreads();
    const size_t head = PASS_HEAD_BYTES + (size_t)P.n_steps * sizeof(DevStep);
    int *cin_tab = reinterpret_cast<int *>(smem + head);
    const int n_cin = 1 << (P.t_in - P.c_in), n_cout = 1 << (P.t_out - P.c_out);
    int *cout_tab = cin_tab + n_cin;
    // tile buffer b (0 or 1) starts at tbuf + b * tile_max
    float2 *tbuf = reinterpret_cast<float2 *>(smem + head + (size_t)((n_cin + n_cout + 3) & ~3) * 4);
    const int tile_max = P.tile_max;
    float2 *bm = tbuf + 2 * tile_max;
    for (int i = threadIdx.x; i < n_cin; i += PASS_THREADS) cin_tab[i] = chunks[P.chunk_in_base + i];
    for (int i = threadIdx.x; i < n_cout; i += PASS_THREADS) cout_tab[i] = chunks[P.chunk_out_base + i];
    // offsets of each step's branch matrix in bm
    __shared__ int bm_off[MAX_PASS_STEPS];
    if (threadIdx.x == 0) {
        int o = 0;
        for (int t = 0; t < P.n_steps; ++t) {
            bm_off[t] = o;
            if (P.steps[t].branch >= 0) o += 1 << (P.steps[t].k + P.steps[t].n);
        }
    }
    const int64_t n_units = (int64_t)ba.n_items * P.n_tiles;
    const int64_t base = ba.state->slice_base;
    const int64_t send = ba.state->slice_end;
    const int tin_n = 1 << P.t_in, tout_n = 1 << P.t_out;
    const int c_in = P.c_in, c_out = P.c_out;
    const int cin_mask = (1 << c_in) - 1, cout_mask = (1 << c_out) - 1;
    const int nfree = P.n_free;
    const unsigned lane = threadIdx.x & 31;
    // this lane's free bit (free bits are disjoint, so offsets combine with OR)
    const unsigned my_fin = lane < (unsigned)nfree ? (unsigned)P.free_in[lane] : 0u;
    const unsigned my_fout = lane < (unsigned)nfree ? (unsigned)P.free_out[lane] : 0u;
    const int st_lo = P.st_lo[threadIdx.x & 63];
    const bool st_pair = c_out >= 1 && P.st_lo[1] == 1;
    __syncthreads();
    // per-thread parts of the load and paired-store offsets (idx = 2 tid + 512 j;
    // the chunk tables are complete after the barrier above)
    const int ld_i0 = 2 * threadIdx.x;
    const int ld_off0 = (ld_i0 < tin_n) ? cin_tab[ld_i0 >> c_in] + (ld_i0 & cin_mask) : 0;
    const int ld_sw0 = dev_swizzle(ld_i0);
    const int st_off0 = (ld_i0 < tout_n) ? cout_tab[ld_i0 >> c_out] + (ld_i0 & cout_mask) : 0;
    const int st_t0 = (ld_i0 < tout_n) ? (P.st_lo[ld_i0 & 63] ^ P.st_hi[ld_i0 >> 6]) : 0;
    // unit u -> (batch item, prefix, slice); invalid past the slice range
    const int SB = ba.SB;
    auto unit_item = [&](int64_t u, int &item, int &p, int64_t &s) {
        item = (int)(u >> nfree);
        const int pl = (SB == 1) ? item : item / SB;
        p = ba.p0 + pl;
        s = base + (item - pl * SB);
        return s < send;
    };
    // issue the cp.async copies of unit u's input tile into buffer dstb:
    // entry pairs (the low input bit is a chunk bit, so pairs are contiguous
    // in HBM, and the swizzle keeps them adjacent in the tile)
    auto issue_load = [&](int64_t u, float2 *dstb) {
        int item, p;
        int64_t s;
        if (!unit_item(u, item, p, s)) return;
        const unsigned tile = (unsigned)(u & (P.n_tiles - 1));
        const unsigned ib = __reduce_or_sync(0xffffffffu, ((tile >> lane) & 1u) ? my_fin : 0u);
        const float2 *src = (P.in_branch >= 0) ? pool + branch_offset(branches[P.in_branch], p, s)
                                               : in + (int64_t)item * P.in_item_stride;
        src += ib;
        if (c_in >= 1) {
            // idx = 2 tid + 512 j: the chunk table and the swizzle are linear
            // over disjoint bits, so the thread's part is fixed per pass and
            // each j adds one block-uniform term
            if (ld_i0 < tin_n) {
                const float2 *s0 = src + ld_off0;
#pragma unroll
                for (int j = 0; j < (1 << MAX_TILE_BITS) / (2 * PASS_THREADS); ++j)
                    if ((j << 9) < tin_n)
                        cp_async16(dstb + (ld_sw0 ^ dev_swizzle(j << 9)), s0 + cin_tab[(j << 9) >> c_in]);
            }
        } else {
            for (int idx = threadIdx.x; idx < tin_n; idx += PASS_THREADS)
                cp_async8(dstb + dev_swizzle(idx), src + cin_tab[idx >> c_in] + (idx & cin_mask));
        }
    };
    int last_item = -1;
    int buf = 0;
    if ((int64_t)blockIdx.x < n_units) issue_load(blockIdx.x, tbuf);
    cp_async_commit();
    for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x, buf ^= 1) {
        if (u + gridDim.x < n_units) issue_load(u + gridDim.x, tbuf + (buf ^ 1) * tile_max);
        cp_async_commit();
        cp_async_wait_prev();
        int item, p;
        int64_t s;
        const bool valid = unit_item(u, item, p, s);  // uniform over the block
        if (valid && item != last_item) {
            for (int t = 0; t < P.n_steps; ++t) {
                const int br = P.steps[t].branch;
                if (br < 0) continue;
                const float2 *bsrc = pool + branch_offset(branches[br], p, s);
                const int cnt = 1 << (P.steps[t].k + P.steps[t].n);
                const int bo = bm_off[t];
                for (int i = threadIdx.x; i < cnt; i += PASS_THREADS) bm[bo + i] = bsrc[i];
            }
            last_item = item;
        }
        __syncthreads();
        if (valid) {
            float2 *tile = tbuf + buf * tile_max;
            if constexpr (CBANK) {
                run_steps_const<0>(tile, P, cpass, bm, bm_off, PASS_THREADS);
            } else {
                for (int t = 0; t < P.n_steps; ++t) {
                    if (P.steps[t].branch < 0) continue;
                    run_step(tile, P.steps[t], bm + bm_off[t], PASS_THREADS);
                    __syncthreads();
                }
            }
            const unsigned tl = (unsigned)(u & (P.n_tiles - 1));
            const unsigned ob = __reduce_or_sync(0xffffffffu, ((tl >> lane) & 1u) ? my_fout : 0u);
            float2 *dst = out + (int64_t)item * P.out_item_stride + ob;
            if (st_pair) {
                // output bit 0 is tile position 0: entry pairs move as 16 bytes
                float2 *d0 = dst + st_off0;
                if (ld_i0 < tout_n) {
#pragma unroll
                    for (int j = 0; j < (1 << MAX_TILE_BITS) / (2 * PASS_THREADS); ++j)
                        if ((j << 9) < tout_n)
                            *reinterpret_cast<float4 *>(d0 + cout_tab[(j << 9) >> c_out]) =
                                *reinterpret_cast<const float4 *>(tile + (st_t0 ^ cpass.st_hi[j << 3]));
                }
            } else {
                for (int idx = threadIdx.x; idx < tout_n; idx += PASS_THREADS)
                    dst[cout_tab[idx >> c_out] + (idx & cout_mask)] = tile[st_lo ^ P.st_hi[idx >> 6]];
            }
        }
        __syncthreads();
    }
    cp_async_wait_all();
}

bool pass_uses_const_bank(const DevPass &h_pass, const BatchArgs &ba) {
    if (ba.n_items != 1) return false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= CB_MAX_DEV) return false;
    {
        std::lock_guard<std::recursive_mutex> lk(g_cb_mutex);
        if (!g_bm_stage_dev[dev]) return false;
    }
    return pass_has_const_steps(h_pass);
}

ConstBankOrder::ConstBankOrder(cudaStream_t st) : st_(st) {
    g_cb_mutex.lock();
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    int dev = 0;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone &&
        cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < CB_MAX_DEV && g_cb_event[dev]) {
        ev_ = g_cb_event[dev];
        if (cudaStreamWaitEvent(st, ev_, 0) != cudaSuccess) ev_ = nullptr;
    }
    cudaGetLastError();
}

ConstBankOrder::~ConstBankOrder() {
    if (ev_) cudaEventRecord(ev_, st_);
    g_cb_mutex.unlock();
}

static size_t pass_smem_bytes(const DevPass &P) {
    size_t b = PASS_HEAD_BYTES + (size_t)P.n_steps * sizeof(DevStep);
    b += (size_t)((((1 << (P.t_in - P.c_in)) + (1 << (P.t_out - P.c_out))) + 3) & ~3) * 4;
    b += 2 * (size_t)P.tile_max * sizeof(float2);
    for (int t = 0; t < P.n_steps; ++t)
        if (P.steps[t].branch >= 0) b += ((size_t)1 << (P.steps[t].k + P.steps[t].n)) * sizeof(float2);
    return b;
}

cudaError_t launch_pass(const DevPass *d_pass, const DevPass &h_pass, const int *d_chunks,
                        const DevBranch *d_branches, const DevBranch *h_branches,
                        const float2 *pool, const float2 *in, float2 *out, BatchArgs ba,
                        cudaStream_t st) {
    (void)h_branches;
    static int num_sms = 0;
    if (!num_sms) {
        int dev;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const size_t smem = pass_smem_bytes(h_pass);
    // three blocks per SM (registers capped at 80) measured faster than two
    // blocks with 96 registers; the 96-register variant is used only when the
    // tile's shared memory does not fit three blocks
    const bool cbank = pass_uses_const_bank(h_pass, ba);
    auto k3 = cbank ? &pass_kernel<3, true> : &pass_kernel<3, false>;
    auto k2 = cbank ? &pass_kernel<2, true> : &pass_kernel<2, false>;
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k3, PASS_THREADS, smem);
    if (e != cudaSuccess) return e;
    const bool small_tile = occ >= 3;
    if (!small_tile) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k2, PASS_THREADS, smem);
        if (e != cudaSuccess) return e;
    }
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int64_t units = (int64_t)ba.n_items * h_pass.n_tiles;
    if (cbank) {
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        stage_bm_kernel<<<1, 64, 0, st>>>(d_pass, d_branches, pool, ba);
        e = cudaMemcpyToSymbolAsync(c_bm, g_bm_stage_dev[dev], sizeof(float2) * CB_ENTRIES, 0,
                                    cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyToSymbolAsync(c_bm2, g_bm2_stage_dev[dev], sizeof(float4) * CB_ENTRIES, 0,
                                    cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(units, (int64_t)num_sms * occ));
    (small_tile ? k3 : k2)<<<(unsigned)grid, PASS_THREADS, smem, st>>>(d_pass, d_chunks, d_branches, pool,
                                                                       in, out, ba, h_pass);
    return cudaGetLastError();
}

// ------------------------------------------------------- small contraction
// Branch pre-computation (Supp. A.3): one pairwise step on small tensors in
// FP64, C[o] = sum_c A[ia(o) + ja(c)] * B[ib(o) + jb(c)]; B == nullptr means
// a permutation of A. The result is stored in FP64 (Cd) or rounded to FP32
// (Cf) when it is a finished branch.
__global__ void small_contract_kernel(const double2 *__restrict__ A, const double2 *__restrict__ B,
                                      double2 *__restrict__ Cd, float2 *__restrict__ Cf,
                                      SmallContract d, int64_t sA, int64_t sB, int64_t sC) {
    // batch item blockIdx.y: operands at item * stride (stride 0: shared)
    A += blockIdx.y * sA;
    if (B) B += blockIdx.y * sB;
    if (Cd) Cd += blockIdx.y * sC;
    if (Cf) Cf += blockIdx.y * sC;
    const int64_t nout = (int64_t)1 << d.rc;
    const int64_t nsum = (int64_t)1 << d.k;
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < nout;
         o += (int64_t)gridDim.x * blockDim.x) {
        int64_t ia = 0, ib = 0;
        for (int j = 0; j < d.rc; ++j) {
            if (!((o >> j) & 1)) continue;
            if (d.a_out[j] >= 0) ia += (int64_t)1 << d.a_out[j];
            if (d.b_out[j] >= 0) ib += (int64_t)1 << d.b_out[j];
        }
        double re, im;
        if (!B) {
            re = A[ia].x;
            im = A[ia].y;
        } else {
            re = 0.0;
            im = 0.0;
            for (int64_t c = 0; c < nsum; ++c) {
                int64_t ja = ia, jb = ib;
                for (int t = 0; t < d.k; ++t)
                    if ((c >> t) & 1) {
                        ja += (int64_t)1 << d.a_k[t];
                        jb += (int64_t)1 << d.b_k[t];
                    }
                const double2 a = A[ja], b = B[jb];
                re = fma(a.x, b.x, re);
                re = fma(-a.y, b.y, re);
                im = fma(a.x, b.y, im);
                im = fma(a.y, b.x, im);
            }
        }
        if (Cf)
            Cf[o] = make_float2((float)re, (float)im);
        else
            Cd[o] = make_double2(re, im);
    }
}

cudaError_t launch_small_contract(const double2 *A, const double2 *B, double2 *Cd, float2 *Cf,
                                  const SmallContract &d, cudaStream_t st) {
    return launch_small_contract_batched(A, 0, B, 0, Cd, Cf, 0, 1, d, st);
}

cudaError_t launch_small_contract_batched(const double2 *A, int64_t sA, const double2 *B, int64_t sB,
                                          double2 *Cd, float2 *Cf, int64_t sC, int items,
                                          const SmallContract &d, cudaStream_t st) {
    if (items < 1 || items > 65535) return cudaErrorInvalidValue;
    const int64_t nout = (int64_t)1 << d.rc;
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((nout + threads - 1) / threads, 4096);
    dim3 grid((unsigned)std::max<int64_t>(blocks, 1), (unsigned)items, 1);
    small_contract_kernel<<<grid, threads, 0, st>>>(A, B, Cd, Cf, d, sA, sB, sC);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- SIMT GEMM
// C[m][nu] = sum_kappa A[m][kappa] * B[kappa][nu] for one batch item per
// blockIdx.z. A block computes a BM x BN tile (BN = min(N, 256), BM =
// min(4096 / BN, 512)), staging 8-wide slabs of A and B in shared memory;
// thread t owns outputs t + 256 i.
constexpr int G_THREADS = 256;
constexpr int G_BK = 8;

struct GemmItemSrc {
    // A / C base per item: base + item * stride; B per item from the branch
    // table (stem steps) or base + item * strideB (plain GEMM).
    const float2 *A;
    float2 *C;
    const float2 *B;
    int64_t sA, sB, sC;
    const DevBranch *br;  // non-null: B from branch storage
    const float2 *pool;
    BatchArgs ba;
    int use_batch;        // 1: items follow BatchArgs (slices/prefixes)
};

__global__ void __launch_bounds__(G_THREADS)
cgemm_simt_kernel(GemmItemSrc g, int64_t M, int K, int N, int BM, int BN) {
    extern __shared__ __align__(16) float2 gsm[];
    float2 *As = gsm;                      // BM x (BK + 1)
    float2 *Bs = gsm + BM * (G_BK + 1);    // BK x BN
    const int64_t item = blockIdx.z;
    const float2 *A = g.A + item * g.sA;
    float2 *C = g.C + item * g.sC;
    const float2 *B;
    if (g.use_batch) {
        const int pl = (int)(item / g.ba.SB);
        const int64_t s = g.ba.state->slice_base + (item - (int64_t)pl * g.ba.SB);
        if (s >= g.ba.state->slice_end) return;
        B = g.br ? g.pool + branch_offset(*g.br, g.ba.p0 + pl, s) : g.B + item * g.sB;
    } else {
        B = g.B + item * g.sB;
    }
    const int64_t m0 = (int64_t)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    const int nout = BM * BN;
    float2 acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < K; k0 += G_BK) {
        const int bk = min(G_BK, K - k0);
        for (int i = threadIdx.x; i < BM * bk; i += G_THREADS) {
            const int r = i / bk, c = i % bk;
            const int64_t m = m0 + r;
            As[r * (G_BK + 1) + c] = (m < M) ? A[m * K + k0 + c] : make_float2(0.f, 0.f);
        }
        for (int i = threadIdx.x; i < bk * BN; i += G_THREADS) {
            const int r = i / BN, c = i % BN;
            Bs[r * BN + c] = (n0 + c < N) ? B[(int64_t)(k0 + r) * N + n0 + c] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int o = threadIdx.x + i * G_THREADS;
            if (o < nout) {
                const int r = o / BN, c = o % BN;
                float2 a = acc[i];
                for (int kk = 0; kk < bk; ++kk) cfma(a, As[r * (G_BK + 1) + kk], Bs[kk * BN + c]);
                acc[i] = a;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int o = threadIdx.x + i * G_THREADS;
        if (o < nout) {
            const int r = o / BN, c = o % BN;
            const int64_t m = m0 + r;
            if (m < M && n0 + c < N) C[m * N + n0 + c] = acc[i];
        }
    }
}

// Small K, N (branch absorption: K, N <= 8): a streaming kernel. Each thread
// owns one row m: it reads A[m][0..K) (16-byte loads when rows and bases are
// 16-byte aligned), multiplies by the K x N matrix held in shared memory and
// writes C[m][0..N). The FMAs run in the order of cgemm_simt_kernel (kappa
// ascending per output), so both kernels give identical results.
template <int K, int N>
__global__ void __launch_bounds__(G_THREADS) cgemm_rows_kernel(GemmItemSrc g, int64_t M, int vec_a,
                                                               int vec_c) {
    __shared__ float2 Bs[K * N];
    const int64_t item = blockIdx.y;
    const float2 *B;
    if (g.use_batch) {
        const int pl = (int)(item / g.ba.SB);
        const int64_t s = g.ba.state->slice_base + (item - (int64_t)pl * g.ba.SB);
        if (s >= g.ba.state->slice_end) return;  // uniform over the block
        B = g.br ? g.pool + branch_offset(*g.br, g.ba.p0 + pl, s) : g.B + item * g.sB;
    } else {
        B = g.B + item * g.sB;
    }
    for (int i = threadIdx.x; i < K * N; i += G_THREADS) Bs[i] = B[i];
    __syncthreads();
    const float2 *A = g.A + item * g.sA;
    float2 *C = g.C + item * g.sC;
    for (int64_t m = (int64_t)blockIdx.x * G_THREADS + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * G_THREADS) {
        float2 x[K];
        if (K % 2 == 0 && vec_a) {
            const float4 *a4 = reinterpret_cast<const float4 *>(A + m * K);
#pragma unroll
            for (int j = 0; j < K / 2; ++j) {
                const float4 v = a4[j];
                x[2 * j] = make_float2(v.x, v.y);
                x[2 * j + 1] = make_float2(v.z, v.w);
            }
        } else {
#pragma unroll
            for (int j = 0; j < K; ++j) x[j] = A[m * K + j];
        }
        float2 y[N];
#pragma unroll
        for (int c = 0; c < N; ++c) {
            float2 a = make_float2(0.f, 0.f);
#pragma unroll
            for (int kk = 0; kk < K; ++kk) cfma(a, x[kk], Bs[kk * N + c]);
            y[c] = a;
        }
        if (N % 2 == 0 && vec_c) {
            float4 *c4 = reinterpret_cast<float4 *>(C + m * N);
#pragma unroll
            for (int j = 0; j < N / 2; ++j) c4[j] = make_float4(y[2 * j].x, y[2 * j].y, y[2 * j + 1].x, y[2 * j + 1].y);
        } else {
#pragma unroll
            for (int c = 0; c < N; ++c) C[m * N + c] = y[c];
        }
    }
}

template <int K>
static void launch_rows_n(int N, dim3 grid, const GemmItemSrc &g, int64_t M, int va, int vc,
                          cudaStream_t st) {
    switch (N) {
        case 1: cgemm_rows_kernel<K, 1><<<grid, G_THREADS, 0, st>>>(g, M, va, vc); break;
        case 2: cgemm_rows_kernel<K, 2><<<grid, G_THREADS, 0, st>>>(g, M, va, vc); break;
        case 4: cgemm_rows_kernel<K, 4><<<grid, G_THREADS, 0, st>>>(g, M, va, vc); break;
        default: cgemm_rows_kernel<K, 8><<<grid, G_THREADS, 0, st>>>(g, M, va, vc); break;
    }
}

static bool pow2_upto8(int64_t x) { return x == 1 || x == 2 || x == 4 || x == 8; }

static cudaError_t run_simt_gemm(const GemmItemSrc &g, int64_t M, int64_t K, int64_t N,
                                 int64_t batch, cudaStream_t st) {
    if (K <= 0 || N <= 0 || M <= 0 || batch <= 0) return cudaSuccess;
    if (batch > 65535) return cudaErrorInvalidValue;
    if (pow2_upto8(K) && pow2_upto8(N)) {
        // 16-byte vector access needs 16-byte aligned rows and item bases
        auto al16 = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
        const int va = al16(g.A) && (K % 2 == 0) && (g.sA % 2 == 0);
        const int vc = al16(g.C) && (N % 2 == 0) && (g.sC % 2 == 0);
        const int64_t blocks = std::min<int64_t>((M + G_THREADS - 1) / G_THREADS, (int64_t)1 << 20);
        dim3 grid((unsigned)blocks, (unsigned)batch, 1);
        switch (K) {
            case 1: launch_rows_n<1>((int)N, grid, g, M, va, vc, st); break;
            case 2: launch_rows_n<2>((int)N, grid, g, M, va, vc, st); break;
            case 4: launch_rows_n<4>((int)N, grid, g, M, va, vc, st); break;
            default: launch_rows_n<8>((int)N, grid, g, M, va, vc, st); break;
        }
        return cudaGetLastError();
    }
    const int BN = (int)std::min<int64_t>(N, 256);
    const int BM = std::min(4096 / BN, 512);
    const int64_t gx = (M + BM - 1) / BM;
    const int64_t gy = (N + BN - 1) / BN;
    if (gx > 0x7fffffffLL || gy > 65535) return cudaErrorInvalidValue;
    const size_t smem = ((size_t)BM * (G_BK + 1) + (size_t)G_BK * BN) * sizeof(float2);
    dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)batch);
    cgemm_simt_kernel<<<grid, G_THREADS, smem, st>>>(g, M, (int)K, (int)N, BM, BN);
    return cudaGetLastError();
}

cudaError_t launch_stem_gemm(const float2 *A, float2 *C, int64_t M, int k, int n, int64_t strideA,
                             int64_t strideC, const DevBranch *d_branch_entry, const float2 *pool,
                             BatchArgs ba, tn_precision prec, cudaStream_t st) {
    if (prec != TN_PREC_FP32_SIMT) {
        if (!tc_gemm_supported(k, n) && !(ba.n_items == 1 && tc_large_stem_supported(M, k, n, prec, A, C)))
            return cudaErrorNotSupported;
        return launch_tc_stem_gemm(A, C, M, k, n, strideA, strideC, d_branch_entry, pool, ba, prec, st);
    }
    GemmItemSrc g{A, C, nullptr, strideA, 0, strideC, d_branch_entry, pool, ba, 1};
    return run_simt_gemm(g, M, (int64_t)1 << k, (int64_t)1 << n, ba.n_items, st);
}

cudaError_t launch_cgemm(const float2 *A, const float2 *B, float2 *C, int64_t M, int64_t K,
                         int64_t N, int64_t batch, int64_t sA, int64_t sB, int64_t sC,
                         tn_precision prec, cudaStream_t st) {
    if (prec != TN_PREC_FP32_SIMT) return launch_tc_cgemm(A, B, C, M, K, N, batch, sA, sB, sC, prec, st);
    GemmItemSrc g{A, C, B, sA, sB, sC, nullptr, nullptr, BatchArgs{nullptr, 1, 0, 0}, 0};
    return run_simt_gemm(g, M, K, N, batch, st);
}

// ---------------------------------------------------- slice sum (FP64)
// Neumaier-compensated running sum, per component.
__device__ __forceinline__ void neumaier(double &sum, double &comp, double v) {
    const double t = sum + v;
    if (fabs(sum) >= fabs(v))
        comp += (sum - t) + v;
    else
        comp += (v - t) + sum;
    sum = t;
}

// One thread per (prefix, open index): adds the batch's slices in slice order.
__global__ void accumulate_kernel(const float2 *__restrict__ fin, int n_open,
                                  const int *__restrict__ pos, double2 *sum, double2 *comp,
                                  BatchArgs ba, int n_prefix_launch, int total_prefix_stride) {
    const int nb = 1 << n_open;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= n_prefix_launch * nb) return;
    const int pl = tid / nb, o = tid % nb;
    int idx = 0;
    for (int i = 0; i < n_open; ++i)
        if ((o >> (n_open - 1 - i)) & 1) idx += 1 << pos[i];
    const int64_t base = ba.state->slice_base, send = ba.state->slice_end;
    const int64_t gi = (int64_t)(ba.p0 + pl) * nb + o;
    (void)total_prefix_stride;
    double sr = sum[gi].x, si = sum[gi].y, cr = comp[gi].x, ci = comp[gi].y;
    for (int j = 0; j < ba.SB; ++j) {
        if (base + j >= send) break;
        const float2 v = fin[((int64_t)pl * ba.SB + j) * nb + idx];
        neumaier(sr, cr, (double)v.x);
        neumaier(si, ci, (double)v.y);
    }
    sum[gi] = make_double2(sr, si);
    comp[gi] = make_double2(cr, ci);
}

cudaError_t launch_accumulate(const float2 *fin, int n_open, const int *d_pos, double2 *sum,
                              double2 *comp, BatchArgs ba, int n_prefix_launch, cudaStream_t st) {
    const int n = n_prefix_launch << n_open;
    accumulate_kernel<<<(n + 127) / 128, 128, 0, st>>>(fin, n_open, d_pos, sum, comp, ba,
                                                       n_prefix_launch, 0);
    return cudaGetLastError();
}

__global__ void advance_kernel(DevState *s, int64_t by) { s->slice_base += by; }

cudaError_t launch_advance(DevState *state, int64_t by, cudaStream_t st) {
    advance_kernel<<<1, 1, 0, st>>>(state, by);
    return cudaGetLastError();
}

__global__ void finalize_kernel(const double2 *sum, const double2 *comp, double2 *out, int64_t n,
                                int accumulate) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 v = make_double2(sum[i].x + comp[i].x, sum[i].y + comp[i].y);
    if (accumulate) {
        v.x += out[i].x;
        v.y += out[i].y;
    }
    out[i] = v;
}

cudaError_t launch_finalize(const double2 *sum, const double2 *comp, double2 *out, int64_t n,
                            int accumulate, cudaStream_t st) {
    finalize_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(sum, comp, out, n, accumulate);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ XEB
// Sum of |amp|^2 in FP64: block tree reduction, then one compensated pass
// over the block partials by a single thread (deterministic order).
__global__ void xeb_partial_kernel(const double2 *__restrict__ a, int64_t n, double *part) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        acc += a[i].x * a[i].x + a[i].y * a[i].y;
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void xeb_final_kernel(const double *part, int nb, double *out) {
    double s = 0.0, c = 0.0;
    for (int i = 0; i < nb; ++i) neumaier(s, c, part[i]);
    *out = s + c;
}

cudaError_t launch_xeb_sum(const double2 *amps, int64_t n, double *out_sum, cudaStream_t st) {
    // out_sum must have room for 1 + 256 doubles: [result, partials...]
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(256, (n + 255) / 256));
    xeb_partial_kernel<<<nb, 256, 0, st>>>(amps, n, out_sum + 1);
    xeb_final_kernel<<<1, 1, 0, st>>>(out_sum + 1, nb, out_sum);
    return cudaGetLastError();
}

// --------------------------------------------------- FP32 FMA peak probe
// Independent FMA chains, enough per thread and enough threads per SM that
// the FP32 pipes never wait on a result: the rate this GPU reaches on plain
// FP32 FMAs (the arithmetic the fused stem pass runs on). Each thread keeps
// FMA_CHAINS accumulators and runs FMA_ITERS rounds; the sum goes to out
// only if it equals a value it cannot reach, which keeps the work live.
constexpr int FMA_CHAINS = 16;
constexpr int FMA_ITERS = 16384;
__global__ void __launch_bounds__(256) fma_peak_kernel(float seed, float *out) {
    float a[FMA_CHAINS];
#pragma unroll
    for (int i = 0; i < FMA_CHAINS; ++i) a[i] = seed + (float)(threadIdx.x + i);
    const float b = 0.999999f, c = 1e-7f;
    for (int it = 0; it < FMA_ITERS; ++it) {
#pragma unroll
        for (int i = 0; i < FMA_CHAINS; ++i) a[i] = fmaf(a[i], b, c);
    }
    float t = 0.f;
#pragma unroll
    for (int i = 0; i < FMA_CHAINS; ++i) t += a[i];
    if (t == -1.2345e30f) out[blockIdx.x] = t;
}

cudaError_t measure_fma_peak(cudaStream_t st, double *tflops, int *sm_count) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = sms * 8;  // 8 blocks of 256 threads per SM: 64 warps
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // first launch warms up
        cudaEventRecord(e0, st);
        fma_peak_kernel<<<blocks, 256, 0, st>>>(1.0f, nullptr);
        cudaEventRecord(e1, st);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && e == cudaSuccess) best = std::min(best, ms);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * FMA_CHAINS * (double)FMA_ITERS * 256.0 * blocks;
    *tflops = flops / (best * 1e-3) / 1e12;
    *sm_count = sms;
    return cudaSuccess;
}

// ------------------------------------------------------- frugal sampling
// Frugal rejection sampling (Sec. 2): one warp per batch of K candidate
// amplitudes. Candidate j is accepted when u[j] < 2^n p / M with
// p = re*re + im*im, each operation rounded on its own (no fused
// multiply-add), so the decision matches an FP64 evaluation of the same
// expression. The batch's sample is the accepted candidate with the smallest
// key (a random visiting order; equal keys go to the lower j).
__global__ void frugal_sample_kernel(const double2 *__restrict__ amps, const double *__restrict__ u,
                                     const double *__restrict__ key, int64_t B, int K, double N,
                                     double M, int32_t *__restrict__ idx, int32_t *__restrict__ cnt,
                                     double2 *__restrict__ picked) {
    const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= B) return;  // uniform over the warp
    const double2 *a = amps + b * K;
    const double *ub = u + b * K, *kb = key + b * K;
    double best_key = 0.0;
    int best_j = -1, c = 0;
    for (int j = lane; j < K; j += 32) {
        const double2 v = a[j];
        const double p = __dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y));
        const double thr = __ddiv_rn(__dmul_rn(p, N), M);
        if (ub[j] < thr) {
            ++c;
            const double k = kb[j];
            if (best_j < 0 || k < best_key) {  // j ascends per lane: ties keep the lower j
                best_key = k;
                best_j = j;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ok = __shfl_xor_sync(0xffffffffu, best_key, o);
        const int oj = __shfl_xor_sync(0xffffffffu, best_j, o);
        if (oj >= 0 && (best_j < 0 || ok < best_key || (ok == best_key && oj < best_j))) {
            best_key = ok;
            best_j = oj;
        }
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
        idx[b] = best_j;
        cnt[b] = c;
        picked[b] = best_j >= 0 ? a[best_j] : make_double2(0.0, 0.0);
    }
}

cudaError_t launch_frugal_sample(const double2 *amps, const double *u, const double *key, int64_t B,
                                 int K, int n_qubits, double M, int32_t *idx, int32_t *cnt,
                                 double2 *picked, cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = (B * 32 + threads - 1) / threads;
    frugal_sample_kernel<<<(unsigned)blocks, threads, 0, st>>>(amps, u, key, B, K, std::ldexp(1.0, n_qubits),
                                                               M, idx, cnt, picked);
    return cudaGetLastError();
}

// ------------------------------------------------------------- permute
// Input bit j -> output bit perm[j]; read coalesced, write through a
// per-byte lookup of the destination offset.
__global__ void permute_kernel(const float2 *__restrict__ in, float2 *__restrict__ out, int rank,
                               const int *__restrict__ tab) {
    const int64_t n = (int64_t)1 << rank;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t o = 0;
        for (int b = 0; b < 4; ++b) o += (int64_t)(unsigned)tab[b * 256 + ((i >> (8 * b)) & 255)];
        out[o] = in[i];
    }
}

cudaError_t launch_permute(const float2 *in, float2 *out, int rank, const int *d_tab,
                           cudaStream_t st) {
    const int64_t n = (int64_t)1 << rank;
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((n + threads - 1) / threads, 152 * 16);
    permute_kernel<<<(unsigned)blocks, threads, 0, st>>>(in, out, rank, d_tab);
    return cudaGetLastError();
}

// Raise the dynamic shared-memory limits once, outside any stream capture.
cudaError_t init_kernels() {
    cudaError_t e = cudaSuccess;
    for (auto k : {&pass_kernel<2, false>, &pass_kernel<3, false>, &pass_kernel<2, true>, &pass_kernel<3, true>}) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
    }
    e = tc_gemm_init();
    if (e != cudaSuccess) return e;
    {
        // per device: the stage buffer's address and the event that orders
        // users of the constant-bank copy
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        std::lock_guard<std::recursive_mutex> lk(g_cb_mutex);
        if (dev >= 0 && dev < CB_MAX_DEV && !g_bm_stage_dev[dev]) {
            if (!g_cb_event[dev]) {
                e = cudaEventCreateWithFlags(&g_cb_event[dev], cudaEventDisableTiming);
                if (e != cudaSuccess) return e;
            }
            void *a = nullptr;
            e = cudaGetSymbolAddress(&a, g_bm_stage);
            if (e != cudaSuccess) return e;
            g_bm_stage_dev[dev] = static_cast<float2 *>(a);
            e = cudaGetSymbolAddress(&a, g_bm2_stage);
            if (e != cudaSuccess) return e;
            g_bm2_stage_dev[dev] = static_cast<float4 *>(a);
        }
    }
    return cudaFuncSetAttribute(cgemm_simt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                96 * 1024);
}

}  // namespace tn
