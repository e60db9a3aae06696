// Tensor-core (tcgen05) complex GEMM for stem steps that are dense
// contractions: C[m][nu] = sum_kappa A[m][kappa] * B[kappa][nu], complex64.
//
// The complex product is a real GEMM on the interleaved storage: A viewed as
// real [M][2K] (re/im as the fastest index) times the real 2K x 2N matrix
// [[Br, Bi], [-Bi, Br]] (arranged per (kappa, re/im) row and (nu, re/im)
// column) gives C as interleaved complex [M][2N]. Precision options split
// each FP32 operand into hi + lo parts of the tensor-core type and sum
// hi*hi + hi*lo + lo*hi (x3), or use one rounded product (x1), always with
// FP32 accumulation in tensor memory. In the x3 modes hi*hi accumulates in one
// TMEM region and the two correction products in a second one; the epilogue
// adds the two in FP32 with round-to-nearest. The tensor core's own FP32
// accumulation truncates toward zero, so every product chained into the
// accumulator that holds the full-size value costs a bias of about half an
// ulp; keeping the corrections (2^-11 smaller) apart leaves one such chain.
//
// One block of 128 threads computes a 128-row tile of C for one batch item
// and up to 256 real output columns: threads load A and B, split and write
// them to shared memory in the 128-byte-swizzled K-major layout, one thread
// issues tcgen05.mma into a TMEM accumulator, a commit arrives on an
// mbarrier, and the four warps read their 32 TMEM lanes back and store C.
// Every wait on the mbarrier is bounded; on time-out the block records an
// error code and skips its output.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "kernels.h"

namespace tn {

namespace {

constexpr int TC_THREADS = 128;
constexpr int TC_BM = 128;        // rows per block (MMA M)
constexpr int TC_MAX_N2 = 256;    // real output columns per block (MMA N)
constexpr int ATOM_BYTES = 1024;  // 8 rows x 128 B swizzle atom
constexpr uint32_t WAIT_LIMIT = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (row r, byte b within the 128-byte row) in a
// K-major tile of 128-byte rows with the 128-byte swizzle: the 16-byte chunk
// index is XORed with the row index modulo 8.
__device__ __forceinline__ uint32_t sw128(int r, int b) {
    return (uint32_t)(r * 128 + ((((b >> 4) ^ (r & 7)) & 7) << 4) + (b & 15));
}

// Shared-memory matrix descriptor: start address, leading byte offset
// (unused for swizzled K-major, 1), stride byte offset (one 8-row atom =
// 1024 B), descriptor version 1, layout 128-byte swizzle (2).
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((ATOM_BYTES >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: D = F32, A and B of type `ab` (TF32 = 2 for
// kind::tf32; BF16 = 1 for kind::f16), both K-major, N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t make_idesc(int ab, int n, int m) {
    return (1u << 4) | ((uint32_t)ab << 7) | ((uint32_t)ab << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
}

template <int KIND>  // 0: tf32, 1: bf16
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc,
                                    uint32_t accum) {
    if constexpr (KIND == 0) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
            "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
            "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
    }
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 32 lanes x 16 consecutive 32-bit TMEM columns into registers (warp-wide).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15}, [%16];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// Split an FP32 value into the tensor-core type: hi = x rounded to nearest,
// lo = the remainder rounded to nearest (x3 modes). Rounding both parts
// (rather than truncating) keeps the split unbiased, so errors of successive
// stem steps do not add up in one direction.
__device__ __forceinline__ float round_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo) {
    hi = round_tf32(x);
    lo = round_tf32(x - hi);
}
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

struct TcArgs {
    const float *A;  // real view [M][K2], item stride sA floats
    const float *B;  // complex [K][N] (interleaved), item stride sB complex entries
    float *C;        // real view [M][N2], item stride sC floats
    int64_t M;
    int K, N;        // complex sizes
    int64_t sA, sB, sC;
    const DevBranch *br;  // stem steps: B from branch storage of (prefix, slice)
    const float2 *pool;
    BatchArgs ba;
    int use_batch;
    int *err;
};

// PREC: 1 = TF32x3, 2 = BF16x3, 3 = BF16x1.
template <int PREC>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_cgemm_kernel(TcArgs g) {
    constexpr int KIND = (PREC == 1) ? 0 : 1;
    constexpr int ESZ = (KIND == 0) ? 4 : 2;       // bytes per tensor-core element
    constexpr int KC = 128 / ESZ;                  // K elements per 128-byte row
    constexpr int KSTEP = 32 / ESZ;                // K per MMA instruction
    constexpr bool X3 = PREC != 3;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned carve-out
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int N2 = 2 * g.N;
    const int n0 = blockIdx.z * TC_MAX_N2;               // first real output column
    const int nb = min(TC_MAX_N2, N2 - n0);              // real columns of this block
    const int nbp = (nb + 15) & ~15;                     // MMA N (multiple of 16)
    unsigned char *sAhi = sm;
    unsigned char *sAlo = sAhi + TC_BM * 128;
    unsigned char *sBhi = sAlo + (X3 ? TC_BM * 128 : 0);
    unsigned char *sBlo = sBhi + TC_MAX_N2 * 128;
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;

    const int64_t item = blockIdx.y;
    const float *A = g.A + item * g.sA;
    float *C = g.C + item * g.sC;
    const float *B;
    if (g.use_batch) {
        const int pl = (int)(item / g.ba.SB);
        const int64_t s = g.ba.state->slice_base + (item - (int64_t)pl * g.ba.SB);
        if (s >= g.ba.state->slice_end) return;  // uniform over the block
        int64_t o = g.br->base + (int64_t)(g.ba.p0 + pl) * g.br->prefix_stride;
        for (int i = 0; i < g.br->n_sl; ++i)
            if ((s >> g.br->sl_bit[i]) & 1) o += (int64_t)1 << g.br->sl_pos[i];
        B = reinterpret_cast<const float *>(g.pool + o);
    } else {
        B = g.B + item * 2 * g.sB;
    }
    const int64_t m0 = (int64_t)blockIdx.x * TC_BM;
    const int tid = threadIdx.x, warp = tid >> 5;

    uint32_t ncols = 32;
    while ((int)ncols < (X3 ? 2 : 1) * nbp) ncols <<= 1;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = make_idesc(KIND == 0 ? 2 : 1, nbp, TC_BM);
    const int K2 = 2 * g.K;
    uint32_t phase = 0;
    bool ok = true;
    int nchunk = (K2 + KC - 1) / KC;
    for (int ch = 0; ch < nchunk && ok; ++ch) {
        const int kbase = ch * KC;
        // A tile: 128 rows x KC elements of this chunk
        for (int i = tid; i < TC_BM * KC; i += TC_THREADS) {
            const int r = i / KC, k = i % KC;
            const int64_t m = m0 + r;
            const int kk = kbase + k;
            const float x = (m < g.M && kk < K2) ? A[m * K2 + kk] : 0.f;
            const uint32_t off = sw128(r, k * ESZ);
            if constexpr (KIND == 0) {
                float hi, lo;
                split_tf32(x, hi, lo);
                if constexpr (PREC == 1) {
                    *reinterpret_cast<float *>(sAhi + off) = hi;
                    *reinterpret_cast<float *>(sAlo + off) = lo;
                }
            } else {
                __nv_bfloat16 hi, lo;
                split_bf16(x, hi, lo);
                *reinterpret_cast<__nv_bfloat16 *>(sAhi + off) = hi;
                if constexpr (X3) *reinterpret_cast<__nv_bfloat16 *>(sAlo + off) = lo;
            }
        }
        // B tile (K-major: one 128-byte row per real output column j):
        // Br_real[(kappa, c)][(nu, d)] = c == d ? Re B : (c == 1 ? -Im B : Im B)
        for (int i = tid; i < nbp * KC; i += TC_THREADS) {
            const int j = i / KC, k = i % KC;
            const int jj = n0 + j, kk = kbase + k;
            float v = 0.f;
            if (jj < N2 && kk < K2) {
                const int nu = jj >> 1, d = jj & 1, kap = kk >> 1, c = kk & 1;
                const float re = B[2 * ((int64_t)kap * g.N + nu)];
                const float im = B[2 * ((int64_t)kap * g.N + nu) + 1];
                v = (c == d) ? re : (c == 1 ? -im : im);
            }
            const uint32_t off = sw128(j, k * ESZ);
            if constexpr (KIND == 0) {
                float hi, lo;
                split_tf32(v, hi, lo);
                *reinterpret_cast<float *>(sBhi + off) = hi;
                *reinterpret_cast<float *>(sBlo + off) = lo;
            } else {
                __nv_bfloat16 hi, lo;
                split_bf16(v, hi, lo);
                *reinterpret_cast<__nv_bfloat16 *>(sBhi + off) = hi;
                if constexpr (X3) *reinterpret_cast<__nv_bfloat16 *>(sBlo + off) = lo;
            }
        }
        // make the generic-proxy writes visible to the tensor core
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            for (int ks = 0; ks < KC / KSTEP; ++ks) {
                const uint32_t kb = (uint32_t)(ks * 32);
                const uint64_t ahi = make_desc(smem_u32(sAhi) + kb);
                const uint64_t bhi = make_desc(smem_u32(sBhi) + kb);
                const uint32_t first = (ch == 0 && ks == 0) ? 0u : 1u;
                mma<KIND>(tmem, ahi, bhi, idesc, first);
                if constexpr (X3) {  // corrections in their own accumulator
                    const uint64_t alo = make_desc(smem_u32(sAlo) + kb);
                    const uint64_t blo = make_desc(smem_u32(sBlo) + kb);
                    mma<KIND>(tmem + (uint32_t)nbp, ahi, blo, idesc, first);
                    mma<KIND>(tmem + (uint32_t)nbp, alo, bhi, idesc, 1u);
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    smem_u32(&mbar)));
        }
        // all threads wait until the MMAs have consumed this chunk
        ok = mbar_wait(smem_u32(&mbar), phase);
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        __syncthreads();
    }
    if (!ok) {
        if (tid == 0) atomicExch(g.err, 5);
        // give MMAs still in flight a second bounded wait before TMEM is freed
        mbar_wait(smem_u32(&mbar), phase ^ 1u);
    } else {
        // epilogue: warp w reads TMEM lanes 32w..32w+31 (rows), 16 columns at a time
        const int64_t row = m0 + warp * 32 + (tid & 31);
        for (int c0 = 0; c0 < nbp; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            tmem_ld16(taddr, v);
            if constexpr (X3) {
                uint32_t w[16];
                tmem_ld16(taddr + (uint32_t)nbp, w);
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    v[q] = __float_as_uint(__fadd_rn(__uint_as_float(v[q]), __uint_as_float(w[q])));
            }
            if (row < g.M) {
                for (int q = 0; q < 16; ++q) {
                    const int col = n0 + c0 + q;
                    if (c0 + q < nb && col < N2) C[row * N2 + col] = __uint_as_float(v[q]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols));
}

// Persistent variant for the stem's tall-skinny shapes (2K <= 64 real
// columns of A, 2N <= 256): each block builds the split B once per batch item,
// keeps two A stages and two TMEM accumulators, and walks 128-row tiles
// t = blockIdx.x, blockIdx.x + gridDim.x, ... over (item, row tile). While the
// tensor core multiplies tile i, the threads load and split tile i+1 into the
// other stage; the epilogue of tile i overlaps the MMAs of tile i+1.
constexpr int P_K2MAX = 64;
// dynamic shared memory allowed per block (opt-in limit minus the static
// barriers), set by tc_gemm_init from the device attribute
size_t P_SMEM_MAX = 200 * 1024;

template <int PREC>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_cgemm_persistent(TcArgs g, int64_t n_items) {
    constexpr int KIND = (PREC == 1) ? 0 : 1;
    constexpr int ESZ = (KIND == 0) ? 4 : 2;
    constexpr int KC = 128 / ESZ;        // elements per 128-byte row block
    constexpr int KSTEP = 32 / ESZ;
    constexpr bool X3 = PREC != 3;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int K2 = 2 * g.K, N2 = 2 * g.N;
    const int nbp = (N2 + 15) & ~15;
    const int kblocks = (K2 + KC - 1) / KC;               // 128-byte row blocks along K
    const size_t a_part = (size_t)kblocks * TC_BM * 128;  // one split part of one stage
    const size_t b_part = (size_t)kblocks * nbp * 128;
    unsigned char *sA[2][2], *sB[2];
    {
        unsigned char *q = sm;
        for (int st = 0; st < 2; ++st)
            for (int h = 0; h < 2; ++h) {
                sA[st][h] = q;
                if (h == 0 || X3) q += a_part;
            }
        sB[0] = q;
        q += b_part;
        sB[1] = q;
    }
    __shared__ uint64_t bars[2];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t mtiles = (g.M + TC_BM - 1) / TC_BM;
    const int64_t n_tiles = mtiles * n_items;
    constexpr int NACC = X3 ? 2 : 1;  // TMEM regions per accumulator (main, corrections)
    uint32_t ncols = 32;
    while ((int)ncols < 2 * NACC * nbp) ncols <<= 1;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tmem_base)), "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bars[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bars[1])));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = make_idesc(KIND == 0 ? 2 : 1, nbp, TC_BM);
    uint32_t phase[2] = {0u, 0u};
    bool ok = true;

    // item -> B source (stem steps: branch of (prefix, slice); else strided)
    auto b_src = [&](int64_t item, bool &valid) -> const float * {
        valid = true;
        if (g.use_batch) {
            const int pl = (int)(item / g.ba.SB);
            const int64_t s = g.ba.state->slice_base + (item - (int64_t)pl * g.ba.SB);
            if (s >= g.ba.state->slice_end) {
                valid = false;
                return nullptr;
            }
            int64_t o = g.br->base + (int64_t)(g.ba.p0 + pl) * g.br->prefix_stride;
            for (int i = 0; i < g.br->n_sl; ++i)
                if ((s >> g.br->sl_bit[i]) & 1) o += (int64_t)1 << g.br->sl_pos[i];
            return reinterpret_cast<const float *>(g.pool + o);
        }
        return g.B + item * 2 * g.sB;
    };
    auto build_b = [&](const float *B) {
        for (int i = tid; i < nbp * kblocks * KC; i += TC_THREADS) {
            const int j = i / (kblocks * KC), kk = i % (kblocks * KC);
            float v = 0.f;
            if (j < N2 && kk < K2) {
                const int nu = j >> 1, d = j & 1, kap = kk >> 1, c = kk & 1;
                const float re = B[2 * ((int64_t)kap * g.N + nu)];
                const float im = B[2 * ((int64_t)kap * g.N + nu) + 1];
                v = (c == d) ? re : (c == 1 ? -im : im);
            }
            const uint32_t off = (uint32_t)((kk / KC) * nbp * 128) + sw128(j, (kk % KC) * ESZ);
            if constexpr (KIND == 0) {
                float hi, lo;
                split_tf32(v, hi, lo);
                *reinterpret_cast<float *>(sB[0] + off) = hi;
                *reinterpret_cast<float *>(sB[1] + off) = lo;
            } else {
                __nv_bfloat16 hi, lo;
                split_bf16(v, hi, lo);
                *reinterpret_cast<__nv_bfloat16 *>(sB[0] + off) = hi;
                if constexpr (X3) *reinterpret_cast<__nv_bfloat16 *>(sB[1] + off) = lo;
            }
        }
    };
    // load + split the 128 x K2 A tile of tile index t into stage st
    auto load_a = [&](int64_t t, int st) {
        const int64_t item = t / mtiles, m0 = (t % mtiles) * TC_BM;
        const float *A = g.A + item * g.sA;
        for (int i = tid; i < TC_BM * (K2 / 4); i += TC_THREADS) {
            const int r = i / (K2 / 4), k4 = (i % (K2 / 4)) * 4;
            const int64_t m = m0 + r;
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
            if (m < g.M) x = *reinterpret_cast<const float4 *>(A + m * K2 + k4);
            const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int kk = k4 + q;
                const uint32_t off = (uint32_t)((kk / KC) * TC_BM * 128) + sw128(r, (kk % KC) * ESZ);
                if constexpr (KIND == 0) {
                    float hi, lo;
                    split_tf32(xs[q], hi, lo);
                    *reinterpret_cast<float *>(sA[st][0] + off) = hi;
                    *reinterpret_cast<float *>(sA[st][1] + off) = lo;
                } else {
                    __nv_bfloat16 hi, lo;
                    split_bf16(xs[q], hi, lo);
                    *reinterpret_cast<__nv_bfloat16 *>(sA[st][0] + off) = hi;
                    if constexpr (X3) *reinterpret_cast<__nv_bfloat16 *>(sA[st][1] + off) = lo;
                }
            }
        }
        // K padding of the last row block stays zero from the first fill
    };
    auto issue = [&](int st, int acc) {
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        const uint32_t d = tmem + (uint32_t)(acc * NACC * nbp);
        const int nks = (K2 + KSTEP - 1) / KSTEP;  // K steps covering 2K (padding is zero)
        for (int ks = 0; ks < nks; ++ks) {
            const uint32_t kb = (uint32_t)((ks * KSTEP) / KC);
            const uint32_t ko = (uint32_t)(((ks * KSTEP) % KC) * ESZ);
            const uint64_t ahi = make_desc(smem_u32(sA[st][0]) + kb * TC_BM * 128 + ko);
            const uint64_t bhi = make_desc(smem_u32(sB[0]) + kb * nbp * 128 + ko);
            mma<KIND>(d, ahi, bhi, idesc, ks == 0 ? 0u : 1u);
            if constexpr (X3) {  // corrections in their own accumulator
                const uint64_t alo = make_desc(smem_u32(sA[st][1]) + kb * TC_BM * 128 + ko);
                const uint64_t blo = make_desc(smem_u32(sB[1]) + kb * nbp * 128 + ko);
                mma<KIND>(d + (uint32_t)nbp, ahi, blo, idesc, ks == 0 ? 0u : 1u);
                mma<KIND>(d + (uint32_t)nbp, alo, bhi, idesc, 1u);
            }
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                smem_u32(&bars[acc])));
    };
    auto epilogue = [&](int64_t t, int acc) {
        const int64_t item = t / mtiles, m0 = (t % mtiles) * TC_BM;
        float *C = g.C + item * g.sC;
        const int64_t row = m0 + warp * 32 + (tid & 31);
        for (int c0 = 0; c0 < nbp; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr =
                tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(acc * NACC * nbp + c0);
            tmem_ld16(taddr, v);
            if constexpr (X3) {
                uint32_t w[16];
                tmem_ld16(taddr + (uint32_t)nbp, w);
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    v[q] = __float_as_uint(__fadd_rn(__uint_as_float(v[q]), __uint_as_float(w[q])));
            }
            if (row < g.M) {
                if (c0 + 16 <= N2 && (N2 & 3) == 0) {
#pragma unroll
                    for (int q = 0; q < 16; q += 4)
                        *reinterpret_cast<float4 *>(C + row * N2 + c0 + q) =
                            make_float4(__uint_as_float(v[q]), __uint_as_float(v[q + 1]),
                                        __uint_as_float(v[q + 2]), __uint_as_float(v[q + 3]));
                } else {
                    for (int q = 0; q < 16 && c0 + q < N2; ++q) C[row * N2 + c0 + q] = __uint_as_float(v[q]);
                }
            }
        }
    };

    // zero both stages once (K padding of partially filled row blocks)
    for (int i = tid; i < (int)((X3 ? 4 : 2) * a_part / 16); i += TC_THREADS)
        reinterpret_cast<int4 *>(sm)[i] = make_int4(0, 0, 0, 0);
    int64_t t = blockIdx.x;
    int64_t cur_item = -1;
    bool item_valid = true;
    if (t < n_tiles) {
        cur_item = t / mtiles;
        const float *B = b_src(cur_item, item_valid);
        if (item_valid) build_b(B);
        load_a(t, 0);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (t < n_tiles && item_valid && tid == 0) issue(0, 0);
    int it = 0;
    while (t < n_tiles && ok) {
        const int st = it & 1, acc = it & 1;
        const int64_t tn = t + gridDim.x;
        const bool more = tn < n_tiles;
        const bool valid_now = item_valid;
        if (more) load_a(tn, st ^ 1);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (valid_now) {
            ok = mbar_wait(smem_u32(&bars[acc]), phase[acc]);
            phase[acc] ^= 1u;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        if (more && ok) {
            const int64_t ni = tn / mtiles;
            if (ni != cur_item) {  // B of a new batch item (its MMAs are done)
                cur_item = ni;
                const float *B = b_src(ni, item_valid);
                if (item_valid) build_b(B);
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                __syncthreads();
            }
            if (item_valid && tid == 0) issue(st ^ 1, acc ^ 1);
        }
        if (ok && valid_now) epilogue(t, acc);
        asm volatile("tcgen05.fence::before_thread_sync;\n");
        __syncthreads();
        t = tn;
        ++it;
    }
    if (!ok) {
        if (tid == 0) atomicExch(g.err, 5);
        mbar_wait(smem_u32(&bars[0]), phase[0]);
        mbar_wait(smem_u32(&bars[1]), phase[1]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols));
}

size_t tc_persistent_smem(int prec, int K2, int N2) {
    const bool x3 = prec != 3;
    const int esz = prec == 1 ? 4 : 2;
    const int kc = 128 / esz;
    const int kblocks = (K2 + kc - 1) / kc;
    const int nbp = (N2 + 15) & ~15;
    return 1024 + (size_t)kblocks * TC_BM * 128 * 2 * (x3 ? 2 : 1) + (size_t)kblocks * nbp * 128 * 2;
}

size_t tc_smem_bytes(int prec) {
    const bool x3 = prec != 3;
    return 1024 + (size_t)TC_BM * 128 * (x3 ? 2 : 1) + (size_t)TC_MAX_N2 * 128 * 2;
}

// Time-out flag of the tensor-core GEMM (0 = none), one per device image.
__device__ int g_tc_err_flag;
int *g_tc_err = nullptr;

cudaError_t run_tc(const TcArgs &a0, int64_t batch, tn_precision prec, cudaStream_t st) {
    TcArgs a = a0;
    if (!g_tc_err) return cudaErrorInitializationError;  // tc_gemm_init() not called
    a.err = g_tc_err;
    const int K2 = 2 * a.K, N2 = 2 * a.N;
    // the persistent kernel holds two accumulators of (x3: two regions of) nbp
    // TMEM columns each within the SM's 512
    const int n2_max_persistent = prec == TN_PREC_BF16x1 ? TC_MAX_N2 : TC_MAX_N2 / 2;
    if (K2 <= P_K2MAX && K2 % 4 == 0 && N2 <= n2_max_persistent && batch <= 65535 &&
        tc_persistent_smem((int)prec, K2, N2) <= P_SMEM_MAX) {
        static int num_sms = 0;
        if (!num_sms) {
            int dev;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
        }
        const int64_t tiles = ((a.M + TC_BM - 1) / TC_BM) * batch;
        const size_t smem = tc_persistent_smem((int)prec, K2, N2);
        // as many resident blocks per SM as shared memory allows (at most 4;
        // each holds 2 x 2N <= 512 TMEM columns in total)
        int per_sm = (int)std::max<size_t>(1, std::min<size_t>(4, (228 * 1024) / (smem + 1024)));
        int ncols = 32;
        while (ncols < (prec == TN_PREC_BF16x1 ? 2 : 4) * ((N2 + 15) & ~15)) ncols <<= 1;
        per_sm = std::max(1, std::min(per_sm, 512 / ncols));  // TMEM: 512 columns per SM
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms * per_sm));
        switch (prec) {
            case TN_PREC_TF32x3: tc_cgemm_persistent<1><<<grid, TC_THREADS, smem, st>>>(a, batch); break;
            case TN_PREC_BF16x3: tc_cgemm_persistent<2><<<grid, TC_THREADS, smem, st>>>(a, batch); break;
            case TN_PREC_BF16x1: tc_cgemm_persistent<3><<<grid, TC_THREADS, smem, st>>>(a, batch); break;
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    const int64_t gx = (a.M + TC_BM - 1) / TC_BM;
    const int gz = (2 * a.N + TC_MAX_N2 - 1) / TC_MAX_N2;
    if (gx > 0x7fffffffLL || batch > 65535 || gz > 65535) return cudaErrorInvalidValue;
    dim3 grid((unsigned)gx, (unsigned)batch, (unsigned)gz);
    const size_t smem = tc_smem_bytes((int)prec);
    switch (prec) {
        case TN_PREC_TF32x3:
            tc_cgemm_kernel<1><<<grid, TC_THREADS, smem, st>>>(a);
            break;
        case TN_PREC_BF16x3:
            tc_cgemm_kernel<2><<<grid, TC_THREADS, smem, st>>>(a);
            break;
        case TN_PREC_BF16x1:
            tc_cgemm_kernel<3><<<grid, TC_THREADS, smem, st>>>(a);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

// Once per process, outside any stream capture: shared-memory limits and the
// device address of the time-out flag.
cudaError_t tc_gemm_init() {
    const int smem3 = (int)tc_smem_bytes(1), smem1 = (int)tc_smem_bytes(3);
    cudaError_t e = cudaFuncSetAttribute(tc_cgemm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem3);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_cgemm_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem3);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_cgemm_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem1);
    int optin = 0, dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) P_SMEM_MAX = (size_t)optin - 2048;
    const int pmax = (int)P_SMEM_MAX;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_cgemm_persistent<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, pmax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_cgemm_persistent<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, pmax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_cgemm_persistent<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, pmax);
    if (e == cudaSuccess && !g_tc_err) e = cudaGetSymbolAddress((void **)&g_tc_err, g_tc_err_flag);
    return e;
}

bool tc_gemm_supported(int k, int n) { return k >= 0 && n >= 0 && k <= 20 && n <= 20; }

cudaError_t launch_tc_stem_gemm(const float2 *A, float2 *C, int64_t M, int k, int n,
                                int64_t strideA, int64_t strideC, const DevBranch *d_branch_entry,
                                const float2 *pool, BatchArgs ba, tn_precision prec,
                                cudaStream_t st) {
    // one batch item and 2^k, 2^n >= 16: the TMA-fed pipelined kernels (the
    // branch of the item's slice is split on the device first)
    if (g_tc_err && ba.n_items == 1 && tc_large_stem_supported(M, k, n, prec, A, C))
        return launch_tc_stem_gemm_large(A, C, M, k, n, d_branch_entry, pool, ba, prec, g_tc_err, st);
    TcArgs a{};
    a.A = reinterpret_cast<const float *>(A);
    a.C = reinterpret_cast<float *>(C);
    a.M = M;
    a.K = 1 << k;
    a.N = 1 << n;
    a.sA = 2 * strideA;
    a.sC = 2 * strideC;
    a.br = d_branch_entry;
    a.pool = pool;
    a.ba = ba;
    a.use_batch = 1;
    return run_tc(a, ba.n_items, prec, st);
}

cudaError_t launch_tc_cgemm(const float2 *A, const float2 *B, float2 *C, int64_t M, int64_t K,
                            int64_t N, int64_t batch, int64_t sA, int64_t sB, int64_t sC,
                            tn_precision prec, cudaStream_t st) {
    if (K > (1 << 20) || N > (1 << 20)) return cudaErrorInvalidValue;
    // large K and N: the TMA-fed pipelined kernel, one launch per batch item
    bool large = g_tc_err != nullptr && batch >= 1;
    for (int64_t b = 0; b < batch && large; ++b)
        large = tc_large_supported(M, K, N, prec, A + b * sA, C + b * sC);
    if (large) {
        for (int64_t b = 0; b < batch; ++b) {
            cudaError_t e = launch_tc_cgemm_large(A + b * sA, B + b * sB, C + b * sC, M, K, N, prec,
                                                  g_tc_err, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    TcArgs a{};
    a.A = reinterpret_cast<const float *>(A);
    a.B = reinterpret_cast<const float *>(B);
    a.C = reinterpret_cast<float *>(C);
    a.M = M;
    a.K = (int)K;
    a.N = (int)N;
    a.sA = 2 * sA;
    a.sB = sB;
    a.sC = 2 * sC;
    a.use_batch = 0;
    return run_tc(a, batch, prec, st);
}

cudaError_t tc_error_flag(int *out) {
    if (!g_tc_err) {
        *out = 0;
        return cudaSuccess;
    }
    return cudaMemcpy(out, g_tc_err, sizeof(int), cudaMemcpyDeviceToHost);
}

}  // namespace tn
