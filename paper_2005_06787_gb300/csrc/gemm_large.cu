// Complex GEMM on the tcgen05 tensor cores for large K and N (tn_cgemm with
// K >= 32 and N >= 64 complex, e.g. a stem step that absorbs a merged branch,
// Supp. A.3 "Branch merging"): C[m][nu] = sum_kappa A[m][kappa] B[kappa][nu],
// complex64, as the real GEMM of A viewed as [M][2K] with the 2K x 2N real
// expansion [[Br, Bi], [-Bi, Br]] of B (the same arithmetic as gemm_tc.cu).
//
// Both kernels here are persistent (one CTA per SM, 128 x BN output tiles in
// m-major order so the CTAs working at one time share A rows in L2) and
// warp-specialised:
//   warp 0      one thread issues TMA loads: the FP32 A tile of a k-block
//               (128-byte-swizzled boxes of 32 floats x 128 rows), prefetched
//               into L2 eight k-blocks ahead, and the pre-split B^T tiles (hi /
//               lo in the tensor-core type, K-major, built once per call by
//               lg_prep_b_kernel);
//   warps 4-11  converters: split every A value into hi + lo of the
//               tensor-core type (both rounded to nearest);
//   warp 1      one thread issues the MMAs: hi*hi into the main TMEM
//               accumulator, (x3) hi*lo + lo*hi into a correction accumulator
//               (the tensor core's FP32 accumulation truncates, so the
//               corrections stay apart from the full-size sum), then commits
//               the stage back to its producer;
//   warps 12-15 epilogue: each thread reads its TMEM lane (one row), adds
//               main + correction with round to nearest and stores the row.
// tc_cgemm_large_kernel splits A in place in the shared-memory stage, with
// TMEM double-buffered where two accumulators fit (the epilogue of a tile
// then overlaps the next tile's MMAs): TF32 x3 on 128-column tiles (3
// stages), BF16 x1 on 256-column tiles (3 stages), BF16 x3 on 256-column
// tiles (2 stages, one accumulator) when the output fills the GPU's waves;
// otherwise BF16 x3 runs on tc_cgemm_tmem_kernel, which stores hi / lo into
// tensor memory and takes A from there (128-column tiles, a 4-stage B ring
// beside a small A staging ring, one accumulator). The epilogues store
// through shared memory with TMA. Every wait is on an mbarrier and bounded
// in time; a wait that gives up records an error code (read by
// tn_device_status), and the kernel then waits (bounded) for its own copies
// and MMAs in flight before freeing TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "kernels.h"

namespace tn {

namespace {

constexpr int LG_THREADS = 512;  // 16 warps
constexpr int W_PRODUCER = 0, W_MMA = 1, W_ALLOC = 2, W_CONV0 = 4, N_CONV = 8, W_EPI0 = 12;
constexpr unsigned long long LG_WAIT_NS = 2000000000ull;  // 2 s per wait
constexpr uint32_t A_BOX_BYTES = 128 * 128;               // 128 rows x 128 B
constexpr uint32_t EPI_BOX_BYTES = 32 * 128;              // epilogue staging: 32 rows x 32 FP32

// x3 with A split in place in shared memory: TF32 (PREC 1: a stage holds 32
// real K; the FP32 box becomes hi, lo goes to a second box; 128-column tiles,
// two accumulator buffers) or BF16 (PREC 2: a stage holds 64 real K as two
// FP32 boxes, which become the hi and lo BF16 boxes of 128 B per row;
// 256-column tiles, so each k-block's 64 KB of B and 32 KB of A feed twice
// the MMAs of a 128-column tile; one accumulator of main + corrections).
// BNX > 0 sets the tile width (32 or 64 for narrow outputs, e.g. the stem's
// own GEMM steps); the ring then holds as many stages as fit (up to 6).
template <int PREC, int BNX = 0>
struct LgCfg {
    static_assert(PREC >= 1 && PREC <= 3, "the shared-memory split kernel serves TF32 x3, BF16 x3 and BF16 x1");
    static constexpr bool X3 = PREC != 3;
    static constexpr bool BF16 = PREC != 1;
    static constexpr int BN = BNX ? BNX : (BF16 ? 256 : 128);  // real output columns per tile
    static_assert(BN % 32 == 0 && BN >= 32 && BN <= 256, "tile width: a multiple of 32 up to 256");
    static constexpr int KBLK = BF16 ? 64 : 32;     // real K per stage (128 B per row of the MMA type)
    static constexpr uint32_t B_BYTES = (uint32_t)BN * 128;
    static constexpr uint32_t STAGE_BYTES = 2 * A_BOX_BYTES + B_BYTES * (X3 ? 2 : 1);
    static constexpr uint32_t TX_BYTES = (BF16 ? 2 : 1) * A_BOX_BYTES + B_BYTES * (X3 ? 2 : 1);
    static constexpr int ACC_COLS = BN * (X3 ? 2 : 1);  // TMEM columns per accumulator buffer (main [, corrections])
    static constexpr int NACC = 2 * ACC_COLS <= 512 ? 2 : 1;  // accumulator buffers
    static constexpr int EPI_NB = 1;                // epilogue staging boxes per epilogue warp
    static constexpr size_t FIXED = 1024 + 4 * EPI_NB * (size_t)EPI_BOX_BYTES + 256;
    static constexpr int STAGES_FIT = (int)((232448 - FIXED) / STAGE_BYTES);
    static constexpr int STAGES = STAGES_FIT > 6 ? 6 : STAGES_FIT;
    static_assert(STAGES >= 2, "at least two stages");
    static constexpr size_t RING = (size_t)STAGES * STAGE_BYTES;
    static constexpr size_t SMEM = 1024 + RING + 4 * EPI_NB * (size_t)EPI_BOX_BYTES;
};
static_assert(LgCfg<1>::STAGES == 3 && LgCfg<2>::STAGES == 2 && LgCfg<3>::STAGES == 3,
              "ring depths of the wide tiles as measured");
static_assert(LgCfg<1>::NACC * LgCfg<1>::ACC_COLS <= 512 && LgCfg<2>::NACC * LgCfg<2>::ACC_COLS <= 512 &&
                  LgCfg<3>::NACC * LgCfg<3>::ACC_COLS <= 512,
              "the accumulator buffers must fit the SM's 512 TMEM columns");
static_assert(LgCfg<1>::SMEM + 256 <= 232448 && LgCfg<2>::SMEM + 256 <= 232448 && LgCfg<3>::SMEM + 256 <= 232448,
              "stages and staging boxes must fit 227 KB of shared memory");

__device__ __forceinline__ uint32_t lg_smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t lg_globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool lg_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
// Wait for the phase of the given parity to complete; false after LG_WAIT_NS.
__device__ __forceinline__ bool lg_wait(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = lg_globaltimer();
    for (uint32_t i = 0;; ++i) {
        if (lg_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u && lg_globaltimer() - t0 > LG_WAIT_NS) return false;
    }
}
__device__ __forceinline__ void lg_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void lg_arrive_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
                 : "memory");
}
// Fetch a tile of the tensor map into L2 only (no shared memory, no barrier).
__device__ __forceinline__ void lg_prefetch2d(const CUtensorMap *map, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];\n" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void lg_tma2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                         uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
        "%3}], [%4];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
// K-major, 128-byte swizzle shared-memory descriptor (8-row atoms of 1024 B).
__device__ __forceinline__ uint64_t lg_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}
__host__ __device__ constexpr uint32_t lg_idesc(int ab, int n, int m) {
    return (1u << 4) | ((uint32_t)ab << 7) | ((uint32_t)ab << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
}
// MMA with both operands in shared memory: kind::tf32, or kind::f16 with
// BF16 operands.
template <bool BF16>
__device__ __forceinline__ void lg_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (BF16)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void lg_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
        : "memory");
}
__device__ __forceinline__ void lg_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15}, [%16];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}
__device__ __forceinline__ float lg_round_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
// Byte offset of 16-byte chunk c of row r in a 128-byte-swizzled tile.
__device__ __forceinline__ uint32_t lg_sw(int r, int c) {
    return (uint32_t)(r * 128 + (((c ^ r) & 7) << 4));
}

// TMA store of a shared-memory box to global memory, tracked by the issuing
// thread's bulk groups (rows and columns past the tensor are not written).
__device__ __forceinline__ void lg_tma_store2d(const CUtensorMap *map, uint32_t src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];\n" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(src), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void lg_bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// at most N of this thread's bulk groups still reading shared memory
template <int N>
__device__ __forceinline__ void lg_bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void lg_bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// Epilogue of one 128 x BN output tile by epilogue warp q (TMEM lanes
// 32q .. 32q+31 = tile rows 32q .. 32q+31, one per lane): 32 columns at a
// time, each lane reads its row from TMEM (for x3 the main and correction
// accumulators, added with round to nearest), writes it into the warp's
// staging box (32 rows x 128 B, 128-byte swizzle, so the eight lanes of a
// quarter-warp hit eight bank groups), and lane 0 stores the box with one
// TMA copy (full 128-byte lines; rows past M are clipped by the copy). A box
// is rewritten only after the copy that last read it has read it (NB boxes
// per warp). The caller skips warps whose 32 rows all lie past M.
template <int BN, bool X3, int NB>
__device__ __forceinline__ void lg_epilogue_tile(uint32_t tbase, const CUtensorMap *tmC, unsigned char *stage,
                                                 uint32_t stage_s, int n0, int row0, int lane, uint32_t &nstore) {
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32, ++nstore) {
        const uint32_t b = nstore % NB;
        if (lane == 0 && nstore >= (uint32_t)NB) lg_bulk_wait_read<NB - 1>();
        __syncwarp();
        unsigned char *box = stage + b * EPI_BOX_BYTES;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t v[16];
            lg_ld16(tbase + (uint32_t)(c0 + 16 * h), v);
            if constexpr (X3) {
                uint32_t w[16];
                lg_ld16(tbase + (uint32_t)(BN + c0 + 16 * h), w);
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    v[j] = __float_as_uint(__fadd_rn(__uint_as_float(v[j]), __uint_as_float(w[j])));
            } else {
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
                *reinterpret_cast<uint4 *>(box + lg_sw(lane, 4 * h + c)) =
                    make_uint4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
        }
        // generic-proxy writes become visible to the copy engine
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncwarp();
        if (lane == 0) {
            lg_tma_store2d(tmC, stage_s + b * EPI_BOX_BYTES, n0 + c0, row0);
            lg_bulk_commit();
        }
    }
}

template <int PREC, int BNX>
__global__ void __launch_bounds__(LG_THREADS, 1)
    tc_cgemm_large_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBh,
                          const __grid_constant__ CUtensorMap tmBl, const __grid_constant__ CUtensorMap tmC,
                          int64_t M, int K2, int N2, int *err) {
    using Cf = LgCfg<PREC, BNX>;
    constexpr int BN = Cf::BN, S = Cf::STAGES, KBLK = Cf::KBLK;
    constexpr bool X3 = Cf::X3;
    extern __shared__ __align__(1024) unsigned char lg_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(lg_raw) + 1023) & ~(uintptr_t)1023);
    constexpr int NACC = Cf::NACC;
    __shared__ __align__(8) uint64_t full_bar[S], conv_bar[S], empty_bar[S], tfull_bar[NACC], tempty_bar[NACC],
        drain_bar;
    __shared__ uint32_t tmem_base;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = N2 / BN;
    const int64_t n_tot = ((M + 127) / 128) * n_tiles;
    const int64_t st0 = blockIdx.x, st_step = gridDim.x;
    // k-blocks along 2K; a last partial one reads zeros past 2K (TMA fill)
    const int kblocks = (K2 + KBLK - 1) / KBLK;
    // first row / column of tile t (rows past M are read as zero and not stored)
    auto tile_m0 = [&](int64_t t) { return (int)((t / n_tiles) * 128); };
    auto tile_n0 = [&](int64_t t) { return (int)((t % n_tiles) * BN); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(lg_smem_u32(&full_bar[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(lg_smem_u32(&conv_bar[s])),
                         "n"(N_CONV));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(lg_smem_u32(&empty_bar[s])));
        }
        for (int a = 0; a < NACC; ++a) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(lg_smem_u32(&tfull_bar[a])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;\n" ::"r"(lg_smem_u32(&tempty_bar[a])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(lg_smem_u32(&drain_bar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
    }
    if (warp == W_ALLOC) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(
            lg_smem_u32(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = tmem_base;
    const uint32_t sbase = lg_smem_u32(sm);

    if (warp == W_PRODUCER) {
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmA)));
            asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmBh)));
            if constexpr (X3) asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmBl)));
            uint32_t it = 0;
            bool ok = true;
            // A k-blocks are first touched in DRAM; they are pulled into L2
            // LG_PREFETCH k-blocks ahead of their shared-memory load, across
            // tile boundaries, so the ring only sees L2 latency
            constexpr int LG_PREFETCH = 8;
            auto prefetch_a = [&](int64_t tt, int kk) {
                while (kk >= kblocks) {
                    kk -= kblocks;
                    tt += st_step;
                }
                if (tt >= n_tot) return;
                lg_prefetch2d(&tmA, kk * KBLK, tile_m0(tt));
                if (Cf::BF16 && kk * KBLK + 32 < K2) lg_prefetch2d(&tmA, kk * KBLK + 32, tile_m0(tt));
            };
            if (st0 < n_tot)
                for (int kk = 0; kk < LG_PREFETCH; ++kk) prefetch_a(st0, kk);
            for (int64_t t = st0; t < n_tot && ok; t += st_step) {
                const int m0 = tile_m0(t), n0 = tile_n0(t);
                for (int kb = 0; kb < kblocks; ++kb, ++it) {
                    prefetch_a(t, kb + LG_PREFETCH);
                    const int s = (int)(it % S);
                    if (!lg_wait(lg_smem_u32(&empty_bar[s]), ((it / S) & 1) ^ 1)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = lg_smem_u32(&full_bar[s]);
                    lg_arrive_tx(fb, Cf::TX_BYTES);
                    const uint32_t st = sbase + (uint32_t)s * Cf::STAGE_BYTES;
                    const int k = kb * KBLK;
                    lg_tma2d(st, &tmA, k, m0, fb);
                    if constexpr (Cf::BF16) lg_tma2d(st + A_BOX_BYTES, &tmA, k + 32, m0, fb);
                    lg_tma2d(st + 2 * A_BOX_BYTES, &tmBh, k, n0, fb);
                    if constexpr (X3) lg_tma2d(st + 2 * A_BOX_BYTES + Cf::B_BYTES, &tmBl, k, n0, fb);
                }
            }
            if (!ok) atomicExch(err, 5);
            // the copies of the last use of every stage have landed before exit
            for (uint32_t u = it > (uint32_t)S ? it - S : 0; u < it; ++u)
                lg_wait(lg_smem_u32(&full_bar[u % S]), (u / S) & 1);
        }
    } else if (warp >= W_CONV0 && warp < W_CONV0 + N_CONV) {
        // warp w of the converters owns rows 16w .. 16w+15; lane l takes
        // half h = (l >> 3) & 1 of row 16w + (l & 7) + 8 (l >> 4), so the 8
        // lanes of each quarter-warp touch 8 different rows of one box, whose
        // swizzled 16-byte chunks sit in 8 different bank groups (the two
        // halves of a row are lanes l and l + 8 of the same warp)
        const int r = 16 * (warp - W_CONV0) + (lane & 7) + 8 * (lane >> 4), h = (lane >> 3) & 1;
        uint32_t it = 0;
        bool ok = true;
        for (int64_t t = st0; t < n_tot && ok; t += st_step) {
            for (int kb = 0; kb < kblocks; ++kb, ++it) {
                const int s = (int)(it % S);
                if (!lg_wait(lg_smem_u32(&full_bar[s]), (it / S) & 1)) {
                    ok = false;
                    break;
                }
                unsigned char *a0 = sm + (size_t)s * Cf::STAGE_BYTES;
                unsigned char *a1 = a0 + A_BOX_BYTES;
                if constexpr (Cf::BF16) {
                    // half h of the row: the 32 FP32 values of box h (k 32h ..
                    // 32h+31) become chunks 4h .. 4h+3 of the hi row (box 0) and
                    // of the lo row (box 1); the other lane of the row reads what
                    // this one writes, so both read before either writes
                    const unsigned char *src = h ? a1 : a0;
                    float x[32];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const float4 v = *reinterpret_cast<const float4 *>(src + lg_sw(r, c));
                        x[4 * c] = v.x; x[4 * c + 1] = v.y; x[4 * c + 2] = v.z; x[4 * c + 3] = v.w;
                    }
                    uint32_t hw[16], lw[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const __nv_bfloat162 hb = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
                        hw[i] = *reinterpret_cast<const uint32_t *>(&hb);
                        if constexpr (X3) {
                            const float2 hf = __bfloat1622float2(hb);
                            const __nv_bfloat162 lb = __floats2bfloat162_rn(x[2 * i] - hf.x, x[2 * i + 1] - hf.y);
                            lw[i] = *reinterpret_cast<const uint32_t *>(&lb);
                        }
                    }
                    __syncwarp();
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        *reinterpret_cast<uint4 *>(a0 + lg_sw(r, 4 * h + c)) =
                            make_uint4(hw[4 * c], hw[4 * c + 1], hw[4 * c + 2], hw[4 * c + 3]);
                        if constexpr (X3)
                            *reinterpret_cast<uint4 *>(a1 + lg_sw(r, 4 * h + c)) =
                                make_uint4(lw[4 * c], lw[4 * c + 1], lw[4 * c + 2], lw[4 * c + 3]);
                    }
                } else {
                    // chunks 4h .. 4h+3 of the row: hi in place, lo into the second box
#pragma unroll
                    for (int c = 4 * h; c < 4 * h + 4; ++c) {
                    float4 *p = reinterpret_cast<float4 *>(a0 + lg_sw(r, c));
                    const float4 x = *p;
                    float4 hi, lo;
                    hi.x = lg_round_tf32(x.x); lo.x = lg_round_tf32(x.x - hi.x);
                    hi.y = lg_round_tf32(x.y); lo.y = lg_round_tf32(x.y - hi.y);
                    hi.z = lg_round_tf32(x.z); lo.z = lg_round_tf32(x.z - hi.z);
                    hi.w = lg_round_tf32(x.w); lo.w = lg_round_tf32(x.w - hi.w);
                    *p = hi;
                    *reinterpret_cast<float4 *>(a1 + lg_sw(r, c)) = lo;
                    }
                }
                // generic-proxy writes become visible to the tensor core; one
                // lane per warp signals once the whole warp is done
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                __syncwarp();
                if (lane == 0) lg_arrive(lg_smem_u32(&conv_bar[s]));
            }
        }
        if (!ok) atomicExch(err, 5);
    } else if (warp == W_MMA) {
        if (lane == 0) {
            constexpr uint32_t idesc = lg_idesc(Cf::BF16 ? 1 : 2, BN, 128);  // BF16 / TF32 operands
            uint32_t it = 0, tile_i = 0;
            bool ok = true;
            for (int64_t t = st0; t < n_tot && ok; t += st_step, ++tile_i) {
                const uint32_t acc = tile_i % NACC, use = tile_i / NACC;
                if (!lg_wait(lg_smem_u32(&tempty_bar[acc]), (use & 1) ^ 1)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n");
                const uint32_t d = tmem + acc * (uint32_t)Cf::ACC_COLS;
                for (int kb = 0; kb < kblocks; ++kb, ++it) {
                    const int s = (int)(it % S);
                    if (!lg_wait(lg_smem_u32(&conv_bar[s]), (it / S) & 1)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;\n");
                    const uint32_t st = sbase + (uint32_t)s * Cf::STAGE_BYTES;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {  // 4 MMAs of 32 bytes of K per 128-byte row
                        const uint32_t ko = (uint32_t)ks * 32;
                        const uint64_t ahi = lg_desc(st + ko), alo = lg_desc(st + A_BOX_BYTES + ko);
                        const uint64_t bhi = lg_desc(st + 2 * A_BOX_BYTES + ko);
                        const uint32_t accum = (kb | ks) != 0;
                        lg_mma<Cf::BF16>(d, ahi, bhi, idesc, accum);
                        if constexpr (X3) {
                            const uint64_t blo = lg_desc(st + 2 * A_BOX_BYTES + Cf::B_BYTES + ko);
                            lg_mma<Cf::BF16>(d + BN, ahi, blo, idesc, accum);
                            lg_mma<Cf::BF16>(d + BN, alo, bhi, idesc, 1u);
                        }
                    }
                    lg_commit(lg_smem_u32(&empty_bar[s]));  // stage free once these MMAs are done
                }
                if (!ok) break;
                lg_commit(lg_smem_u32(&tfull_bar[acc]));
            }
            if (!ok) {
                atomicExch(err, 5);
                lg_commit(lg_smem_u32(&drain_bar));  // every MMA issued so far has finished
                lg_wait(lg_smem_u32(&drain_bar), 0);
            }
        }
    } else if (warp >= W_EPI0) {
        const int q = warp & 3;  // TMEM lanes 32q .. 32q+31 of this warp
        unsigned char *stage = sm + Cf::RING + (size_t)q * Cf::EPI_NB * EPI_BOX_BYTES;
        const uint32_t stage_s = lg_smem_u32(stage);
        uint32_t tile_i = 0, nstore = 0;
        bool ok = true;
        for (int64_t t = st0; t < n_tot; t += st_step, ++tile_i) {
            const uint32_t acc = tile_i % NACC, use = tile_i / NACC;
            if (!lg_wait(lg_smem_u32(&tfull_bar[acc]), use & 1)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            const int row0 = tile_m0(t) + 32 * q;
            const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + acc * (uint32_t)Cf::ACC_COLS;
            if ((int64_t)row0 < M)
                lg_epilogue_tile<BN, X3, Cf::EPI_NB>(tbase, &tmC, stage, stage_s, tile_n0(t), row0, lane, nstore);
            asm volatile("tcgen05.fence::before_thread_sync;\n");
            __syncwarp();
            if (lane == 0) lg_arrive(lg_smem_u32(&tempty_bar[acc]));
        }
        if (!ok) atomicExch(err, 5);
        if (lane == 0) lg_bulk_wait_all();  // every output copy has completed
        __syncwarp();
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (warp == W_ALLOC) {
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem));
    }
}

// ------------------------------------------------------------------------
// Variant with the A operand in tensor memory. The converters read the FP32
// A rows from a staging slot (released as soon as it is read), split them and
// store hi / lo straight into TMEM with tcgen05.st; the MMAs take A from TMEM
// and only B from shared memory. Shared memory then carries the TMA copies,
// one read of A and the B operand reads, and holds a 4-stage B ring beside a
// small A staging ring. TMEM holds one accumulator (main + corrections for x3)
// and four A slots, so the epilogue of a tile runs before the next tile's
// MMAs start.
template <int PREC>
struct LtCfg {
    static_assert(PREC == 2 || PREC == 3, "the tensor-memory kernel serves BF16 x3 and x1");
    static constexpr bool X3 = PREC == 2;
    static constexpr int BN = X3 ? 128 : 256;
    static constexpr int KBLK = 64;                       // real K per stage (128 B of BF16 per row)
    static constexpr uint32_t A_SLOT = 2 * A_BOX_BYTES;   // FP32 rows of one k-block (two boxes)
#ifndef LT_SA
#define LT_SA 2
#endif
#ifndef LT_SB
#define LT_SB 4
#endif
    static constexpr int S_A = LT_SA;                     // staging slots
    static constexpr int S_B = LT_SB;                     // B stages (= TMEM A slots)
    static constexpr uint32_t B_BYTES = (uint32_t)BN * 128;
    static constexpr uint32_t B_STAGE = B_BYTES * (X3 ? 2 : 1);
    static constexpr int ACC_COLS = BN * (X3 ? 2 : 1);
    static constexpr int A_COLS = 32 * (X3 ? 2 : 1);     // TMEM columns of one A slot (hi [+ lo])
#ifndef LT_EPI_NB
#define LT_EPI_NB 1
#endif
    static constexpr int EPI_NB = LT_EPI_NB;              // epilogue staging boxes per epilogue warp
    static constexpr size_t RING = (size_t)S_A * A_SLOT + (size_t)S_B * B_STAGE;
    static constexpr size_t SMEM = 1024 + RING + 4 * EPI_NB * (size_t)EPI_BOX_BYTES;
};
static_assert(LtCfg<2>::ACC_COLS + LtCfg<2>::S_B * LtCfg<2>::A_COLS <= 512 &&
                  LtCfg<3>::ACC_COLS + LtCfg<3>::S_B * LtCfg<3>::A_COLS <= 512,
              "accumulator and A slots must fit the SM's 512 TMEM columns");
static_assert(LtCfg<2>::SMEM + 256 <= 232448 && LtCfg<3>::SMEM + 256 <= 232448,
              "staging ring and B stages must fit 227 KB of shared memory per block");

__device__ __forceinline__ void lt_st16(uint32_t taddr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16};\n" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}
// kind::f16 MMA (BF16 operands) with A in tensor memory, B in shared memory.
__device__ __forceinline__ void lt_mma(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
}

template <int PREC>
__global__ void __launch_bounds__(LG_THREADS, 1)
    tc_cgemm_tmem_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBh,
                         const __grid_constant__ CUtensorMap tmBl, const __grid_constant__ CUtensorMap tmC,
                         int64_t M, int K2, int N2, int *err) {
    using Cf = LtCfg<PREC>;
    constexpr int BN = Cf::BN, SA = Cf::S_A, SB = Cf::S_B, KBLK = Cf::KBLK;
    constexpr bool X3 = Cf::X3;
    extern __shared__ __align__(1024) unsigned char lt_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(lt_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t a_full[SA], a_empty[SA], b_full[SB], b_empty[SB], conv_bar[SB],
        tfull_bar, tempty_bar, drain_bar;
    __shared__ uint32_t tmem_base;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = N2 / BN;
    const int64_t n_tot = ((M + 127) / 128) * n_tiles;
    const int kblocks = K2 / KBLK;
    auto tile_m0 = [&](int64_t t) { return (int)((t / n_tiles) * 128); };
    auto tile_n0 = [&](int64_t t) { return (int)((t % n_tiles) * BN); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < SA; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(lg_smem_u32(&a_full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(lg_smem_u32(&a_empty[s])),
                         "n"(N_CONV));
        }
        for (int s = 0; s < SB; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(lg_smem_u32(&b_full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(lg_smem_u32(&b_empty[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(lg_smem_u32(&conv_bar[s])),
                         "n"(N_CONV));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(lg_smem_u32(&tfull_bar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;\n" ::"r"(lg_smem_u32(&tempty_bar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(lg_smem_u32(&drain_bar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
    }
    if (warp == W_ALLOC) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(
            lg_smem_u32(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = tmem_base;
    const uint32_t sa_base = lg_smem_u32(sm);
    const uint32_t sb_base = sa_base + (uint32_t)SA * Cf::A_SLOT;
    auto a_cols = [&](int j) { return (uint32_t)(Cf::ACC_COLS + j * Cf::A_COLS); };

    if (warp == W_PRODUCER) {
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmA)));
            asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmBh)));
            if constexpr (X3) asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmBl)));
            constexpr int LG_PREFETCH = 8;  // k-blocks of A pulled into L2 ahead of their copy
            auto prefetch_a = [&](int64_t tt, int kk) {
                while (kk >= kblocks) {
                    kk -= kblocks;
                    tt += gridDim.x;
                }
                if (tt >= n_tot) return;
                lg_prefetch2d(&tmA, kk * KBLK, tile_m0(tt));
                lg_prefetch2d(&tmA, kk * KBLK + 32, tile_m0(tt));
            };
            if ((int64_t)blockIdx.x < n_tot)
                for (int kk = 0; kk < LG_PREFETCH; ++kk) prefetch_a(blockIdx.x, kk);
            uint32_t it = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < n_tot && ok; t += gridDim.x) {
                const int m0 = tile_m0(t), n0 = tile_n0(t);
                for (int kb = 0; kb < kblocks; ++kb, ++it) {
                    prefetch_a(t, kb + LG_PREFETCH);
                    const int sa = (int)(it % SA), sb = (int)(it % SB);
                    if (!lg_wait(lg_smem_u32(&a_empty[sa]), ((it / SA) & 1) ^ 1) ||
                        !lg_wait(lg_smem_u32(&b_empty[sb]), ((it / SB) & 1) ^ 1)) {
                        ok = false;
                        break;
                    }
                    const int k = kb * KBLK;
                    const uint32_t fa = lg_smem_u32(&a_full[sa]), fb = lg_smem_u32(&b_full[sb]);
                    const uint32_t da = sa_base + (uint32_t)sa * Cf::A_SLOT;
                    const uint32_t db = sb_base + (uint32_t)sb * Cf::B_STAGE;
                    lg_arrive_tx(fa, Cf::A_SLOT);
                    lg_tma2d(da, &tmA, k, m0, fa);
                    lg_tma2d(da + A_BOX_BYTES, &tmA, k + 32, m0, fa);
                    lg_arrive_tx(fb, Cf::B_STAGE);
                    lg_tma2d(db, &tmBh, k, n0, fb);
                    if constexpr (X3) lg_tma2d(db + Cf::B_BYTES, &tmBl, k, n0, fb);
                }
            }
            if (!ok) atomicExch(err, 5);
            // before exit: every copy issued has landed
            for (uint32_t u = it > (uint32_t)SA ? it - SA : 0; u < it; ++u)
                lg_wait(lg_smem_u32(&a_full[u % SA]), (u / SA) & 1);
            for (uint32_t u = it > (uint32_t)SB ? it - SB : 0; u < it; ++u)
                lg_wait(lg_smem_u32(&b_full[u % SB]), (u / SB) & 1);
        }
    } else if (warp >= W_CONV0 && warp < W_CONV0 + N_CONV) {
        // warp w converts rows 32 (w % 4) .. +31 (its TMEM lane quarter),
        // half h = (w - 4) / 4 of the k-block: lane l owns row 32 (w % 4) + l
        const int q = warp & 3, h = (warp - W_CONV0) >> 2;
        const int r = 32 * q + lane;
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        uint32_t it = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; t < n_tot && ok; t += gridDim.x) {
            for (int kb = 0; kb < kblocks; ++kb, ++it) {
                const int sa = (int)(it % SA), sb = (int)(it % SB);
                if (!lg_wait(lg_smem_u32(&a_full[sa]), (it / SA) & 1)) {
                    ok = false;
                    break;
                }
                const unsigned char *slot = sm + (size_t)sa * Cf::A_SLOT;
                uint32_t hw[16], lw[16];
                // the k-block's 64 FP32 columns: box h of the row (32 values)
                const unsigned char *src = slot + (size_t)h * A_BOX_BYTES;
                float x[32];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float4 v = *reinterpret_cast<const float4 *>(src + lg_sw(r, c));
                    x[4 * c] = v.x; x[4 * c + 1] = v.y; x[4 * c + 2] = v.z; x[4 * c + 3] = v.w;
                }
                __syncwarp();
                if (lane == 0) lg_arrive(lg_smem_u32(&a_empty[sa]));  // staging slot read
                // TMEM column i of the half holds BF16 elements 2i (low half) and 2i + 1
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const __nv_bfloat162 hb = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
                    hw[i] = *reinterpret_cast<const uint32_t *>(&hb);
                    if constexpr (X3) {
                        const float2 hf = __bfloat1622float2(hb);
                        const __nv_bfloat162 lb = __floats2bfloat162_rn(x[2 * i] - hf.x, x[2 * i + 1] - hf.y);
                        lw[i] = *reinterpret_cast<const uint32_t *>(&lb);
                    }
                }
                // the TMEM slot is free once the MMAs of its previous use are done
                if (!lg_wait(lg_smem_u32(&b_empty[sb]), ((it / SB) & 1) ^ 1)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n");
                const uint32_t ta = tmem + lane_base + a_cols(sb) + (uint32_t)(16 * h);
                lt_st16(ta, hw);
                if constexpr (X3) lt_st16(ta + 32, lw);
                asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;\n");
                __syncwarp();
                if (lane == 0) lg_arrive(lg_smem_u32(&conv_bar[sb]));
            }
        }
        if (!ok) atomicExch(err, 5);
    } else if (warp == W_MMA) {
        if (lane == 0) {
            constexpr uint32_t idesc = lg_idesc(1, BN, 128);  // BF16 operands
            uint32_t it = 0, tile_i = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < n_tot && ok; t += gridDim.x, ++tile_i) {
                if (!lg_wait(lg_smem_u32(&tempty_bar), (tile_i & 1) ^ 1)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n");
                for (int kb = 0; kb < kblocks; ++kb, ++it) {
                    const int sb = (int)(it % SB);
                    if (!lg_wait(lg_smem_u32(&conv_bar[sb]), (it / SB) & 1) ||
                        !lg_wait(lg_smem_u32(&b_full[sb]), (it / SB) & 1)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;\n");
                    const uint32_t bst = sb_base + (uint32_t)sb * Cf::B_STAGE;
                    const uint32_t ahi = tmem + a_cols(sb);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {  // 32 bytes of K per MMA: 8 TMEM columns of A
                        const uint32_t ko = (uint32_t)ks * 32;
                        const uint64_t bhi = lg_desc(bst + ko);
                        const uint32_t accum = (kb | ks) != 0;
                        lt_mma(tmem, ahi + 8 * ks, bhi, idesc, accum);
                        if constexpr (X3) {
                            const uint64_t blo = lg_desc(bst + Cf::B_BYTES + ko);
                            lt_mma(tmem + BN, ahi + 8 * ks, blo, idesc, accum);
                            lt_mma(tmem + BN, ahi + 32 + 8 * ks, bhi, idesc, 1u);
                        }
                    }
                    lg_commit(lg_smem_u32(&b_empty[sb]));  // B stage and A slot free when done
                }
                if (!ok) break;
                lg_commit(lg_smem_u32(&tfull_bar));
            }
            if (!ok) {
                atomicExch(err, 5);
                lg_commit(lg_smem_u32(&drain_bar));
                lg_wait(lg_smem_u32(&drain_bar), 0);
            }
        }
    } else if (warp >= W_EPI0) {
        const int q = warp & 3;
        unsigned char *stage = sm + Cf::RING + (size_t)q * Cf::EPI_NB * EPI_BOX_BYTES;
        const uint32_t stage_s = lg_smem_u32(stage);
        uint32_t tile_i = 0, nstore = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; t < n_tot; t += gridDim.x, ++tile_i) {
            if (!lg_wait(lg_smem_u32(&tfull_bar), tile_i & 1)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            const int row0 = tile_m0(t) + 32 * q;
            const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16);
            if ((int64_t)row0 < M)
                lg_epilogue_tile<BN, X3, Cf::EPI_NB>(tbase, &tmC, stage, stage_s, tile_n0(t), row0, lane, nstore);
            asm volatile("tcgen05.fence::before_thread_sync;\n");
            __syncwarp();
            if (lane == 0) lg_arrive(lg_smem_u32(&tempty_bar));
        }
        if (!ok) atomicExch(err, 5);
        if (lane == 0) lg_bulk_wait_all();  // every output copy has completed
        __syncwarp();
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (warp == W_ALLOC) {
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem));
    }
}

// B^T expanded to the real 2N x 2K matrix (row j = real output column, K
// contiguous) and split into the tensor-core type: bt[j][kk] with
// expansion[kk][j] = c == d ? Re B[kappa][nu] : (c == 1 ? -Im : Im) for
// kk = 2 kappa + c, j = 2 nu + d.
template <int PREC>
__global__ void lg_prep_b_kernel(const float2 *__restrict__ B, int K, int N, void *hi_out, void *lo_out) {
    const int64_t K2 = 2 * (int64_t)K, total = 2 * (int64_t)N * K2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i / K2, kk = i % K2;
        const int nu = (int)(j >> 1), d = (int)(j & 1), kap = (int)(kk >> 1), c = (int)(kk & 1);
        const float2 b = B[(int64_t)kap * N + nu];
        const float v = (c == d) ? b.x : (c == 1 ? -b.y : b.y);
        if constexpr (PREC == 1) {
            const float h = lg_round_tf32(v);
            reinterpret_cast<float *>(hi_out)[i] = h;
            reinterpret_cast<float *>(lo_out)[i] = lg_round_tf32(v - h);
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            reinterpret_cast<__nv_bfloat16 *>(hi_out)[i] = h;
            if constexpr (PREC == 2)
                reinterpret_cast<__nv_bfloat16 *>(lo_out)[i] = __float2bfloat16_rn(v - __bfloat162float(h));
        }
    }
}

// The same split for a stem GEMM step with one batch item: B is the branch's
// matrix for the launch's prefix and slice (read from the device-side batch
// state, so a captured graph replays it for every slice).
template <int PREC>
__global__ void lg_prep_b_stem_kernel(const DevBranch *__restrict__ br, const float2 *__restrict__ pool,
                                      BatchArgs ba, int K, int N, void *hi_out, void *lo_out) {
    int64_t o = br->base + (int64_t)ba.p0 * br->prefix_stride;
    const int64_t sl = ba.state->slice_base;
    for (int i = 0; i < br->n_sl; ++i)
        if ((sl >> br->sl_bit[i]) & 1) o += (int64_t)1 << br->sl_pos[i];
    const float2 *B = pool + o;
    const int64_t K2 = 2 * (int64_t)K, total = 2 * (int64_t)N * K2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i / K2, kk = i % K2;
        const int nu = (int)(j >> 1), d = (int)(j & 1), kap = (int)(kk >> 1), c = (int)(kk & 1);
        const float2 b = B[(int64_t)kap * N + nu];
        const float v = (c == d) ? b.x : (c == 1 ? -b.y : b.y);
        if constexpr (PREC == 1) {
            const float h = lg_round_tf32(v);
            reinterpret_cast<float *>(hi_out)[i] = h;
            reinterpret_cast<float *>(lo_out)[i] = lg_round_tf32(v - h);
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            reinterpret_cast<__nv_bfloat16 *>(hi_out)[i] = h;
            if constexpr (PREC == 2)
                reinterpret_cast<__nv_bfloat16 *>(lo_out)[i] = __float2bfloat16_rn(v - __bfloat162float(h));
        }
    }
}

// Where B comes from: a complex K x N matrix, or (stem steps) a branch of
// the pool selected for the launch's batch item on the device.
struct LgBSource {
    const float2 *B = nullptr;
    const DevBranch *br = nullptr;
    const float2 *pool = nullptr;
    BatchArgs ba{};
};

// The driver's tensor-map encoder, looked up through the runtime so that the
// library does not link against the driver library itself (it then still
// loads on hosts without a GPU driver, where only the planner is used).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

bool encode_2d(CUtensorMap *map, CUtensorMapDataType dt, size_t esz, const void *base, uint64_t inner,
               uint64_t outer, uint32_t box_inner, uint32_t box_outer) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {inner * esz};
    const cuuint32_t box[2] = {box_inner, box_outer};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, dt, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int PREC, int BNX = 0>
cudaError_t run_large(const float2 *A, const LgBSource &bs, float2 *C, int64_t M, int K, int N, int *err,
                      cudaStream_t st) {
    using Cf = LgCfg<PREC, BNX>;
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    static int num_sms = 0;
    std::call_once(attr_once, [] {
        attr_err = cudaFuncSetAttribute(tc_cgemm_large_kernel<PREC, BNX>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cf::SMEM);
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    });
    if (attr_err != cudaSuccess) return attr_err;
    const int K2 = 2 * K, N2 = 2 * N;
    const size_t esz = Cf::BF16 ? 2 : 4;  // BF16, or TF32 in FP32 words
    const size_t part = (size_t)N2 * K2 * esz;
    void *ws = nullptr;
    cudaError_t e = cudaMallocAsync(&ws, part * 2, st);
    if (e != cudaSuccess) return e;
    unsigned char *bhi = static_cast<unsigned char *>(ws), *blo = bhi + part;
    const int64_t total = (int64_t)N2 * K2;
    const unsigned pgrid = (unsigned)std::min<int64_t>((total + 255) / 256, 4096);
    if (bs.br)
        lg_prep_b_stem_kernel<PREC><<<pgrid, 256, 0, st>>>(bs.br, bs.pool, bs.ba, K, N, bhi, blo);
    else
        lg_prep_b_kernel<PREC><<<pgrid, 256, 0, st>>>(bs.B, K, N, bhi, blo);
    e = cudaGetLastError();
    CUtensorMap ma, mbh, mbl, mc;  // A, B^T hi / lo, C
    const CUtensorMapDataType bt = Cf::BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const uint32_t bbox = Cf::BF16 ? 64 : 32;  // 128 bytes of K per row
    if (e == cudaSuccess &&
        !(encode_2d(&ma, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, A, (uint64_t)K2, (uint64_t)M, 32, 128) &&
          encode_2d(&mbh, bt, esz, bhi, (uint64_t)K2, (uint64_t)N2, bbox, Cf::BN) &&
          encode_2d(&mbl, bt, esz, blo, (uint64_t)K2, (uint64_t)N2, bbox, Cf::BN) &&
          encode_2d(&mc, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, C, (uint64_t)N2, (uint64_t)M, 32, 32)))
        e = cudaErrorInvalidValue;
    if (e == cudaSuccess) {
        const int64_t tiles = ((M + 127) / 128) * (N2 / Cf::BN);
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, num_sms));
        tc_cgemm_large_kernel<PREC, BNX><<<grid, LG_THREADS, Cf::SMEM, st>>>(ma, mbh, mbl, mc, M, K2, N2, err);
        e = cudaGetLastError();
    }
    cudaError_t f = cudaFreeAsync(ws, st);
    return e != cudaSuccess ? e : f;
}

template <int PREC>
cudaError_t run_tmem(const float2 *A, const float2 *B, float2 *C, int64_t M, int K, int N, int *err,
                     cudaStream_t st) {
    using Cf = LtCfg<PREC>;
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    static int num_sms = 0;
    std::call_once(attr_once, [] {
        attr_err = cudaFuncSetAttribute(tc_cgemm_tmem_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)Cf::SMEM);
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    });
    if (attr_err != cudaSuccess) return attr_err;
    const int K2 = 2 * K, N2 = 2 * N;
    const size_t esz = 2;  // BF16
    const size_t part = (size_t)N2 * K2 * esz;
    void *ws = nullptr;
    cudaError_t e = cudaMallocAsync(&ws, part * (Cf::X3 ? 2 : 1), st);
    if (e != cudaSuccess) return e;
    unsigned char *bhi = static_cast<unsigned char *>(ws), *blo = Cf::X3 ? bhi + part : bhi;
    const int64_t total = (int64_t)N2 * K2;
    lg_prep_b_kernel<PREC><<<(unsigned)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, st>>>(
        B, K, N, bhi, blo);
    e = cudaGetLastError();
    CUtensorMap ma, mbh, mbl, mc;  // A, B^T hi / lo, C
    const CUtensorMapDataType bt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const uint32_t bbox = 64;  // 128 bytes of K per row
    if (e == cudaSuccess &&
        !(encode_2d(&ma, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, A, (uint64_t)K2, (uint64_t)M, 32, 128) &&
          encode_2d(&mbh, bt, esz, bhi, (uint64_t)K2, (uint64_t)N2, bbox, Cf::BN) &&
          encode_2d(&mbl, bt, esz, blo, (uint64_t)K2, (uint64_t)N2, bbox, Cf::BN) &&
          encode_2d(&mc, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, C, (uint64_t)N2, (uint64_t)M, 32, 32)))
        e = cudaErrorInvalidValue;
    if (e == cudaSuccess) {
        const int64_t tiles = ((M + 127) / 128) * (N2 / Cf::BN);
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, num_sms));
        tc_cgemm_tmem_kernel<PREC><<<grid, LG_THREADS, Cf::SMEM, st>>>(ma, mbh, mbl, mc, M, K2, N2, err);
        e = cudaGetLastError();
    }
    cudaError_t f = cudaFreeAsync(ws, st);
    return e != cudaSuccess ? e : f;
}

// 3xBF16 kernel choice: 256-column tiles with A split in shared memory
// (measured 7-8 % faster per tile pair than the 128-column tensor-memory
// kernel at full waves) unless they leave more of the last wave idle, e.g.
// M = 16384, 2N = 1024: 512 wide tiles are 4 waves of 152, 1024 narrow ones
// 7 waves.
bool bf16x3_wide_tiles(int64_t M, int64_t N) {
    const int64_t N2 = 2 * N;
    if (N2 % LgCfg<2>::BN) return false;
    static int num_sms = 0;
    if (!num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || num_sms < 1)
            num_sms = 1;
    }
    const int64_t mt = (M + 127) / 128;
    const int64_t waves_wide = (mt * (N2 / LgCfg<2>::BN) + num_sms - 1) / num_sms;
    const int64_t waves_narrow = (mt * (N2 / LtCfg<2>::BN) + num_sms - 1) / num_sms;
    return (double)waves_wide * 2.0 / 1.075 < (double)waves_narrow;
}

// Kernel for a shape: 0 none; 1 the precision's default tile width; 2 the
// 3xBF16 tensor-memory kernel (128 columns); 3 / 4 the shared-memory split
// kernel on 64- / 32-column tiles (narrow outputs such as the stem's own
// GEMM steps). plain_b: B is a plain matrix (the tensor-memory kernel reads
// no branch pool).
int large_variant(tn_precision prec, int64_t M, int64_t K2, int64_t N2, bool plain_b) {
    if (K2 % 32 || N2 % 32) return 0;
    const bool dflt = N2 % LgCfg<(int)TN_PREC_TF32x3>::BN == 0;
    switch (prec) {
        case TN_PREC_TF32x3:
            if (dflt) return 1;
            break;
        case TN_PREC_BF16x3:
            if (N2 % LgCfg<2>::BN == 0 && bf16x3_wide_tiles(M, N2 / 2)) return 1;
            if (plain_b && N2 % LtCfg<2>::BN == 0 && K2 % LtCfg<2>::KBLK == 0) return 2;
            break;
        case TN_PREC_BF16x1:
            if (N2 % LgCfg<3>::BN == 0) return 1;
            break;
        default: return 0;
    }
    return N2 % 64 == 0 ? 3 : 4;
}

template <int PREC>
cudaError_t run_variant(int v, const float2 *A, const LgBSource &bs, float2 *C, int64_t M, int K, int N, int *err,
                        cudaStream_t st) {
    switch (v) {
        case 1: return run_large<PREC>(A, bs, C, M, K, N, err, st);
        case 2:
            if constexpr (PREC == 2) return run_tmem<PREC>(A, bs.B, C, M, K, N, err, st);
            return cudaErrorInvalidValue;
        case 3: return run_large<PREC, 64>(A, bs, C, M, K, N, err, st);
        case 4: return run_large<PREC, 32>(A, bs, C, M, K, N, err, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t run_any(tn_precision prec, const float2 *A, const LgBSource &bs, float2 *C, int64_t M, int64_t K,
                    int64_t N, int *err, cudaStream_t st) {
    const int v = large_variant(prec, M, 2 * K, 2 * N, bs.br == nullptr);
    // measured per precision (M = 65536, K = N = 512): TF32 x3 and BF16 x1 run
    // faster with A split in place in shared memory (0.62 vs 0.59 of the TF32
    // peak; 0.42 vs 0.38), BF16 x3 on 256-column tiles in shared memory (0.59
    // vs 0.55 on 128-column tiles with A in tensor memory)
    switch (prec) {
        case TN_PREC_TF32x3: return run_variant<1>(v, A, bs, C, M, (int)K, (int)N, err, st);
        case TN_PREC_BF16x3: return run_variant<2>(v, A, bs, C, M, (int)K, (int)N, err, st);
        case TN_PREC_BF16x1: return run_variant<3>(v, A, bs, C, M, (int)K, (int)N, err, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool tc_large_supported(int64_t M, int64_t K, int64_t N, tn_precision prec, const void *A, const void *C) {
    if (prec == TN_PREC_FP32_SIMT) return false;
    const bool aligned = !((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(C)) & 15);
    return aligned && M >= 128 && M < ((int64_t)1 << 31) && K >= 16 && K <= (1 << 20) && N <= (1 << 20) &&
           large_variant(prec, M, 2 * K, 2 * N, true) != 0;
}

cudaError_t launch_tc_cgemm_large(const float2 *A, const float2 *B, float2 *C, int64_t M, int64_t K,
                                  int64_t N, tn_precision prec, int *err, cudaStream_t st) {
    LgBSource bs;
    bs.B = B;
    return run_any(prec, A, bs, C, M, K, N, err, st);
}

bool tc_large_stem_supported(int64_t M, int k, int n, tn_precision prec, const void *A, const void *C) {
    if (prec == TN_PREC_FP32_SIMT) return false;
    const int64_t K = (int64_t)1 << k, N = (int64_t)1 << n;
    const bool aligned = !((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(C)) & 15);
    return aligned && M >= 128 && M < ((int64_t)1 << 31) && K >= 16 && N >= 16 &&
           large_variant(prec, M, 2 * K, 2 * N, false) != 0;
}

cudaError_t launch_tc_stem_gemm_large(const float2 *A, float2 *C, int64_t M, int k, int n,
                                      const DevBranch *d_branch_entry, const float2 *pool, BatchArgs ba,
                                      tn_precision prec, int *err, cudaStream_t st) {
    LgBSource bs;
    bs.br = d_branch_entry;
    bs.pool = pool;
    bs.ba = ba;
    return run_any(prec, A, bs, C, M, (int64_t)1 << k, (int64_t)1 << n, err, st);
}

}  // namespace tn
