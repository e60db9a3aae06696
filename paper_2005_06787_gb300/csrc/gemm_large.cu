// Complex GEMM on the tcgen05 tensor cores for large K and N (tn_cgemm with
// K >= 32 and N >= 64 complex, e.g. a stem step that absorbs a merged branch,
// Supp. A.3 "Branch merging"): C[m][nu] = sum_kappa A[m][kappa] B[kappa][nu],
// complex64, as the real GEMM of A viewed as [M][2K] with the 2K x 2N real
// expansion [[Br, Bi], [-Bi, Br]] of B (the same arithmetic as gemm_tc.cu).
//
// Design (one CTA per SM, persistent over 128 x BN output tiles, m-major so
// the CTAs working at one time share A rows in L2):
//   warp 0     one thread issues TMA loads into a ring of STAGES stages:
//              the FP32 A tile of the k-block (128-byte swizzled boxes of 32
//              floats x 128 rows) and the pre-split B tiles (B^T hi / lo in
//              the tensor-core type, K-major, built once per call by
//              lg_prep_b_kernel);
//   warps 4-11 converters: two threads (lanes l, l + 8) own row r of the A
//              tile, read it from the stage, split every value into hi + lo
//              of the tensor-core type (both rounded to nearest) and write
//              them back in the K-major 128-byte-swizzled layout the MMA
//              descriptors name - BF16: thread h reads box h of the row, and
//              after a warp barrier (both have read) writes the hi and lo
//              chunks of its 32 values over the first and second box; TF32:
//              thread h splits chunks 4h..4h+3, hi in place, lo into the
//              second box; one lane per warp then signals the stage;
//   warp 1     one thread issues the MMAs of a converted stage: hi*hi into
//              the main TMEM accumulator and (x3) hi*lo + lo*hi into a
//              correction accumulator (the tensor core's FP32 accumulation
//              truncates, so corrections stay apart from the full-size sum),
//              then commits the stage back to the producer;
//   warps 12-15 epilogue: after the tile's last commit, each thread reads its
//              TMEM lane (one row), adds main + correction with round to
//              nearest and stores the row; TMEM is double-buffered so the
//              epilogue of tile i overlaps the MMAs of tile i+1.
// Every wait is on an mbarrier and bounded in time; a wait that gives up
// records an error code (read by tn_device_status), and the kernel then waits
// (bounded) for its own copies and MMAs in flight before freeing TMEM.
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

// PREC 1: TF32 x3, 2: BF16 x3, 3: BF16 x1.
template <int PREC>
struct LgCfg {
    static constexpr bool X3 = PREC != 3;
    static constexpr bool TF32 = PREC == 1;
    static constexpr int BN = X3 ? 128 : 256;       // real output columns per tile
    static constexpr int KBLK = TF32 ? 32 : 64;     // real K per stage (128 B of operand per row)
    static constexpr int STAGES = 3;
    static constexpr uint32_t B_BYTES = (uint32_t)BN * 128;
    static constexpr uint32_t STAGE_BYTES = 2 * A_BOX_BYTES + B_BYTES * (X3 ? 2 : 1);
    static constexpr uint32_t TX_BYTES = (TF32 ? 1 : 2) * A_BOX_BYTES + B_BYTES * (X3 ? 2 : 1);
    static constexpr int ACC_COLS = BN * (X3 ? 2 : 1);  // TMEM columns per accumulator buffer
    static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE_BYTES;
};
static_assert(2 * LgCfg<1>::ACC_COLS <= 512 && 2 * LgCfg<2>::ACC_COLS <= 512 &&
                  2 * LgCfg<3>::ACC_COLS <= 512,
              "two accumulator buffers must fit the SM's 512 TMEM columns");

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
    // cluster-scope acquire: arrivals and copies may come from the other CTAs
    // of the cluster (multicast loads, multicast commits)
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
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
// The same tile copy delivered to the CTAs of the cluster in cta_mask, each at
// this CTA-relative address and signalled on the barrier at this address.
__device__ __forceinline__ void lg_tma2d_mc(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar, uint16_t cta_mask) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
        " [%0], [%1, {%2, %3}], [%4], %5;\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar), "h"(cta_mask)
        : "memory");
}
__device__ __forceinline__ void lg_commit_mc(uint32_t bar, uint16_t cta_mask) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], "
        "%1;\n" ::"r"(bar),
        "h"(cta_mask)
        : "memory");
}
__device__ __forceinline__ void lg_cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
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
template <bool TF32>
__device__ __forceinline__ void lg_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    }
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

// Cluster of CLM x CLN CTAs (rank = CLN * mr + nr) computing a CLM x CLN
// block of output tiles: CTA (mr, nr) takes m-tile CLM * i + mr and n-tile
// CLN * j + nr of super-tile (i, j). The CTAs of one m-tile share its A tile:
// each loads 1/CLN of it and multicasts it to them; the CTAs of one n-tile
// share its B tiles the same way. A stage is free once every CTA of the
// cluster has consumed it (each MMA commit is multicast to all of them).
template <int PREC, int CLM, int CLN>
__global__ void __launch_bounds__(LG_THREADS, 1)
    tc_cgemm_large_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBh,
                          const __grid_constant__ CUtensorMap tmBl, float *__restrict__ C, int64_t M,
                          int K2, int N2, int *err) {
    using Cf = LgCfg<PREC>;
    constexpr int BN = Cf::BN, S = Cf::STAGES, KBLK = Cf::KBLK;
    constexpr bool X3 = Cf::X3, TF32 = Cf::TF32;
    constexpr int CL = CLM * CLN;
    extern __shared__ __align__(1024) unsigned char lg_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(lg_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[S], conv_bar[S], empty_bar[S], tfull_bar[2], tempty_bar[2],
        drain_bar;
    __shared__ uint32_t tmem_base;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rank = (int)(blockIdx.x % CL), mr = rank / CLN, nr = rank % CLN;
    const int sn_tiles = N2 / BN / CLN;                        // super-tile columns
    const int64_t sm_tiles = ((M + 127) / 128 + CLM - 1) / CLM;  // super-tile rows
    const int64_t n_tot = sm_tiles * sn_tiles;                 // super-tiles
    const int64_t st0 = blockIdx.x / CL, st_step = gridDim.x / CL;
    const int kblocks = K2 / KBLK;
    // first row / column of this CTA's tile in super-tile t (rows past M are
    // read as zero and not stored)
    auto tile_m0 = [&](int64_t t) { return (int)(((t / sn_tiles) * CLM + mr) * 128); };
    auto tile_n0 = [&](int64_t t) { return (int)(((t % sn_tiles) * CLN + nr) * BN); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(lg_smem_u32(&full_bar[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(lg_smem_u32(&conv_bar[s])),
                         "n"(N_CONV));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(lg_smem_u32(&empty_bar[s])),
                         "n"(CL));
        }
        for (int a = 0; a < 2; ++a) {
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
    if constexpr (CL > 1) lg_cluster_sync();  // every barrier of the cluster is initialised
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
            // this CTA's share of the stage: A box nr (BF16: the k-block's
            // second 32 columns; TF32: rows 64 nr ..) for the CTAs of its
            // m-tile, B rows mr * BN / CLM .. for the CTAs of its n-tile
            uint16_t mask_a = 0, mask_b = 0;
            for (int j = 0; j < CLN; ++j) mask_a |= (uint16_t)(1u << (mr * CLN + j));
            for (int i = 0; i < CLM; ++i) mask_b |= (uint16_t)(1u << (i * CLN + nr));
            constexpr uint32_t B_PART = Cf::B_BYTES / CLM;
            auto a_part = [&](int k, int m0, uint32_t &off, int &x, int &y) {
                if constexpr (CLN == 1) {
                    off = 0; x = k; y = m0;
                } else if constexpr (TF32) {
                    off = (uint32_t)nr * (A_BOX_BYTES / 2); x = k; y = m0 + 64 * nr;
                } else {
                    off = (uint32_t)nr * A_BOX_BYTES; x = k + 32 * nr; y = m0;
                }
            };
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
                uint32_t off;
                int x, y;
                a_part(kk * KBLK, tile_m0(tt), off, x, y);
                lg_prefetch2d(&tmA, x, y);
                if constexpr (!TF32 && CLN == 1) lg_prefetch2d(&tmA, x + 32, y);
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
                    lg_arrive_tx(fb, Cf::TX_BYTES);  // the whole stage lands here, whoever loads it
                    const uint32_t st = sbase + (uint32_t)s * Cf::STAGE_BYTES;
                    const int k = kb * KBLK;
                    uint32_t aoff;
                    int ax, ay;
                    a_part(k, m0, aoff, ax, ay);
                    const uint32_t bh = st + 2 * A_BOX_BYTES + (uint32_t)mr * B_PART;
                    const uint32_t bl = bh + Cf::B_BYTES;
                    const int by = n0 + mr * (BN / CLM);
                    if constexpr (CLN == 1) {
                        lg_tma2d(st, &tmA, ax, ay, fb);
                        if constexpr (!TF32) lg_tma2d(st + A_BOX_BYTES, &tmA, ax + 32, ay, fb);
                    } else {
                        lg_tma2d_mc(st + aoff, &tmA, ax, ay, fb, mask_a);
                    }
                    if constexpr (CLM == 1) {
                        lg_tma2d(bh, &tmBh, k, by, fb);
                        if constexpr (X3) lg_tma2d(bl, &tmBl, k, by, fb);
                    } else {
                        lg_tma2d_mc(bh, &tmBh, k, by, fb, mask_b);
                        if constexpr (X3) lg_tma2d_mc(bl, &tmBl, k, by, fb, mask_b);
                    }
                }
            }
            if (!ok) atomicExch(err, 5);
            // before exit: the copies of the last use of every stage have
            // landed, and every CTA of the cluster has released it (no more
            // arrivals on this CTA's barriers will come)
            for (uint32_t u = it > (uint32_t)S ? it - S : 0; u < it; ++u) {
                lg_wait(lg_smem_u32(&full_bar[u % S]), (u / S) & 1);
                lg_wait(lg_smem_u32(&empty_bar[u % S]), (u / S) & 1);
            }
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
                if constexpr (TF32) {
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
                } else {
                    // row elements 32h .. 32h+31: box h of the row
                    const unsigned char *src = h ? a1 : a0;
                    float x[32];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const float4 v = *reinterpret_cast<const float4 *>(src + lg_sw(r, c));
                        x[4 * c] = v.x; x[4 * c + 1] = v.y; x[4 * c + 2] = v.z; x[4 * c + 3] = v.w;
                    }
                    __syncwarp();  // the partner lane has read its box of the row too
                    // BF16 chunk 4h + c of the row holds elements 32h + 8c .. 32h + 8c + 7
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float u0 = x[8 * c + 2 * q], u1 = x[8 * c + 2 * q + 1];
                            const __nv_bfloat162 hb = __floats2bfloat162_rn(u0, u1);
                            hw[q] = *reinterpret_cast<const uint32_t *>(&hb);
                            if constexpr (X3) {
                                const float2 hf = __bfloat1622float2(hb);
                                const __nv_bfloat162 lb = __floats2bfloat162_rn(u0 - hf.x, u1 - hf.y);
                                lw[q] = *reinterpret_cast<const uint32_t *>(&lb);
                            }
                        }
                        *reinterpret_cast<uint4 *>(a0 + lg_sw(r, 4 * h + c)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        if constexpr (X3)
                            *reinterpret_cast<uint4 *>(a1 + lg_sw(r, 4 * h + c)) =
                                make_uint4(lw[0], lw[1], lw[2], lw[3]);
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
            constexpr uint32_t idesc = lg_idesc(TF32 ? 2 : 1, BN, 128);
            uint32_t it = 0, tile_i = 0;
            bool ok = true;
            for (int64_t t = st0; t < n_tot && ok; t += st_step, ++tile_i) {
                const uint32_t acc = tile_i & 1, use = tile_i >> 1;
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
                        lg_mma<TF32>(d, ahi, bhi, idesc, accum);
                        if constexpr (X3) {
                            const uint64_t blo = lg_desc(st + 2 * A_BOX_BYTES + Cf::B_BYTES + ko);
                            lg_mma<TF32>(d + BN, ahi, blo, idesc, accum);
                            lg_mma<TF32>(d + BN, alo, bhi, idesc, 1u);
                        }
                    }
                    // stage free (in every CTA of the cluster) once these MMAs are done
                    if constexpr (CL == 1)
                        lg_commit(lg_smem_u32(&empty_bar[s]));
                    else
                        lg_commit_mc(lg_smem_u32(&empty_bar[s]), (uint16_t)((1u << CL) - 1));
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
        const int row = q * 32 + lane;
        uint32_t tile_i = 0;
        bool ok = true;
        for (int64_t t = st0; t < n_tot; t += st_step, ++tile_i) {
            const uint32_t acc = tile_i & 1, use = tile_i >> 1;
            if (!lg_wait(lg_smem_u32(&tfull_bar[acc]), use & 1)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            const int64_t m = (int64_t)tile_m0(t) + row;
            const int n0 = tile_n0(t);
            float *crow = C + m * (int64_t)N2 + n0;
            const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + acc * (uint32_t)Cf::ACC_COLS;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 16) {
                uint32_t v[16];
                lg_ld16(tbase + (uint32_t)c0, v);
                if constexpr (X3) {
                    uint32_t w[16];
                    lg_ld16(tbase + (uint32_t)(BN + c0), w);
                    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        v[j] = __float_as_uint(__fadd_rn(__uint_as_float(v[j]), __uint_as_float(w[j])));
                } else {
                    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                }
                if (m < M) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4 *>(crow + c0 + j) =
                            make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]),
                                        __uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]));
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n");
            __syncwarp();
            if (lane == 0) lg_arrive(lg_smem_u32(&tempty_bar[acc]));
        }
        if (!ok) atomicExch(err, 5);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if constexpr (CL > 1) lg_cluster_sync();  // no CTA leaves while others may still signal it
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

template <int PREC, int CLM, int CLN>
cudaError_t launch_large(const CUtensorMap &ma, const CUtensorMap &mbh, const CUtensorMap &mbl, float *C,
                         int64_t M, int K2, int N2, int *err, cudaStream_t st) {
    using Cf = LgCfg<PREC>;
    constexpr int CL = CLM * CLN;
    auto kern = tc_cgemm_large_kernel<PREC, CLM, CLN>;
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    static int max_clusters = 0;
    std::call_once(attr_once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cf::SMEM);
        if (attr_err == cudaSuccess && CL > 1)
            attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 0);
        if (attr_err != cudaSuccess) return;
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = CL;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(sms / CL * CL), 1, 1);
        cfg.blockDim = dim3(LG_THREADS, 1, 1);
        cfg.dynamicSmemBytes = Cf::SMEM;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg) != cudaSuccess || max_clusters < 1) {
            cudaGetLastError();
            max_clusters = std::max(1, sms / CL);
        }
    });
    if (attr_err != cudaSuccess) return attr_err;
    const int64_t n_super = (((M + 127) / 128 + CLM - 1) / CLM) * (N2 / Cf::BN / CLN);
    const int64_t clusters = std::max<int64_t>(1, std::min<int64_t>(n_super, max_clusters));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(clusters * CL), 1, 1);
    cfg.blockDim = dim3(LG_THREADS, 1, 1);
    cfg.dynamicSmemBytes = Cf::SMEM;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, ma, mbh, mbl, C, M, K2, N2, err);
}

template <int PREC>
cudaError_t run_large(const float2 *A, const float2 *B, float2 *C, int64_t M, int K, int N, int *err,
                      cudaStream_t st) {
    using Cf = LgCfg<PREC>;
    const int K2 = 2 * K, N2 = 2 * N;
    // one CTA per cluster: sharing A and B tiles between the CTAs of a 2 x 2
    // cluster by multicast was measured slower (each SM still takes in and
    // turns over the same bytes per stage, and a stage is then free only when
    // all four CTAs have consumed it)
    const int CLN = 1, CLM = 1;
    const size_t esz = Cf::TF32 ? 4 : 2;
    const size_t part = (size_t)N2 * K2 * esz;
    void *ws = nullptr;
    cudaError_t e = cudaMallocAsync(&ws, part * (Cf::X3 ? 2 : 1), st);
    if (e != cudaSuccess) return e;
    unsigned char *bhi = static_cast<unsigned char *>(ws), *blo = Cf::X3 ? bhi + part : bhi;
    const int64_t total = (int64_t)N2 * K2;
    lg_prep_b_kernel<PREC><<<(unsigned)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, st>>>(
        B, K, N, bhi, blo);
    e = cudaGetLastError();
    CUtensorMap ma, mbh, mbl;
    const CUtensorMapDataType bt = Cf::TF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const uint32_t bbox = Cf::TF32 ? 32 : 64;  // 128 bytes of K per row
    // per-CTA copies: TF32 A tiles split by rows between the two CTAs of an
    // m-tile, B tiles by rows between the CLM CTAs of an n-tile
    const uint32_t a_rows = (Cf::TF32 && CLN == 2) ? 64 : 128;
    const uint32_t b_rows = (uint32_t)(Cf::BN / CLM);
    if (e == cudaSuccess &&
        !(encode_2d(&ma, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, A, (uint64_t)K2, (uint64_t)M, 32, a_rows) &&
          encode_2d(&mbh, bt, esz, bhi, (uint64_t)K2, (uint64_t)N2, bbox, b_rows) &&
          encode_2d(&mbl, bt, esz, blo, (uint64_t)K2, (uint64_t)N2, bbox, b_rows)))
        e = cudaErrorInvalidValue;
    if (e == cudaSuccess) {
        float *Cf32 = reinterpret_cast<float *>(C);
        e = (CLM == 2 && CLN == 2) ? launch_large<PREC, 2, 2>(ma, mbh, mbl, Cf32, M, K2, N2, err, st)
                                   : launch_large<PREC, 1, 1>(ma, mbh, mbl, Cf32, M, K2, N2, err, st);
    }
    cudaError_t f = cudaFreeAsync(ws, st);
    return e != cudaSuccess ? e : f;
}

}  // namespace

bool tc_large_supported(int64_t M, int64_t K, int64_t N, tn_precision prec, const void *A, const void *C) {
    if (prec == TN_PREC_FP32_SIMT) return false;
    const int64_t bn = prec == TN_PREC_BF16x1 ? LgCfg<3>::BN : LgCfg<2>::BN;
    const bool aligned = !((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(C)) & 15);
    return aligned && M >= 128 && M < ((int64_t)1 << 31) && K >= 32 && (2 * K) % 64 == 0 &&
           K <= (1 << 20) && (2 * N) % bn == 0 && N <= (1 << 20);
}

cudaError_t launch_tc_cgemm_large(const float2 *A, const float2 *B, float2 *C, int64_t M, int64_t K,
                                  int64_t N, tn_precision prec, int *err, cudaStream_t st) {
    switch (prec) {
        case TN_PREC_TF32x3: return run_large<1>(A, B, C, M, (int)K, (int)N, err, st);
        case TN_PREC_BF16x3: return run_large<2>(A, B, C, M, (int)K, (int)N, err, st);
        case TN_PREC_BF16x1: return run_large<3>(A, B, C, M, (int)K, (int)N, err, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tn
