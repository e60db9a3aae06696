/*
 * tnstem: stem contraction of random-circuit tensor networks on one GB300.
 *
 * C interface of libtnstem.so. Every entry point returns a tn_status and never
 * throws; tn_last_error() gives the calling thread's last message.
 *
 * What the library computes (paper: "Classical Simulation of Quantum
 * Supremacy Circuits", Huang et al., arXiv:2005.06787):
 *   - the tensor network of a Sycamore-style random circuit (Sec. 2, Sec. 3);
 *   - a slicing-incorporated contraction scheme (E_s, T) (Supp. A.1,
 *     "Slicing") whose contraction tree has a stem and branches (Sec. 4,
 *     Supp. A.2), found by stem growth, local optimisation and dynamic
 *     slicing (Sec. 4, Supp. A.2), or given by the caller;
 *   - for a range of slices, the sum of the sub-network values (Supp. A.1):
 *     the amplitudes of a batch of bitstrings whose open qubits take every
 *     assignment (Sec. 3, "open tensor network", 64 amplitudes for 6 open
 *     qubits), with branches pre-computed once (Supp. A.3).
 *
 * Conventions.
 *   Qubits are 0..n-1. A bitstring prefix gives one bit per closed qubit
 *   (qubits not listed as open), in ascending qubit order.
 *   Amplitude index: the open qubits in the order given, first one = most
 *   significant bit. Amplitudes are returned as interleaved (re, im) doubles.
 *   Edges of the network are wire segments (q, s): segment s of qubit q
 *   follows the s-th gate acting on q (segment 0 follows |0>).
 *   Leaves are numbered: |0> on qubits 0..n-1; then per cycle t < m the
 *   single-qubit gates of layer t on qubits 0..n-1 followed by the two-qubit
 *   gates of layer t in listed order; then the final single-qubit layer; then
 *   one projector per closed qubit, ascending. An order is an SSA pair list:
 *   the k-th pair creates node n_leaves + k.
 *   Slice id s fixes sliced edge j (in the plan's sliced list) to bit j of s.
 *
 * Ownership. Handles are opaque and owned by the library until destroyed.
 * Input arrays are copied. Output arrays are owned by the caller.
 */
#ifndef TNSTEM_H
#define TNSTEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TN_OK = 0,
    TN_ERR_INVALID_ARG = 1,     /* bad pointer, size, range, order or edge */
    TN_ERR_OOM = 2,             /* device or host allocation failed */
    TN_ERR_CUDA = 3,            /* a CUDA call failed (message has the name) */
    TN_ERR_PLAN_INFEASIBLE = 4, /* no scheme within the width limit */
    TN_ERR_TIMEOUT = 5,         /* a bounded device wait ran out */
    TN_ERR_UNSUPPORTED = 6      /* shape outside what the kernels handle */
} tn_status;

/* Arithmetic of the stem's GEMM steps (Sec. 6 notes tensor cores were left
 * unused by the paper; these are this library's options). Fused memory-bound
 * passes always compute in FP32 on the CUDA cores. */
typedef enum {
    TN_PREC_FP32_SIMT = 0, /* FP32 FMA on CUDA cores */
    TN_PREC_TF32x3 = 1,    /* tcgen05, split TF32 hi/lo, 3 products, FP32 accumulate */
    TN_PREC_BF16x3 = 2,    /* tcgen05, split BF16 hi/lo, 3 products, FP32 accumulate */
    TN_PREC_BF16x1 = 3     /* tcgen05, one BF16 product, FP32 accumulate */
} tn_precision;

/* How the stem is executed. */
typedef enum {
    TN_EXEC_PLAIN = 0, /* per stem step: a permute then a complex GEMM, one slice per launch */
    TN_EXEC_FUSED = 1  /* consecutive steps fused into one HBM pass, slices batched, graph replay */
} tn_exec_mode;

typedef struct {
    int32_t n_qubits;
    int32_t n_cycles;            /* m */
    const int8_t *gates_1q;      /* (m+1) * n_qubits ids: 0 sqrt(X), 1 sqrt(Y), 2 sqrt(W) */
    const int32_t *pair_offsets; /* m + 1 offsets into pairs (in pairs, not ints) */
    const int32_t *pairs;        /* flattened (qa, qb), qa < qb, per two-qubit layer */
    double theta, phi;           /* fSim parameters, the same on every coupler */
} tn_circuit;

typedef struct tn_network tn_network;
typedef struct tn_plan tn_plan;

typedef struct {
    int32_t cw_limit;         /* max log2 entries of any intermediate tensor, e.g. 30 */
    int32_t min_sliced;       /* slice at least this many edges (0 = only as needed) */
    int32_t max_sliced;       /* give up beyond this many sliced edges */
    int32_t restarts;         /* randomised stem-growth restarts */
    int32_t local_opt_iters;  /* local-optimisation sweeps before/between/after slicing */
    int32_t branch_rank;      /* max rank of a branch cluster (default 4) */
    int32_t slice_batch;      /* batch items per launch in fused mode (0 = auto) */
    int32_t tile_bits;        /* fused-pass tile size log2 (0 = auto, <= 12) */
    int32_t max_pass_steps;   /* steps fused into one pass (0 = auto) */
    int32_t gemm_min_kn;      /* steps with k or n >= this run as GEMM (0 = auto) */
    int32_t merge_group;      /* Supp. A.3 branch merging: merge runs of this many
                                 consecutive stem branches into one (0/1 = off);
                                 < 0: choose the merges branch by branch, each
                                 join kept when the plain FLOP-and-memory model
                                 predicts the whole plan faster (tn_plan_search
                                 makes the same choice with the learned model) */
    int32_t merge_rank_cap;   /* largest rank of a merged branch (0 = 10) */
    int32_t anneal_iters;     /* simulated-annealing moves on the stem order per
                                 restart (0 = auto: 600 per branch cluster, at
                                 most 200000; < 0 = none) */
    int32_t slice_restarts;   /* slice and refine only this many of the restarts'
                                 annealed stems, the best by unsliced cost plus
                                 width excess (0 = all) */
    uint64_t seed;
    int32_t start_cluster;    /* the first restart grows its stem from this branch
                                 cluster (clusters are numbered for the seed's
                                 random stream), without noise (default 0) */
    int32_t stem_starts;      /* > 0: instead of the restarts, grow stems without
                                 noise from this many start clusters spread
                                 evenly over all clusters (every cluster when
                                 there are fewer), each annealed, sliced and
                                 refined on the host's threads; the cheapest
                                 scheme wins, whatever the thread count (0 = off) */
    double width_area_weight; /* > 0: the unsliced stem anneal also scores this
                                 weight times the stem's excess width summed
                                 over its tensors (sum of max(0, rank -
                                 cw_limit)), so stems that stay wide only
                                 briefly win; pays where slicing must remove
                                 many bits of width (0 = off) */
} tn_plan_opts;

typedef struct {
    double log2_tc;           /* log2 tc((E_s, T)) over all slices */
    double stem_tc_per_slice; /* sum over stem steps of 2^|E_u|, one slice */
    double branch_tc;         /* pre-computation cost, once per prefix */
    int32_t cw;               /* contraction width (sliced) */
    int32_t n_sliced;
    int32_t n_stem_steps;
    int32_t n_branches;
    int32_t n_passes_fused;
    int32_t n_gemm_steps;     /* steps run as a GEMM in fused mode */
    int32_t n_open;
    int32_t n_prefixes;
    int32_t batch_items;      /* items (prefix, slice) per fused launch */
    double stem_bytes_plain;  /* algorithmic HBM bytes per slice, plain mode */
    double stem_bytes_fused;  /* algorithmic HBM bytes per slice, fused mode */
    double max_stem_elems;    /* largest stem tensor, entries */
    int64_t device_bytes;     /* device memory held by the plan */
    int32_t n_passes_cbank;   /* fused passes that take branch matrices from
                                 the constant bank ((2,2) steps and paired
                                 (2,1), (1,3), (1,2) steps, in launches with
                                 one batch item); each launch of one is
                                 preceded by a one-block staging kernel and a
                                 device-to-device copy */
    int32_t pad_;
} tn_plan_stats;

/* One stem step as the plan runs it (features for cost models). */
typedef struct {
    int32_t r_in, r_out;      /* stem rank before / after */
    int32_t k, n;             /* contracted / new bits: C[m,n] = sum_k S[m,k] B[k,n] */
    int32_t pass;             /* fused pass index holding this step (-1: GEMM step) */
    int32_t gemm;             /* 1 if run as a tensor-core GEMM in fused mode */
    int32_t pair;             /* 1 if its fused pass takes the rest indices in
                                 adjacent pairs (16-byte shared-memory accesses) */
} tn_step_info;

/* Sec. 2-3: build the network of circuit c with the listed open qubits and the
 * closed qubits projected on closed_bits (n_qubits - n_open bytes, 0/1).
 * No device work. */
tn_status tn_build_network(const tn_circuit *c, const int32_t *open_qubits, int32_t n_open,
                           const uint8_t *closed_bits, tn_network **out);

/* Sec. 3 and Supp. A.1 (a network is a multi-hypergraph; hyperedges carry
 * the diagonal parts of gates): the same circuit as tn_build_network, with
 * each fSim(pi/2, phi) written as the wire swap times
 * diag(1, -i, -i, e^{-i phi}) - a rank-2 leaf on the two current wire
 * indices, which the two wires then exchange. An index is created only by
 * |0> and single-qubit gates: edge e is index (qubit[e], segment[e]), the one
 * qubit[e]'s segment[e]-th single-qubit gate created (segment 0: its |0>),
 * and it may join more than two leaves. Leaves are numbered as for
 * tn_build_network (a two-qubit gate is one leaf either way). Plans of such a
 * network (tn_plan_create) take a given order or a greedy one in which each
 * step keeps the shared edges that other tensors still hold, are not sliced
 * (sliced_edges must be NULL; TN_ERR_PLAN_INFEASIBLE above opts->cw_limit),
 * and contract on the GPU as FP64 pairwise steps for the single slice [0, 1)
 * whatever the precision and mode arguments; tn_plan_steps, tn_plan_profile,
 * tn_plan_features, tn_contract_stem_noalloc and tn_plan_search answer
 * TN_ERR_UNSUPPORTED for them. Needs |cos theta| <= 1e-12, else
 * TN_ERR_UNSUPPORTED. No device work. */
tn_status tn_build_hypernetwork(const tn_circuit *c, const int32_t *open_qubits, int32_t n_open,
                                const uint8_t *closed_bits, tn_network **out);

/* Number of leaves and edges; edge e is wire segment (qubit[e], segment[e]).
 * Any output pointer may be NULL; arrays hold n_edges entries. */
tn_status tn_network_info(const tn_network *net, int32_t *n_leaves, int32_t *n_edges,
                          int32_t *qubit, int32_t *segment);

/* Sec. 3: re-value the closed-qubit projectors <b| of net with a new prefix
 * (n_qubits - n_open bytes, 0/1; else TN_ERR_INVALID_ARG and net unchanged).
 * The network's structure is kept, so an order or sliced set found for it
 * stays valid. Plans copy the network when created: a plan made before this
 * call keeps its old prefix (tn_plan_prepare takes explicit prefixes). Host
 * only. */
tn_status tn_set_prefix(tn_network *net, const uint8_t *closed_bits);

/* Supp. A.1-A.2: make a contraction scheme. order (n_pairs = n_leaves - 1
 * SSA pairs) may be NULL: the planner then grows a stem (Sec. 4). sliced_edges
 * may be NULL: the planner then slices greedily (Supp. A.2, "Dynamic slicing")
 * until the width is within opts->cw_limit. Host-only; no device work. */
tn_status tn_plan_create(tn_network *net, const int32_t *order, int32_t n_pairs,
                         const int32_t *sliced_edges, int32_t n_sliced,
                         const tn_plan_opts *opts, tn_plan **out);

/* Upload leaves for n_prefixes bitstring prefixes (n_prefixes * n_closed
 * bytes; NULL = the network's own prefix) and pre-compute every branch on
 * the device, once (Supp. A.3, "Pre-computation"). Allocates device memory
 * on the current CUDA device; tn_contract_stem, tn_contract_stem_noalloc and
 * tn_plan_profile must then be called with that device current (else
 * TN_ERR_INVALID_ARG). Must precede tn_contract_stem; may be called again to
 * change prefixes. */
tn_status tn_plan_prepare(tn_plan *plan, const uint8_t *prefixes, int32_t n_prefixes,
                          void *cuda_stream);

tn_status tn_plan_info(const tn_plan *plan, tn_plan_stats *out);

/* Export the scheme: order (2*(n_leaves-1) ints, SSA pairs over the leaves),
 * sliced edge ids (n_sliced ints, slice-bit order). Either may be NULL. */
tn_status tn_plan_export(const tn_plan *plan, int32_t *order, int32_t *sliced_edges);

/* Per-step shapes; writes min(max_steps, n_stem_steps) records. */
tn_status tn_plan_steps(const tn_plan *plan, tn_step_info *out, int32_t max_steps,
                        int32_t *n_written);

/* Supp. A.1 "Slicing": contract slices [slice_begin, slice_end) for every
 * prepared prefix and add their values. amps_out holds n_prefixes * 2^n_open
 * (re, im) doubles, prefix-major; host or device memory. With accumulate != 0
 * the result is added to amps_out. The slice sum is kept in FP64 with
 * Neumaier compensation on the device, so disjoint ranges add. Asynchronous
 * on cuda_stream when amps_out is device memory; synchronises otherwise.
 * slice_end <= 2^n_sliced, else TN_ERR_INVALID_ARG. */
tn_status tn_contract_stem(tn_plan *plan, uint64_t slice_begin, uint64_t slice_end,
                           tn_precision prec, tn_exec_mode mode, void *cuda_stream,
                           double *amps_out, int32_t accumulate);

/* One kernel launch of a profiled batch. */
typedef struct {
    int32_t kind;     /* 0 fused pass, 1 GEMM step, 2 permute (plain), 3 slice sum */
    int32_t index;    /* position in the batch's launch sequence */
    int32_t r_in, r_out;
    int32_t n_steps;  /* stem steps applied by this launch */
    int32_t k, n;     /* GEMM steps: contracted / new bits */
    int32_t items;    /* batch items (prefix, slice) processed */
    double ms;        /* CUDA-event duration on the launch stream */
    double bytes;     /* algorithmic HBM bytes: 8 * (2^r_in + 2^r_out) per item */
    double flops;     /* algorithmic flops: 8 * sum of 2^|E_u| over its steps, per item */
} tn_launch_record;

/* Run one batch starting at slice_begin launch by launch, timing each launch
 * with CUDA events on cuda_stream (per-step timing, Supp. A.4 "explicit
 * simulations of subtasks"). Writes up to max_records records; n_records
 * receives the count. Synchronises cuda_stream. */
tn_status tn_plan_profile(tn_plan *plan, uint64_t slice_begin, tn_precision prec,
                          tn_exec_mode mode, void *cuda_stream, tn_launch_record *out,
                          int32_t max_records, int32_t *n_records);

/* Allocation-free variant of tn_contract_stem (fused mode, FP32). The paper
 * has no counterpart; this exists for callers that must not allocate device
 * memory while contracting: cudaMalloc synchronises the device and can fail
 * under a memory budget owned by someone else (a framework's pooling
 * allocator, a GPU shared under a fixed quota). Scratch lives in one static
 * device array of the library (two stem buffers of 2^20 complex64 entries and
 * 2^14 compensated FP64 sums, about 16.5 MiB held on every GPU that loads the
 * library until exit). Requirements: the plan is prepared (tn_plan_prepare
 * allocates; this call does not), n_prefixes * 2^max_rank <= 2^20 and
 * n_prefixes * 2^n_open <= 2^14, else TN_ERR_UNSUPPORTED; amps_out is device
 * memory (else TN_ERR_INVALID_ARG). Arguments and result are as for
 * tn_contract_stem. The first call on each device looks up the array's
 * address (cudaGetSymbolAddress) and must come before any stream capture on
 * the calling thread. All calls share the array and each clears the sums it
 * uses first; calls that overlap on the GPU race, so serialise them.
 * Asynchronous on cuda_stream. */
tn_status tn_contract_stem_noalloc(tn_plan *plan, uint64_t slice_begin, uint64_t slice_end,
                                   void *cuda_stream, double *amps_out, int32_t accumulate);

/* Free a handle (NULL is a no-op). tn_destroy_plan / tn_destroy_network are
 * the same calls under their short names. Synchronise the stream that used
 * a plan before destroying it. */
void tn_plan_destroy(tn_plan *plan);
void tn_network_destroy(tn_network *net);
void tn_destroy_plan(tn_plan *plan);
void tn_destroy_network(tn_network *net);

/* ---- learned step-time cost model and plan search (no counterpart in the
 * paper, whose order search is KaHyPar + CMA-ES; here candidate plans are
 * scored per kernel launch) ---- */

/* Features of each kernel launch of one batch, in launch order (the order of
 * tn_plan_profile's records of kinds 0-2): is_pass, is_gemm, is_permute,
 * log2(items)/16, r_in/32, r_out/32, steps/8, sum k/16, sum n/16,
 * tile bits in/16, tile bits out/16, log2(bytes)/40, log2(flops+1)/50,
 * GEMM precision one-hot (tf32x3, bf16x3, bf16x1). flop_ms receives the plain
 * FLOP-and-memory model's time of each launch (max of bytes / HBM bandwidth
 * and flops / arithmetic rate, plus launch overhead). */
#define TN_N_FEATURES 16
tn_status tn_plan_features(const tn_plan *plan, tn_precision prec, tn_exec_mode mode, float *X,
                           double *flop_ms, int32_t max_rows, int32_t *n_rows);

/* MLP n_in -> h1 (ReLU) -> h2 (ReLU) -> 1, trained and run on the GPU by the
 * library's own kernels. Parameters, one FP32 vector: W1 [h1][n_in], b1 [h1],
 * W2 [h2][h1], b2 [h2], W3 [h2], b3. Loss: mean squared error. Host arrays:
 * X row-major [rows][n_in], targets t [rows]. */
typedef struct tn_mlp tn_mlp;
tn_status tn_mlp_create(int32_t n_in, int32_t h1, int32_t h2, uint64_t seed, tn_mlp **out);
tn_status tn_mlp_n_params(const tn_mlp *m, int64_t *n);
tn_status tn_mlp_set_params(tn_mlp *m, const float *params, int64_t n);
tn_status tn_mlp_get_params(const tn_mlp *m, float *params, int64_t n);
/* One forward + backward pass over all rows: loss and gradient (grad may be NULL). */
tn_status tn_mlp_loss_grad(tn_mlp *m, const float *X, const float *t, int32_t rows,
                           double *loss, float *grad);
/* Mini-batch Adam; final_loss = mean batch loss of the last epoch. */
tn_status tn_mlp_train(tn_mlp *m, const float *X, const float *t, int32_t rows, int32_t epochs,
                       int32_t batch, float lr, uint64_t seed, double *final_loss);
tn_status tn_mlp_predict(tn_mlp *m, const float *X, int32_t rows, float *y);
void tn_mlp_destroy(tn_mlp *m);

typedef struct {
    int32_t n_seeds;        /* stem-growth seeds (each gives 3 x 5 x 3 variants, plus
                               one with branch merges chosen branch by branch by
                               the primary model from the seed's best unmerged
                               variant, merge_group -1) */
    double fallback_factor;    /* fall back if the MLP pick's plain-model time exceeds
                               this factor times the plain model's best (0 = 4) */
} tn_search_opts;

typedef struct {
    int32_t n_candidates, n_launch_rows, used_mlp;
    tn_plan_opts chosen, mlp_pick, flop_pick;
    double mlp_pick_mlp_ms, mlp_pick_flop_ms;   /* predicted time over all slices */
    double flop_pick_mlp_ms, flop_pick_flop_ms;
} tn_search_report;

/* Search candidate plans (base options with varied seed, tile bits, steps per
 * pass and branch merging), score every launch of every candidate with the
 * MLP (NULL: plain model only) for precision prec, and return the chosen plan
 * (not prepared) and a report of both models' picks. */
tn_status tn_plan_search(tn_network *net, const tn_plan_opts *base, const tn_search_opts *so,
                         tn_mlp *mlp, tn_precision prec, tn_plan **out, tn_search_report *report);

/* Device-side waits (no counterpart in the paper): every wait inside a
 * kernel of this library on a tensor-core operation is bounded; one that
 * gives up records a flag instead of hanging. This call synchronises the
 * device, reads the flag and returns TN_ERR_TIMEOUT if a wait ever gave up,
 * else TN_OK. Results of calls made after a wait gave up are not to be
 * trusted. */
tn_status tn_device_status(void);

/* Sec. 2 (after the frugal rejection sampling the paper cites as MFI+18):
 * turn amplitude batches into samples. amps_dev holds n_batches x batch_size
 * complex amplitudes (FP64 re, im interleaved; e.g. the 2^n_open amplitudes
 * of one bitstring prefix per batch, as tn_contract_stem writes them).
 * Candidate j of batch b is accepted when u[b][j] < 2^n_qubits p / M, p =
 * re^2 + im^2 (acceptance probability min(1, 2^n p / M) for u uniform in
 * [0, 1)), evaluated in FP64 without fused multiply-adds. The batch's sample
 * is the accepted candidate with the smallest key[b][j] (a random visiting
 * order), or -1. u_dev and key_dev are n_batches x batch_size doubles; the
 * caller draws them, so results are reproducible. Outputs (device,
 * caller-owned): index_dev[b], accepted_dev[b] (number accepted) and
 * picked_dev[2b..2b+1] (the sampled amplitude, 0 if none). All pointers must
 * be device memory (else TN_ERR_INVALID_ARG); 1 <= batch_size <= 2^20,
 * 1 <= n_qubits <= 1000, M > 0. Asynchronous on cuda_stream. */
tn_status tn_frugal_sample(const double *amps_dev, const double *u_dev, const double *key_dev,
                           int64_t n_batches, int32_t batch_size, int32_t n_qubits, double M,
                           void *cuda_stream, int32_t *index_dev, int32_t *accepted_dev,
                           double *picked_dev);

/* Roofline denominator of the fused stem pass (no counterpart in the paper,
 * whose Table 1 efficiencies divide by a nominal 15.7 TFLOP/s): the FP32 FMA
 * rate this GPU reaches, measured by a kernel of independent FMA chains on
 * every SM (best of three timed launches after one warm-up, CUDA events on
 * cuda_stream). Writes TFLOP/s (2 flops per FMA) to *tflops and the SM count
 * to *sm_count (host pointers). Synchronises cuda_stream. */
tn_status tn_fp32_fma_peak(void *cuda_stream, double *tflops, int32_t *sm_count);

/* Sec. 2: linear XEB 2^n <p> - 1 of count amplitudes (interleaved re, im,
 * device memory), p = |amp|^2, computed in FP64 on the device. out is a host
 * double. Synchronises cuda_stream. */
tn_status tn_linear_xeb(const double *amps_dev, int64_t count, int32_t n_qubits,
                        void *cuda_stream, double *out);

/* ---- single kernels, for tests and tuning (device pointers, complex64 as
 * interleaved float pairs) ---- */

/* Bit permutation of a 2^rank tensor: input bit j moves to output bit
 * perm[j]. Supp. A.1 "up to transposition". For rank >= 4 and 16-byte
 * aligned tensors it runs as a tiled pass through shared memory (128-byte
 * chunks in and out); otherwise element by element. in and out must not
 * overlap. Synchronises cuda_stream. */
tn_status tn_permute(const float *in, float *out, int32_t rank, const int32_t *perm,
                     void *cuda_stream);

/* Complex GEMM C[b][m][n] = sum_k A[b][m][k] * B[b][k][n], row-major, batch
 * strides in complex elements (0 broadcasts). One stem step, Supp. A.1
 * (a pairwise contraction is a GEMM after permutation); large K and N are the
 * steps that absorb merged branches (Supp. A.3 "Branch merging"). FP32 runs
 * on the CUDA cores; the tensor-core precisions on tcgen05, with a
 * TMA-pipelined kernel when K >= 32, 2N is a multiple of 128 (x3) or 256
 * (BF16 x1), M >= 128 and A, C are 16-byte aligned (it allocates a
 * stream-ordered workspace of 2 x 2N x 2K operand elements for the split B).
 * Asynchronous on cuda_stream: a tensor-core wait that gave up is reported by
 * tn_device_status. */
tn_status tn_cgemm(const float *A, const float *B, float *C, int64_t M, int64_t K, int64_t N,
                   int64_t batch, int64_t strideA, int64_t strideB, int64_t strideC,
                   tn_precision prec, void *cuda_stream);

const char *tn_last_error(void);
const char *tn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TNSTEM_H */
