// The executable plan: scheme + stem plan + device resources.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <memory>

#include "internal.h"
#include "kernels.h"

namespace tn {

BuiltStem build_stem_plan(const Network &net, const Scheme &s, const tn_plan_opts &o);
// A pure-permutation pass (input bit j -> output bit perm[j]) for a rank-r
// tensor, its chunk table appended to chunks; validated.
DevPass make_permute_pass(int rank, const std::vector<int> &perm, std::vector<int> &chunks);

// ---- cost models and search (costmodel.cpp, mlp.cu)
constexpr int N_FEATURES = TN_N_FEATURES;
struct LaunchDesc {
    int kind;  // 0 fused pass, 1 GEMM step, 2 permute (plain)
    int items, r_in, r_out, n_steps, sum_k, sum_n, t_in, t_out;
    double bytes, flops;
};
int choose_batch(int max_rank, int n_sliced, int n_prefixes, int slice_batch);
std::vector<LaunchDesc> launch_list(const StemPlan &sp, tn_exec_mode mode, int items);
void launch_features(const LaunchDesc &d, tn_precision prec, float *f);
double flop_model_ms(const LaunchDesc &d, tn_precision prec);
struct Mlp;
Mlp *mlp_create(int n_in, int h1, int h2, uint64_t seed);
void mlp_destroy(Mlp *m);
int64_t mlp_n_params(const Mlp &m);
void mlp_set_params(Mlp &m, const float *p, int64_t n);
void mlp_get_params(const Mlp &m, float *p, int64_t n);
void mlp_loss_grad_host(Mlp &m, const float *X, const float *t, int rows, double *loss, float *grad);
double mlp_train(Mlp &m, const float *X, const float *t, int rows, int epochs, int batch, float lr,
                 uint64_t seed);
void mlp_predict(Mlp &m, const float *X, int rows, float *y);
struct SearchResult {
    int n_candidates = 0, n_launch_rows = 0;
    bool used_mlp = false;
    tn_plan_opts opts{}, mlp_opts{}, flop_opts{};
    double mlp_pick_mlp_ms = 0, mlp_pick_flop_ms = 0, flop_pick_mlp_ms = 0, flop_pick_flop_ms = 0;
    Scheme scheme;
    BuiltStem stem;
};
// Branch merges chosen one by one along the stem by the model's predicted
// time (mlp == nullptr: the plain model); returns the merged scheme.
Scheme choose_merges(const Network &net, const Scheme &base, const tn_plan_opts &o, Mlp *mlp,
                     tn_precision prec, int *n_joins);
SearchResult plan_search(const Network &net, const tn_plan_opts &base, const tn_search_opts &so,
                         Mlp *mlp, tn_precision prec);

struct DeviceArena {
    void *ptr = nullptr;
    size_t bytes = 0;
};

struct Plan {
    Network net;
    Scheme scheme;
    tn_plan_opts opts{};
    StemPlan sp;
    std::vector<BranchLayout> layouts;
    std::vector<DevBranch> h_branches;  // per cluster

    // device resources
    bool prepared = false;
    int device = -1;            // CUDA device the plan was prepared on
    int n_prefix = 0;
    int SB = 1;                 // slices per fused batch
    float2 *d_pool = nullptr;   // branch storage
    int64_t pool_elems = 0;
    DevBranch *d_branches = nullptr;
    DevPass *d_plain = nullptr, *d_fused = nullptr;
    int *d_chunks = nullptr;
    float2 *d_buf[2] = {nullptr, nullptr};
    int64_t buf_elems = 0;
    DevState *d_state = nullptr;
    double2 *d_sum = nullptr, *d_comp = nullptr, *d_out = nullptr;
    int *d_pos_plain = nullptr, *d_pos_fused = nullptr;
    int64_t device_bytes = 0;
    std::map<int, cudaGraphExec_t> graphs;  // per precision
    cudaStream_t graph_stream = nullptr;

    // hypergraph networks: a sequence of FP64 pairwise contractions
    bool hyper = false;
    HyperScheme hs;
    double2 *d_hleaf = nullptr;   // leaf values per prefix (FP64)
    int64_t h_leaf_total = 0;     // entries per prefix copy
    std::vector<int64_t> h_leaf_off;

    ~Plan();
    void release();
};

void plan_prepare(Plan &p, const uint8_t *prefixes, int n_prefixes, cudaStream_t st);
// Fails with TN_ERR_INVALID_ARG unless the plan is prepared and the current
// device is the one it was prepared on (its buffers live there).
void require_plan_device(const Plan &p);
std::vector<tn_launch_record> plan_profile(Plan &p, uint64_t s0, tn_precision prec,
                                          tn_exec_mode mode, cudaStream_t st);
void plan_contract_noalloc(Plan &p, uint64_t s0, uint64_t s1, cudaStream_t st, double *amps_out,
                           int accumulate);
void plan_contract(Plan &p, uint64_t s0, uint64_t s1, tn_precision prec, tn_exec_mode mode,
                   cudaStream_t st, double *amps_out, int accumulate);
// Hypergraph plans (hyper.cpp, executor.cu): upload the leaves of each prefix;
// contract slice range [0, 1) (no slicing) as FP64 pairwise steps on the GPU.
void hyper_prepare(Plan &p, const uint8_t *prefixes, int n_prefixes, cudaStream_t st);
void hyper_contract(Plan &p, uint64_t s0, uint64_t s1, cudaStream_t st, double *amps_out,
                    int accumulate);

#define TN_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t _e = (call);                                                           \
        if (_e != cudaSuccess)                                                             \
            ::tn::fail(_e == cudaErrorMemoryAllocation ? TN_ERR_OOM : TN_ERR_CUDA,         \
                       std::string(#call) + ": " + cudaGetErrorString(_e));                \
    } while (0)

}  // namespace tn
