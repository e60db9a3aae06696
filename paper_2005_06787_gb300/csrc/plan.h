// The executable plan: scheme + stem plan + device resources.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <memory>

#include "internal.h"
#include "kernels.h"

namespace tn {

struct BuiltStem;
BuiltStem build_stem_plan(const Network &net, const Scheme &s, const tn_plan_opts &o);

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

    ~Plan();
    void release();
};

void plan_prepare(Plan &p, const uint8_t *prefixes, int n_prefixes, cudaStream_t st);
std::vector<tn_launch_record> plan_profile(Plan &p, uint64_t s0, tn_precision prec,
                                          tn_exec_mode mode, cudaStream_t st);
void plan_contract_noalloc(Plan &p, uint64_t s0, uint64_t s1, cudaStream_t st, double *amps_out,
                           int accumulate);
void plan_contract(Plan &p, uint64_t s0, uint64_t s1, tn_precision prec, tn_exec_mode mode,
                   cudaStream_t st, double *amps_out, int accumulate);

#define TN_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t _e = (call);                                                           \
        if (_e != cudaSuccess)                                                             \
            ::tn::fail(_e == cudaErrorMemoryAllocation ? TN_ERR_OOM : TN_ERR_CUDA,         \
                       std::string(#call) + ": " + cudaGetErrorString(_e));                \
    } while (0)

}  // namespace tn
