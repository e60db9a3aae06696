// Internal data structures of libtnstem: network, contraction scheme, stem
// plan and the device descriptors the kernels read.
#pragma once

#include <complex>
#include <cstddef>
#include <cstdint>
#include <random>
#include <string>
#include <vector>

#include "tnstem.h"

namespace tn {

using cd = std::complex<double>;

// ----------------------------------------------------------------- errors
struct Error {
    tn_status code;
    std::string msg;
};
[[noreturn]] void fail(tn_status code, const std::string &msg);
void set_last_error(const std::string &msg);

// ----------------------------------------------------------------- bitset
struct Bits {
    std::vector<uint64_t> w;
    Bits() = default;
    explicit Bits(int nbits) : w((size_t)((nbits + 63) / 64), 0ull) {}
    void set(int i) { w[(size_t)i >> 6] |= 1ull << (i & 63); }
    void reset(int i) { w[(size_t)i >> 6] &= ~(1ull << (i & 63)); }
    bool test(int i) const { return (w[(size_t)i >> 6] >> (i & 63)) & 1ull; }
    int count() const {
        int c = 0;
        for (uint64_t x : w) c += __builtin_popcountll(x);
        return c;
    }
    Bits &operator^=(const Bits &o) {
        for (size_t i = 0; i < w.size(); ++i) w[i] ^= o.w[i];
        return *this;
    }
    Bits &operator|=(const Bits &o) {
        for (size_t i = 0; i < w.size(); ++i) w[i] |= o.w[i];
        return *this;
    }
    Bits &operator&=(const Bits &o) {
        for (size_t i = 0; i < w.size(); ++i) w[i] &= o.w[i];
        return *this;
    }
    Bits andnot(const Bits &o) const {
        Bits r = *this;
        for (size_t i = 0; i < w.size(); ++i) r.w[i] &= ~o.w[i];
        return r;
    }
    bool any() const {
        for (uint64_t x : w)
            if (x) return true;
        return false;
    }
    bool operator==(const Bits &o) const { return w == o.w; }
    std::vector<int> list() const {
        std::vector<int> r;
        for (size_t i = 0; i < w.size(); ++i) {
            uint64_t x = w[i];
            while (x) {
                int b = __builtin_ctzll(x);
                r.push_back((int)(i * 64 + b));
                x &= x - 1;
            }
        }
        return r;
    }
};
inline Bits operator^(Bits a, const Bits &b) { return a ^= b; }
inline Bits operator|(Bits a, const Bits &b) { return a |= b; }
inline Bits operator&(Bits a, const Bits &b) { return a &= b; }
inline int count_and(const Bits &a, const Bits &b) {
    int c = 0;
    for (size_t i = 0; i < a.w.size(); ++i) c += __builtin_popcountll(a.w[i] & b.w[i]);
    return c;
}
inline int count_or(const Bits &a, const Bits &b) {
    int c = 0;
    for (size_t i = 0; i < a.w.size(); ++i) c += __builtin_popcountll(a.w[i] | b.w[i]);
    return c;
}
inline int count_xor(const Bits &a, const Bits &b) {
    int c = 0;
    for (size_t i = 0; i < a.w.size(); ++i) c += __builtin_popcountll(a.w[i] ^ b.w[i]);
    return c;
}

// ----------------------------------------------------------------- network
// LEAF_DIAG: in a hypergraph network, the rank-2 diagonal part of fSim(pi/2,
// phi) on the two wire indices of a gate (the wires then exchange indices).
enum LeafKind { LEAF_ZERO = 0, LEAF_1Q = 1, LEAF_2Q = 2, LEAF_PROJ = 3, LEAF_DIAG = 4 };

struct Leaf {
    int kind;
    int qa, qb;              // qubits (qb = -1 for one-qubit leaves)
    int gate;                // single-qubit gate id, or closed index for projectors
    std::vector<int> edges;  // edge at bit position j of the value index
    std::vector<cd> vals;    // 2^rank values, index = sum_j a_{edges[j]} 2^j
};

struct EdgeInfo {
    int qubit, segment;
    int ends[2];
    int n_ends;
    bool open;
};

struct Network {
    bool hyper = false;  // multi-hypergraph (an index may join more than two leaves)
    int n_qubits = 0, n_cycles = 0;
    double theta = 0, phi = 0;
    std::vector<Leaf> leaves;
    std::vector<EdgeInfo> edges;
    std::vector<int> open_qubits, open_edges;  // open_edges[i] belongs to open_qubits[i]
    std::vector<int> closed_qubits;
    std::vector<uint8_t> closed_bits;
    std::vector<int> proj_leaf;  // leaf id of the projector of closed qubit i
    int n_edges() const { return (int)edges.size(); }
    int n_leaves() const { return (int)leaves.size(); }
};

// hyper = true: the multi-hypergraph form (Supp. A.1; Sec. 3, hyperedges for
// diagonal gate parts): needs fSim(pi/2, phi), the wire swap times a diagonal
// gate; each two-qubit gate becomes a LEAF_DIAG on the two wire indices.
Network build_network(const tn_circuit &c, const int32_t *open_qubits, int n_open,
                      const uint8_t *closed_bits, bool hyper = false);

// Contraction scheme of a hypergraph network: SSA pairs over the leaves and
// the edges each new node keeps (E*_AB of Supp. A.1: the pair's edges that
// are open or still held by another tensor); the last node keeps the open
// edges, the first open qubit at the most significant bit. tc sums 2^|E_AB|,
// cw maxes |E*_AB|.
struct HyperScheme {
    std::vector<std::pair<int, int>> pairs;
    std::vector<std::vector<int>> node_edges;
    double log2_tc = 0;
    int cw = 0;
};
// order == nullptr: greedy pairs (smallest 2^|out| - 2^|a| - 2^|b|, ties by
// the smaller ids), over `restarts` runs (all but the first with noise on the
// scores, from `seed`): the cheapest scheme within cw_limit, else the
// narrowest; otherwise the given SSA order, validated.
HyperScheme hyper_scheme(const Network &net, const std::vector<std::pair<int, int>> *order, int restarts,
                         uint64_t seed, int cw_limit);
// Re-value the closed-qubit projectors (Sec. 3 post-selection); the structure,
// and so any plan made from it, is unchanged.
void set_prefix(Network &net, const uint8_t *closed_bits);
void gate_matrix_1q(int id, cd out[4]);
void fsim_matrix(double theta, double phi, cd out[16]);

// ----------------------------------------------------------------- scheme
// A subtree is a list of SSA-style pairs over "refs": ref >= 0 is a leaf id,
// ref < 0 is -(j+1) for the j-th pair of the same list.
using PairList = std::vector<std::pair<int, int>>;

struct Cluster {
    std::vector<int> leaves;
    PairList pairs;  // internal pairs (leaves.size() - 1 of them)
    Bits out;        // output edges over the full network (sliced included)
};

// One stem step: the stem absorbs cluster `branch`.
struct StemStep {
    int branch;
    std::vector<int> K;     // contracted edges (stem ∩ branch), unsliced
    std::vector<int> Nnew;  // new edges (branch \ stem), unsliced
    int r_in, r_out;        // stem ranks (unsliced) before/after
};

struct Scheme {
    std::vector<Cluster> clusters;
    int seed_cluster = -1;
    std::vector<int> stem_order;  // clusters absorbed by the stem, in order
    Bits sliced;
    std::vector<int> sliced_list;  // in slice-bit order
    double log2_tc = 0, stem_tc = 0, branch_tc = 0;
    int cw = 0;
};

// cost helpers
double log2_add(double a, double b);
struct StemCost {
    double tc = 0;      // sum of 2^|E_u| over stem steps (unsliced edges only)
    int max_rank = 0;   // max |E*_u| over stem tensors
};

Scheme plan_scheme(const Network &net, const tn_plan_opts &opts);
Scheme scheme_from_order(const Network &net, const std::vector<std::pair<int, int>> &order,
                         const std::vector<int> &sliced, const tn_plan_opts &opts);
void evaluate_scheme(const Network &net, Scheme &s);
void merge_branches(const Network &net, Scheme &s, int group, int rank_cap);
int merge_branch_runs(const Network &net, Scheme &s, const std::vector<char> &join, int rank_cap);
std::vector<std::pair<int, int>> export_order(const Network &net, const Scheme &s);

// ----------------------------------------------------------------- device plan
constexpr int MAX_PASS_STEPS = 8;
constexpr int MAX_STEP_K = 4;    // k + n <= 4 inside fused passes
constexpr int MAX_TILE_BITS = 12;
constexpr int MAX_BRANCH_SLICED = 24;
constexpr int MAX_FREE = 40;

// Shared-memory tiles are addressed through a bank swizzle: tile position
// bit 4+j also flips offset bit 1 + (j mod 3), i.e. tile_swizzle(p) = p ^
// (s << 1) with s the XOR of the 3-bit fields of p >> 4. Offset bit 0 never
// moves, so entry pairs (2i, 2i+1) stay adjacent and tiles move with 16-byte
// copies; strides of 16 entries and more still land on distinct bank pairs.
// The map is linear over GF(2), so offsets of disjoint bit sets combine with
// XOR.
inline int tile_swizzle(int p) {
    const int x = (p >> 4) & 255;
    return p ^ (((x ^ (x >> 3) ^ (x >> 6)) & 7) << 1);
}

// All offsets are in complex elements; tile offsets are swizzled positions.
// Steps run in place: a step reads the 2^k entries of each rest index at
// lo/hi(rest) ^ koff[kappa] and writes its 2^n results at lo/hi(rest) ^
// noff[nu] in the same buffer. Rest bits keep their tile positions; the nu
// bits take the positions the kappa bits held, then free ones. The write set
// of a rest index holds its read set or lies inside it, and different rest
// indices touch disjoint entries, so no entry is read after another thread
// wrote it within a step.
struct alignas(16) DevStep {
    int k, n, rest;
    int branch;                 // index into DevBranch table (-1: no step)
    int koff[16], noff[16];     // tile offsets of kappa / nu bits
    int lo[64], hi[64];         // rest index bits 0-5 / 6-11 -> tile offset
    int pair;                   // 1: rest bit 0 is tile position 0 (offset 1),
                                // so rest indices 2i, 2i+1 are adjacent entries
    int pad_[3];
};
struct DevBranch {
    int64_t base;           // offset into the branch pool
    int64_t prefix_stride;  // 0 when independent of the prefix
    int k, n;               // matrix rows 2^k (kappa), cols 2^n (nu); nu fastest
    int n_sl;               // sliced edges stored as dims
    int sl_bit[MAX_BRANCH_SLICED];  // slice-id bit of each
    int sl_pos[MAX_BRANCH_SLICED];  // storage bit position of each
};

// 16-byte aligned: kernels copy it to shared memory with 16-byte loads.
struct alignas(16) DevPass {
    int r_in, r_out;
    int t_in, t_out;        // tile bits in / out
    int c_in, c_out;        // contiguous chunk bits in / out
    int n_free;
    int tile_max;           // max tile entries over the pass's states
    int n_steps;
    int in_branch;          // >= 0: input is this branch's storage (seed)
    int64_t in_item_stride, out_item_stride;
    int64_t n_tiles;        // 2^n_free
    int chunk_in_base, chunk_out_base;  // offsets into the chunk table
    int64_t free_in[MAX_FREE], free_out[MAX_FREE];  // strides of free bits
    int st_lo[64], st_hi[64];  // tile-out index bits 0-5 / 6-11 -> tile offset
    DevStep steps[MAX_PASS_STEPS];
};
static_assert(sizeof(DevPass) % 16 == 0, "DevPass must be a multiple of 16 bytes");
static_assert(sizeof(DevStep) % 16 == 0, "DevStep must be a multiple of 16 bytes");
static_assert(offsetof(DevPass, steps) % 16 == 0, "DevPass steps must start 16-byte aligned");

// Host-side description of the executable stem.
struct ExecStep {  // plain mode: permute pass + GEMM
    int permute_pass;   // index into plain passes
    int branch;
    int k, n;
    int64_t M;          // 2^(r_in - k)
    int r_in, r_out;
};

struct FusedItem {  // fused mode: either a pass or a GEMM step
    int kind;           // 0 pass, 1 gemm (permute pass before it is a separate item)
    int pass;           // index into fused passes
    int branch, k, n;
    int64_t M;
    int r_in, r_out;
};

struct StemPlan {
    // layouts: edge at each bit position
    std::vector<std::vector<int>> plain_layouts;  // after each plain step
    std::vector<DevPass> plain_passes;
    std::vector<ExecStep> plain_steps;
    std::vector<DevPass> fused_passes;
    std::vector<FusedItem> fused_items;
    std::vector<int> chunk_table;                 // chunk offsets of all passes
    std::vector<int> final_layout_plain, final_layout_fused;
    int max_rank = 0;
    double bytes_plain = 0, bytes_fused = 0;
    std::vector<int> step_pass;                   // fused pass of each stem step
    std::vector<int> step_gemm;
};

// Branch storage layout chosen by the planner.
struct BranchLayout {
    std::vector<int> bits;  // edge at storage bit j (nu..., kappa..., sliced...)
    int k = 0, n = 0;       // kappa / nu counts (seed: n = rank, k = 0)
    bool prefix_dependent = false;
    std::vector<int> sliced_edges;  // global edge ids at the top positions
};

struct BuiltStem {
    StemPlan sp;
    std::vector<BranchLayout> layouts;  // per cluster
};

struct Plan;  // defined in plan.h

}  // namespace tn
