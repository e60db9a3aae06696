// Turn a scheme (stem order + branches + sliced edges) into what the kernels
// run: bit layouts of every stem tensor and branch, the fused HBM passes, and
// the plain permute + GEMM steps.
//
// A stem tensor of rank r is 2^r complex64 values; its layout lists the edge
// held by each bit of the linear index (bit 0 = contiguous). A fused pass
// reads tiles made of 2^c-entry contiguous chunks, applies several stem steps
// to each tile in shared memory and writes the tile in the next layout, so a
// run of steps costs one read and one write of the stem tensor.
#include <algorithm>
#include <cmath>
#include <map>
#include <set>

#include "internal.h"
#include "plan.h"

namespace tn {

namespace {

struct StepSets {
    std::vector<int> K, N;  // branch kappa / nu edges, ascending
    int r_in, r_out;
};

int pos_of(const std::vector<int> &layout, int e) {
    for (size_t i = 0; i < layout.size(); ++i)
        if (layout[i] == e) return (int)i;
    return -1;
}

// Steps the fused pass kernel applies in shared memory: at least one
// contracted bit and a branch matrix of at most 2^4 entries (kept in
// registers); anything else runs as a GEMM step.
bool fusable_step(int k, int n, int gemm_min) {
    return k >= 1 && k + n <= MAX_STEP_K && k < gemm_min && n < gemm_min;
}

// Index of the first step >= from that contracts e (never: 1 << 30).
int next_use(int e, const std::vector<StepSets> &steps, int from) {
    for (int i = from; i < (int)steps.size(); ++i)
        for (int x : steps[(size_t)i].K)
            if (x == e) return i;
    return 1 << 30;
}

// Order edges by the step that next contracts them, soonest first (or latest
// first), ties by edge id.
std::vector<int> sort_by_next_use(std::vector<int> edges, const std::vector<StepSets> &steps,
                                  int from, bool latest_first = false) {
    std::map<int, int> use;
    for (int e : edges) use[e] = next_use(e, steps, from);
    std::sort(edges.begin(), edges.end(), [&](int a, int b) {
        if (use[a] != use[b]) return latest_first ? use[a] > use[b] : use[a] < use[b];
        return a < b;
    });
    return edges;
}

// Bank pair (low four bits of the swizzled offset) that a one-bit stride at
// tile position q lands on.
int bank_vec(int q) { return tile_swizzle(1 << q) & 15; }

// Steps whose rest indices a thread handles in adjacent pairs (16-byte
// shared-memory accesses) when tile position 0 is a rest bit; the others keep
// a register footprint the pass kernel can afford only one rest index at a
// time.
bool pair_shape(int k, int n) { return (k <= 2 && k + n <= 4) || (k == 3 && n == 0); }

// GF(2) span helper over 4-bit bank vectors: adds v when independent.
bool take_independent(uint32_t &span, int v) {
    if (v == 0 || ((span >> v) & 1u)) return false;
    uint32_t add = 0;
    for (int x = 0; x < 16; ++x)
        if ((span >> x) & 1u) add |= 1u << (x ^ v);
    span |= add;
    return true;
}

// Order a step's rest edges into rest-index bits. Plain steps: rest-index
// bits 0-3 vary across the 16 lanes of a half-warp and get edges whose bank
// vectors are independent over GF(2) where the tile allows, so every
// half-warp's 8-byte accesses fall on 16 distinct bank pairs. Paired steps:
// bit 0 is the position-0 edge (the pair inside a thread), and bits 1-3 vary
// across the 8 lanes of a quarter-warp, whose 16-byte accesses are
// conflict-free when those edges move distinct combinations of offset bits
// 1-3. The others follow by position.
std::vector<int> order_rest(std::vector<int> rest, const std::map<int, int> &pos, bool pair) {
    std::sort(rest.begin(), rest.end(), [&](int a, int b) { return pos.at(a) < pos.at(b); });
    std::vector<int> lanes, others;
    uint32_t span = 1;  // bit v set: vector v is in the span of the chosen vectors
    size_t start = 0;
    if (pair) {
        lanes.push_back(rest[0]);  // position 0
        start = 1;
        span |= 1u << 1;           // offset bit 0 is inside the pair
    }
    const size_t want = 4;
    for (size_t i = start; i < rest.size(); ++i) {
        const int e = rest[i];
        const int v = bank_vec(pos.at(e));
        if (lanes.size() < want && take_independent(span, v))
            lanes.push_back(e);
        else
            others.push_back(e);
    }
    lanes.insert(lanes.end(), others.begin(), others.end());
    return lanes;
}

// Tables of one in-place step: kappa offsets at the positions before the
// step, nu offsets at the positions after it, rest offsets (unchanged).
void fill_step(DevStep &st, const std::vector<int> &rest, const std::vector<int> &kpos,
               const std::vector<int> &npos, const std::map<int, int> &pos, bool pair) {
    st.pair = pair ? 1 : 0;
    st.k = (int)kpos.size();
    st.n = (int)npos.size();
    st.rest = (int)rest.size();
    if (st.rest > 12) fail(TN_ERR_UNSUPPORTED, "internal: tile rest exceeds 12 bits");
    for (int kk = 0; kk < 16; ++kk) {
        int o = 0;
        for (int b = 0; b < st.k; ++b)
            if ((kk >> b) & 1) o ^= tile_swizzle(1 << kpos[(size_t)b]);
        st.koff[kk] = (kk < (1 << st.k)) ? o : 0;
    }
    for (int nn = 0; nn < 16; ++nn) {
        int o = 0;
        for (int b = 0; b < st.n; ++b)
            if ((nn >> b) & 1) o ^= tile_swizzle(1 << npos[(size_t)b]);
        st.noff[nn] = (nn < (1 << st.n)) ? o : 0;
    }
    for (int v = 0; v < 64; ++v) {
        int a = 0, b = 0;
        for (int j = 0; j < 6; ++j) {
            if (!((v >> j) & 1)) continue;
            if (j < st.rest) a ^= tile_swizzle(1 << pos.at(rest[(size_t)j]));
            if (j + 6 < st.rest) b ^= tile_swizzle(1 << pos.at(rest[(size_t)(j + 6)]));
        }
        st.lo[v] = a;
        st.hi[v] = b;
    }
}

// Build a pass from in-layout to out-layout applying `group` steps (indices
// into steps, with branch ids br). tile_in_edges must contain the low c_in
// input edges and every input edge the group contracts.
//
// The tile is loaded with input tile edge i (by ascending input position) at
// tile position i. Each step runs in place: rest edges keep their positions,
// the nu edges take the kappa edges' positions, then the lowest free ones.
// The store reads the final positions through the st_lo / st_hi tables, so
// the output layout costs nothing extra.
DevPass build_pass(const std::vector<int> &Lin, const std::vector<int> &Lout, int c_in, int c_out,
                   const std::set<int> &tile_in_edges, const std::vector<int> &group,
                   const std::vector<StepSets> &steps, const std::vector<int> &branch_of_step,
                   std::vector<int> &chunk_table) {
    DevPass P{};
    P.r_in = (int)Lin.size();
    P.r_out = (int)Lout.size();
    P.c_in = c_in;
    P.c_out = c_out;
    P.in_branch = -1;
    std::vector<int> lam_in;
    for (int e : Lin)
        if (tile_in_edges.count(e)) lam_in.push_back(e);
    P.t_in = (int)lam_in.size();
    std::map<int, int> pos;
    for (size_t i = 0; i < lam_in.size(); ++i) pos[lam_in[i]] = (int)i;
    int max_t = P.t_in;
    auto used = [&]() {
        uint32_t m = 0;
        for (auto &kv : pos) m |= 1u << kv.second;
        return m;
    };
    if (group.empty()) {
        P.n_steps = 1;
        std::vector<int> rest = order_rest(lam_in, pos, false);
        fill_step(P.steps[0], rest, {}, {}, pos, false);
        P.steps[0].branch = -1;
    } else {
        P.n_steps = (int)group.size();
        for (size_t t = 0; t < group.size(); ++t) {
            const StepSets &S = steps[(size_t)group[t]];
            std::vector<int> kpos;
            for (int e : S.K) {
                auto it = pos.find(e);
                if (it == pos.end()) fail(TN_ERR_UNSUPPORTED, "internal: contracted edge not in tile");
                kpos.push_back(it->second);
            }
            std::vector<int> rest;
            for (auto &kv : pos)
                if (std::find(S.K.begin(), S.K.end(), kv.first) == S.K.end()) rest.push_back(kv.first);
            bool pair = pair_shape((int)S.K.size(), (int)S.N.size());
            if (pair) {
                pair = false;
                for (int e : rest)
                    if (pos.at(e) == 0) pair = true;
            }
            rest = order_rest(rest, pos, pair);
            for (int e : S.K) pos.erase(e);
            std::vector<int> free_pos = kpos;
            const uint32_t occ = used();
            for (int q = 0; q < 32 && free_pos.size() < S.N.size(); ++q)
                if (!((occ >> q) & 1u) && std::find(kpos.begin(), kpos.end(), q) == kpos.end())
                    free_pos.push_back(q);
            std::vector<int> npos(free_pos.begin(), free_pos.begin() + (long)S.N.size());
            for (size_t b = 0; b < S.N.size(); ++b) pos[S.N[b]] = npos[b];
            fill_step(P.steps[t], rest, kpos, npos, pos, pair);
            P.steps[t].branch = branch_of_step[(size_t)group[t]];
            max_t = std::max(max_t, (int)pos.size());
        }
    }
    // tile-local output layout: tile-out edges by ascending output position
    std::vector<int> lam_out;
    for (int e : Lout)
        if (pos.count(e)) lam_out.push_back(e);
    if (lam_out.size() != pos.size()) fail(TN_ERR_UNSUPPORTED, "internal: tile-out mismatch");
    P.t_out = (int)lam_out.size();
    P.tile_max = 1 << max_t;
    for (int v = 0; v < 64; ++v) {
        int a = 0, b = 0;
        for (int j = 0; j < 6; ++j) {
            if (!((v >> j) & 1)) continue;
            if (j < P.t_out) a ^= tile_swizzle(1 << pos.at(lam_out[(size_t)j]));
            if (j + 6 < P.t_out) b ^= tile_swizzle(1 << pos.at(lam_out[(size_t)(j + 6)]));
        }
        P.st_lo[v] = a;
        P.st_hi[v] = b;
    }
    std::set<int> tile_out_set(lam_out.begin(), lam_out.end());
    // low c_in input positions must be tile edges; low c_out output positions too
    for (int p = 0; p < c_in; ++p)
        if (!tile_in_edges.count(Lin[(size_t)p])) fail(TN_ERR_UNSUPPORTED, "internal: c_in");
    for (int p = 0; p < c_out; ++p)
        if (!tile_out_set.count(Lout[(size_t)p])) fail(TN_ERR_UNSUPPORTED, "internal: c_out");
    // free edges
    P.n_free = 0;
    for (int e : Lin) {
        if (tile_in_edges.count(e)) continue;
        int po = pos_of(Lout, e);
        if (po < 0) fail(TN_ERR_UNSUPPORTED, "internal: free edge missing from output");
        if (P.n_free >= MAX_FREE) fail(TN_ERR_UNSUPPORTED, "too many free bits");
        P.free_in[P.n_free] = 1ll << pos_of(Lin, e);
        P.free_out[P.n_free] = 1ll << po;
        P.n_free++;
    }
    if (P.r_out - P.t_out != P.n_free) fail(TN_ERR_UNSUPPORTED, "internal: free count");
    P.n_tiles = 1ll << P.n_free;
    // chunk tables
    P.chunk_in_base = (int)chunk_table.size();
    for (int j = 0; j < (1 << (P.t_in - c_in)); ++j) {
        int o = 0;
        for (int b = 0; b < P.t_in - c_in; ++b)
            if ((j >> b) & 1) o += 1 << pos_of(Lin, lam_in[(size_t)(c_in + b)]);
        chunk_table.push_back(o);
    }
    P.chunk_out_base = (int)chunk_table.size();
    for (int j = 0; j < (1 << (P.t_out - c_out)); ++j) {
        int o = 0;
        for (int b = 0; b < P.t_out - c_out; ++b)
            if ((j >> b) & 1) o += 1 << pos_of(Lout, lam_out[(size_t)(c_out + b)]);
        chunk_table.push_back(o);
    }
    P.in_item_stride = 1ll << P.r_in;
    P.out_item_stride = 1ll << P.r_out;
    return P;
}

// Check that a pass's descriptors address exactly the tensors they claim:
// the input (output) bit positions used by chunks, chunk tables and free
// bits partition [0, r_in) ([0, r_out)), every step's rest and kappa offsets
// partition the tile positions it reads, its nu offsets avoid the rest
// positions (so in-place writes never touch another rest index's entries),
// and the store tables cover the final positions. Any violation would index
// outside a buffer or race, so it is rejected here on the host.
void validate_pass(const DevPass &P, const std::vector<int> &chunks) {
    auto bad = [](const char *what) { fail(TN_ERR_UNSUPPORTED, std::string("internal: pass ") + what); };
    if (P.r_in < 0 || P.r_in > 31 || P.r_out < 0 || P.r_out > 31) bad("rank");
    if (P.c_in > P.t_in || P.c_out > P.t_out) bad("chunk bits");
    if (P.n_steps < 1 || P.n_steps > MAX_PASS_STEPS) bad("step count");
    if (P.n_free > 32) bad("more than 32 free bits");
    auto check_side = [&](int r, int t, int c, int base, const int64_t *free) {
        uint64_t mask = (c > 0) ? ((1ull << c) - 1) : 0;
        int bits = c;
        for (int b = 0; b < t - c; ++b) {
            int v = chunks[(size_t)base + (1u << b)];
            if (v <= 0 || (v & (v - 1))) bad("chunk table entry");
            if (mask & (uint64_t)v) bad("chunk overlap");
            mask |= (uint64_t)v;
            ++bits;
        }
        for (int f = 0; f < P.n_free; ++f) {
            uint64_t v = (uint64_t)free[f];
            if (!v || (v & (v - 1))) bad("free stride");
            if (mask & v) bad("free overlap");
            mask |= v;
            ++bits;
        }
        if (bits != r || mask != ((r == 64) ? ~0ull : ((1ull << r) - 1))) bad("index partition");
        // chunk table entries are sums of the single-bit entries
        for (int j = 0; j < (1 << (t - c)); ++j) {
            int o = 0;
            for (int b = 0; b < t - c; ++b)
                if ((j >> b) & 1) o += chunks[(size_t)base + (1u << b)];
            if (chunks[(size_t)base + (size_t)j] != o) bad("chunk table sum");
        }
    };
    check_side(P.r_in, P.t_in, P.c_in, P.chunk_in_base, P.free_in);
    check_side(P.r_out, P.t_out, P.c_out, P.chunk_out_base, P.free_out);
    // in-place steps: track which tile positions hold entries
    if (P.tile_max < 1 || (P.tile_max & (P.tile_max - 1)) || P.tile_max > (1 << MAX_TILE_BITS))
        bad("tile size");
    if (P.t_in > MAX_TILE_BITS || P.t_out > MAX_TILE_BITS) bad("tile bits");
    const uint32_t tile_mask = (uint32_t)P.tile_max - 1;
    // undo the swizzle: tile_swizzle maps position bit q to a value whose top
    // bit is q, and it is invertible on the tile
    auto unswz = [&](int v) {
        for (int q = 0; q < MAX_TILE_BITS; ++q)
            if (tile_swizzle(1 << q) == v) return q;
        return -1;
    };
    // single-bit images -> positions (distinct, inside the tile); every table
    // entry must be the XOR of its single-bit entries
    auto bits_of = [&](const int *tab, int nbits, int nentries, const char *what) {
        uint32_t m = 0;
        for (int b = 0; b < nbits; ++b) {
            const int q = unswz(tab[1 << b]);
            if (q < 0 || (m >> q) & 1u || !((tile_mask >> q) & 1u)) bad(what);
            m |= 1u << q;
        }
        for (int v = 0; v < nentries; ++v) {
            int o = 0;
            for (int b = 0; b < nbits; ++b)
                if ((v >> b) & 1) o ^= tab[1 << b];
            if (tab[v] != o || (uint32_t)tab[v] > tile_mask) bad(what);
        }
        return m;
    };
    uint32_t occ = (P.t_in >= 32) ? 0u : ((1u << P.t_in) - 1);
    if (occ & ~tile_mask) bad("input tile size");
    for (int i = 0; i < P.n_steps; ++i) {
        const DevStep &S = P.steps[i];
        if (S.k < 0 || S.n < 0 || S.k + S.n > MAX_STEP_K) bad("step k/n");
        if (S.branch >= 0 && S.k < 1) bad("fused step without contracted bits");
        if (S.branch < 0 && (S.k || S.n)) bad("copy step with k/n");
        if (S.rest != __builtin_popcount(occ) - S.k || S.rest > 12) bad("rest bits");
        const int lo_bits = std::min(S.rest, 6), hi_bits = std::max(S.rest - 6, 0);
        const uint32_t R = bits_of(S.lo, lo_bits, 1 << lo_bits, "rest offset") |
                           bits_of(S.hi, hi_bits, 1 << hi_bits, "rest offset");
        if (__builtin_popcount(R) != S.rest) bad("rest offset overlap");
        const uint32_t Kp = bits_of(S.koff, S.k, 1 << S.k, "kappa offset");
        const uint32_t Np = bits_of(S.noff, S.n, 1 << S.n, "nu offset");
        if ((R & Kp) || (R | Kp) != occ) bad("step reads");
        if (S.pair && (S.rest < 1 || S.lo[1] != 1 || !pair_shape(S.k, S.n))) bad("paired step");
        if (S.k == S.n)  // the kernel writes k == n results at the kappa offsets
            for (int v = 0; v < (1 << S.k); ++v)
                if (S.noff[v] != S.koff[v]) bad("k == n step not in place");
        if (R & Np) bad("step writes");
        occ = R | Np;
    }
    if (__builtin_popcount(occ) != P.t_out) bad("final tile bits");
    {
        const int lo_bits = std::min(P.t_out, 6), hi_bits = std::max(P.t_out - 6, 0);
        const uint32_t O = bits_of(P.st_lo, lo_bits, 1 << lo_bits, "store offset") |
                           bits_of(P.st_hi, hi_bits, 1 << hi_bits, "store offset");
        if (O != occ) bad("store positions");
    }
    if (P.n_tiles != (1ll << P.n_free)) bad("tile count");
}

// Tile of a pure permutation: the low c input bits and the low c output bits
// (both contiguous in their tensors), widened with further input bits up to
// 2^t_max entries so each block iteration moves a full tile.
std::set<int> permute_tile(const std::vector<int> &lay, const std::vector<int> &perm_out, int c,
                           int t_max) {
    std::set<int> tile;
    for (int p = 0; p < c; ++p) {
        tile.insert(lay[(size_t)p]);
        tile.insert(perm_out[(size_t)p]);
    }
    for (size_t p = 0; p < lay.size() && (int)tile.size() < t_max; ++p) tile.insert(lay[p]);
    return tile;
}

}  // namespace

DevPass make_permute_pass(int rank, const std::vector<int> &perm, std::vector<int> &chunks) {
    // input bit j holds "edge" j; output bit perm[j] receives it
    std::vector<int> Lin((size_t)rank), Lout((size_t)rank);
    for (int j = 0; j < rank; ++j) {
        Lin[(size_t)j] = j;
        Lout[(size_t)perm[(size_t)j]] = j;
    }
    const int c = std::min(4, rank);
    std::set<int> tile = permute_tile(Lin, Lout, c, 11);
    DevPass P = build_pass(Lin, Lout, c, c, tile, {}, {}, {}, chunks);
    validate_pass(P, chunks);
    return P;
}

BuiltStem build_stem_plan(const Network &net, const Scheme &s, const tn_plan_opts &o) {
    BuiltStem R;
    const int T_MAX = (o.tile_bits > 0) ? std::min(o.tile_bits, MAX_TILE_BITS) : 12;
    const int C_BITS = 4;
    const int max_steps = (o.max_pass_steps > 0) ? std::min(o.max_pass_steps, MAX_PASS_STEPS) : 8;
    const int gemm_min = (o.gemm_min_kn > 0) ? o.gemm_min_kn : 5;
    const Bits &sl = s.sliced;
    std::vector<Bits> B;
    for (auto &c : s.clusters) B.push_back(c.out.andnot(sl));
    const int L = (int)s.stem_order.size();

    // step sets
    std::vector<StepSets> steps((size_t)L);
    Bits S = B[(size_t)s.seed_cluster];
    int maxr = S.count();
    for (int i = 0; i < L; ++i) {
        const Bits &b = B[(size_t)s.stem_order[(size_t)i]];
        steps[(size_t)i].K = (S & b).list();
        steps[(size_t)i].N = b.andnot(S).list();
        steps[(size_t)i].r_in = S.count();
        S ^= b;
        steps[(size_t)i].r_out = S.count();
        maxr = std::max(maxr, S.count());
    }
    std::vector<int> final_edges = S.list();
    {
        std::vector<int> oe(net.open_edges.begin(), net.open_edges.end());
        std::sort(oe.begin(), oe.end());
        if (final_edges != oe) fail(TN_ERR_INVALID_ARG, "scheme does not end on the open edges");
    }
    if (maxr > 31) fail(TN_ERR_UNSUPPORTED, "stem tensors above 2^31 entries are not supported");
    R.sp.max_rank = maxr;

    // branch layouts
    R.layouts.resize(s.clusters.size());
    std::vector<int> branch_of_step((size_t)L);
    for (int i = 0; i < L; ++i) {
        int c = s.stem_order[(size_t)i];
        BranchLayout &bl = R.layouts[(size_t)c];
        bl.n = (int)steps[(size_t)i].N.size();
        bl.k = (int)steps[(size_t)i].K.size();
        bl.bits = steps[(size_t)i].N;
        bl.bits.insert(bl.bits.end(), steps[(size_t)i].K.begin(), steps[(size_t)i].K.end());
        branch_of_step[(size_t)i] = c;
    }
    std::vector<int> L0;
    {
        std::vector<int> e0 = B[(size_t)s.seed_cluster].list();
        L0 = sort_by_next_use(e0, steps, 0);
        BranchLayout &bl = R.layouts[(size_t)s.seed_cluster];
        bl.bits = L0;
        bl.n = (int)L0.size();
        bl.k = 0;
    }
    for (size_t c = 0; c < s.clusters.size(); ++c) {
        BranchLayout &bl = R.layouts[c];
        // every sliced edge touching the cluster, including edges between two
        // of its own leaves: those are carried through the branch contraction
        // as batch dimensions (never summed) and fixed by the slice offset
        Bits touch(net.n_edges());
        for (int leaf : s.clusters[c].leaves)
            for (int e : net.leaves[(size_t)leaf].edges) touch.set(e);
        for (int e : (touch & sl).list()) bl.sliced_edges.push_back(e);
        std::sort(bl.sliced_edges.begin(), bl.sliced_edges.end(), [&](int a, int b) {
            return std::find(s.sliced_list.begin(), s.sliced_list.end(), a) <
                   std::find(s.sliced_list.begin(), s.sliced_list.end(), b);
        });
        for (int e : bl.sliced_edges) bl.bits.push_back(e);
        for (int leaf : s.clusters[c].leaves)
            if (net.leaves[(size_t)leaf].kind == LEAF_PROJ) bl.prefix_dependent = true;
        if ((int)bl.sliced_edges.size() > MAX_BRANCH_SLICED)
            fail(TN_ERR_UNSUPPORTED, "a branch carries too many sliced edges");
    }

    // ---------------- plain mode: per step a permute to [K | rest] then a GEMM
    {
        std::vector<int> lay = L0;
        for (int i = 0; i < L; ++i) {
            const StepSets &st = steps[(size_t)i];
            std::vector<int> perm_out = st.K;  // kappa order
            for (int e : lay)
                if (std::find(st.K.begin(), st.K.end(), e) == st.K.end()) perm_out.push_back(e);
            int r = (int)lay.size();
            int c = std::min(C_BITS, r);
            std::set<int> tile = permute_tile(lay, perm_out, c, std::min(11, T_MAX));
            DevPass P = build_pass(lay, perm_out, c, c, tile, {}, steps, branch_of_step,
                                   R.sp.chunk_table);
            if (i == 0) P.in_branch = s.seed_cluster;
            R.sp.plain_passes.push_back(P);
            ExecStep es{};
            es.permute_pass = (int)R.sp.plain_passes.size() - 1;
            es.branch = branch_of_step[(size_t)i];
            es.k = (int)st.K.size();
            es.n = (int)st.N.size();
            es.M = 1ll << (r - es.k);
            es.r_in = st.r_in;
            es.r_out = st.r_out;
            R.sp.plain_steps.push_back(es);
            R.sp.bytes_plain += 8.0 * (2.0 * std::exp2(r) + std::exp2(r) + std::exp2(st.r_out));
            // GEMM output layout: [N (nu order) | rest (m order)]
            std::vector<int> nl = st.N;
            for (size_t p = st.K.size(); p < perm_out.size(); ++p) nl.push_back(perm_out[p]);
            lay = nl;
        }
        if (L == 0) {
            // no stem step: a single identity pass from the seed
            int r = (int)lay.size();
            int c = std::min(C_BITS, r);
            std::set<int> tile(lay.begin(), lay.begin() + c);
            DevPass P = build_pass(lay, lay, c, c, tile, {}, steps, branch_of_step, R.sp.chunk_table);
            P.in_branch = s.seed_cluster;
            R.sp.plain_passes.push_back(P);
        }
        R.sp.final_layout_plain = lay;
    }

    // ---------------- fused mode
    {
        std::vector<int> lay = L0;
        int i = 0;
        bool first = true;
        R.sp.step_pass.assign((size_t)L, -1);
        R.sp.step_gemm.assign((size_t)L, 0);
        while (i < L || (L == 0 && first)) {
            const int r = (int)lay.size();
            const int c_in = std::min(C_BITS, r);
            if (L > 0) {
                const StepSets &st = steps[(size_t)i];
                int k = (int)st.K.size(), n = (int)st.N.size();
                if (!fusable_step(k, n, gemm_min)) {
                    // GEMM step: permute to [K | rest], then GEMM -> [N | rest]
                    std::vector<int> perm_out = st.K;
                    for (int e : lay)
                        if (std::find(st.K.begin(), st.K.end(), e) == st.K.end())
                            perm_out.push_back(e);
                    std::set<int> tile = permute_tile(lay, perm_out, c_in, std::min(11, T_MAX));
                    DevPass P = build_pass(lay, perm_out, c_in, c_in, tile, {}, steps,
                                           branch_of_step, R.sp.chunk_table);
                    if (first) P.in_branch = s.seed_cluster;
                    first = false;
                    R.sp.fused_passes.push_back(P);
                    FusedItem fp{0, (int)R.sp.fused_passes.size() - 1, -1, 0, 0, 0, r, r};
                    R.sp.fused_items.push_back(fp);
                    FusedItem g{1, -1, branch_of_step[(size_t)i], k, n, 1ll << (r - k), st.r_in,
                                st.r_out};
                    R.sp.fused_items.push_back(g);
                    R.sp.bytes_fused += 8.0 * (2.0 * std::exp2(r) + std::exp2(r) + std::exp2(st.r_out));
                    R.sp.step_gemm[(size_t)i] = 1;
                    std::vector<int> nl = st.N;
                    for (size_t p = st.K.size(); p < perm_out.size(); ++p) nl.push_back(perm_out[p]);
                    lay = nl;
                    ++i;
                    continue;
                }
            }
            // grow a group of fusable steps
            std::set<int> in_tile(lay.begin(), lay.begin() + c_in);
            std::vector<int> group;
            {
                // simulate tile states
                std::set<int> in_set(lay.begin(), lay.end());
                int j = i;
                while (j < L && (int)group.size() < max_steps) {
                    const StepSets &st = steps[(size_t)j];
                    int k = (int)st.K.size(), n = (int)st.N.size();
                    if (!fusable_step(k, n, gemm_min)) break;
                    std::set<int> trial = in_tile;
                    // edges needed from the input: K_j edges that are input edges
                    for (int e : st.K)
                        if (in_set.count(e)) trial.insert(e);
                    // check tile sizes through the group + this step
                    std::vector<int> g2 = group;
                    g2.push_back(j);
                    std::set<int> cur = trial;
                    int mx = (int)cur.size();
                    bool ok = true;
                    for (int s2 : g2) {
                        for (int e : steps[(size_t)s2].K)
                            if (!cur.count(e)) ok = false;
                        for (int e : steps[(size_t)s2].K) cur.erase(e);
                        for (int e : steps[(size_t)s2].N) cur.insert(e);
                        mx = std::max(mx, (int)cur.size());
                    }
                    if (!ok || mx > T_MAX) break;
                    // rest bits of each step must be <= 12
                    in_tile = trial;
                    group.push_back(j);
                    ++j;
                }
            }
            if (group.empty() && L > 0) {
                // the single step does not fit the tile: fall back to a GEMM step
                const StepSets &st = steps[(size_t)i];
                int k = (int)st.K.size(), n = (int)st.N.size();
                std::vector<int> perm_out = st.K;
                for (int e : lay)
                    if (std::find(st.K.begin(), st.K.end(), e) == st.K.end()) perm_out.push_back(e);
                std::set<int> tile = permute_tile(lay, perm_out, c_in, std::min(11, T_MAX));
                DevPass P = build_pass(lay, perm_out, c_in, c_in, tile, {}, steps, branch_of_step,
                                       R.sp.chunk_table);
                if (first) P.in_branch = s.seed_cluster;
                first = false;
                R.sp.fused_passes.push_back(P);
                R.sp.fused_items.push_back({0, (int)R.sp.fused_passes.size() - 1, -1, 0, 0, 0, r, r});
                R.sp.fused_items.push_back(
                    {1, -1, branch_of_step[(size_t)i], k, n, 1ll << (r - k), st.r_in, st.r_out});
                R.sp.bytes_fused += 8.0 * (2.0 * std::exp2(r) + std::exp2(r) + std::exp2(st.r_out));
                R.sp.step_gemm[(size_t)i] = 1;
                std::vector<int> nl = st.N;
                for (size_t p = st.K.size(); p < perm_out.size(); ++p) nl.push_back(perm_out[p]);
                lay = nl;
                ++i;
                continue;
            }
            // output edges after the group
            std::set<int> cur = in_tile;
            std::set<int> out_all(lay.begin(), lay.end());
            for (int s2 : group) {
                for (int e : steps[(size_t)s2].K) {
                    cur.erase(e);
                    out_all.erase(e);
                }
                for (int e : steps[(size_t)s2].N) {
                    cur.insert(e);
                    out_all.insert(e);
                }
            }
            int next = group.empty() ? i : group.back() + 1;
            std::vector<int> tile_out(cur.begin(), cur.end());
            // carriers: the contiguous low output bits are the tile-out bits used
            // last, so the next pass can keep them at its low tile positions
            tile_out = sort_by_next_use(tile_out, steps, next, true);
            int c_out = std::min(C_BITS, (int)tile_out.size());
            std::vector<int> low(tile_out.begin(), tile_out.begin() + c_out);
            std::vector<int> others;
            for (int e : out_all)
                if (std::find(low.begin(), low.end(), e) == low.end()) others.push_back(e);
            others = sort_by_next_use(others, steps, next);
            std::vector<int> Lout = low;
            Lout.insert(Lout.end(), others.begin(), others.end());
            DevPass P = build_pass(lay, Lout, c_in, c_out, in_tile, group, steps, branch_of_step,
                                   R.sp.chunk_table);
            if (first) P.in_branch = s.seed_cluster;
            first = false;
            R.sp.fused_passes.push_back(P);
            int pidx = (int)R.sp.fused_passes.size() - 1;
            R.sp.fused_items.push_back({0, pidx, -1, 0, 0, 0, r, (int)Lout.size()});
            R.sp.bytes_fused += 8.0 * (std::exp2(r) + std::exp2((double)Lout.size()));
            for (int s2 : group) R.sp.step_pass[(size_t)s2] = pidx;
            lay = Lout;
            i = next;
            if (L == 0) break;
        }
        R.sp.final_layout_fused = lay;
    }
    for (auto &P : R.sp.plain_passes) validate_pass(P, R.sp.chunk_table);
    for (auto &P : R.sp.fused_passes) validate_pass(P, R.sp.chunk_table);
    return R;
}

}  // namespace tn
