// Tensor network of a Sycamore-style random circuit (Sec. 2, Sec. 3,
// Supp. A.1): one leaf per |0>, gate and closed-qubit projector; one edge per
// wire segment; open edges on the open qubits' last segments.
#include <cmath>
#include <set>

#include "internal.h"

namespace tn {

// Sec. 2: sqrt(X), sqrt(Y), sqrt(W); sqrt(i) read as e^{i pi/4}, sqrt(-i) as
// e^{-i pi/4}. Row-major [out][in].
void gate_matrix_1q(int id, cd g[4]) {
    const double s = std::sqrt(0.5);
    const cd i(0.0, 1.0);
    if (id == 0) {
        g[0] = s; g[1] = -i * s; g[2] = -i * s; g[3] = s;
    } else if (id == 1) {
        g[0] = s; g[1] = -s; g[2] = s; g[3] = s;
    } else if (id == 2) {
        const double q = M_PI / 4.0;
        g[0] = s;
        g[1] = -std::polar(1.0, q) * s;
        g[2] = std::polar(1.0, -q) * s;
        g[3] = s;
    } else {
        fail(TN_ERR_INVALID_ARG, "single-qubit gate id must be 0, 1 or 2");
    }
}

// Sec. 2: fSim(theta, phi), basis |00>,|01>,|10>,|11> with the first qubit of
// the pair as the high bit. Row-major [out][in].
void fsim_matrix(double theta, double phi, cd f[16]) {
    for (int k = 0; k < 16; ++k) f[k] = 0.0;
    const cd mi(0.0, -1.0);
    f[0] = 1.0;
    f[1 * 4 + 1] = std::cos(theta);
    f[1 * 4 + 2] = mi * std::sin(theta);
    f[2 * 4 + 1] = mi * std::sin(theta);
    f[2 * 4 + 2] = std::cos(theta);
    f[3 * 4 + 3] = std::polar(1.0, -phi);
}

Network build_network(const tn_circuit &c, const int32_t *open_qubits, int n_open,
                      const uint8_t *closed_bits, bool hyper) {
    if (c.n_qubits <= 0 || c.n_qubits > 4096 || c.n_cycles < 0 || c.n_cycles > 4096)
        fail(TN_ERR_INVALID_ARG, "n_qubits / n_cycles out of range");
    if (!c.gates_1q || !c.pair_offsets || (c.pair_offsets[c.n_cycles] > 0 && !c.pairs))
        fail(TN_ERR_INVALID_ARG, "null circuit array");
    if (n_open < 0 || n_open > c.n_qubits || (n_open > 0 && !open_qubits))
        fail(TN_ERR_INVALID_ARG, "bad open-qubit list");
    if (n_open < c.n_qubits && !closed_bits) fail(TN_ERR_INVALID_ARG, "closed_bits is null");
    const int n = c.n_qubits, m = c.n_cycles;
    if (hyper && std::abs(std::cos(c.theta)) > 1e-12)
        fail(TN_ERR_UNSUPPORTED, "a hyperedge network needs fSim(pi/2, phi): a wire swap times a diagonal gate");
    Network net;
    net.hyper = hyper;
    net.n_qubits = n;
    net.n_cycles = m;
    net.theta = c.theta;
    net.phi = c.phi;
    std::set<int> opened;
    for (int i = 0; i < n_open; ++i) {
        int q = open_qubits[i];
        if (q < 0 || q >= n || opened.count(q)) fail(TN_ERR_INVALID_ARG, "bad open qubit");
        opened.insert(q);
        net.open_qubits.push_back(q);
    }
    for (int q = 0; q < n; ++q)
        if (!opened.count(q)) net.closed_qubits.push_back(q);
    for (size_t i = 0; i < net.closed_qubits.size(); ++i) {
        if (closed_bits[i] > 1) fail(TN_ERR_INVALID_ARG, "closed bits must be 0 or 1");
        net.closed_bits.push_back(closed_bits[i]);
    }

    std::vector<int> cur(n);  // current edge id of each qubit's wire
    std::vector<int> seg(n, 0);
    auto new_edge = [&](int q, int s) {
        EdgeInfo e{q, s, {-1, -1}, 0, false};
        net.edges.push_back(e);
        return (int)net.edges.size() - 1;
    };
    auto attach = [&](int e, int leaf) {
        EdgeInfo &E = net.edges[e];
        if (E.n_ends >= 2 && !hyper) fail(TN_ERR_INVALID_ARG, "internal: edge with three ends");
        if (E.n_ends < 2) E.ends[E.n_ends] = leaf;
        ++E.n_ends;  // a hyperedge may join more than two leaves
    };
    auto add_leaf = [&](Leaf L) {
        int id = (int)net.leaves.size();
        for (int e : L.edges) attach(e, id);
        net.leaves.push_back(std::move(L));
        return id;
    };

    for (int q = 0; q < n; ++q) {
        cur[q] = new_edge(q, 0);
        Leaf L{LEAF_ZERO, q, -1, 0, {cur[q]}, {1.0, 0.0}};
        add_leaf(L);
    }
    cd f[16];
    fsim_matrix(c.theta, c.phi, f);
    for (int t = 0; t <= m; ++t) {
        for (int q = 0; q < n; ++q) {
            int id = c.gates_1q[(int64_t)t * n + q];
            cd g[4];
            gate_matrix_1q(id, g);
            int ein = cur[q];
            int eout = new_edge(q, ++seg[q]);
            // bit 0 = input, bit 1 = output: value[in + 2 out] = G[out][in]
            Leaf L{LEAF_1Q, q, -1, id, {ein, eout}, std::vector<cd>(4)};
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) L.vals[a + 2 * b] = g[b * 2 + a];
            add_leaf(L);
            cur[q] = eout;
        }
        if (t == m) break;
        int p0 = c.pair_offsets[t], p1 = c.pair_offsets[t + 1];
        if (p0 < 0 || p1 < p0) fail(TN_ERR_INVALID_ARG, "bad pair offsets");
        std::set<int> used;
        for (int p = p0; p < p1; ++p) {
            int qa = c.pairs[2 * p], qb = c.pairs[2 * p + 1];
            if (qa < 0 || qb < 0 || qa >= n || qb >= n || qa >= qb)
                fail(TN_ERR_INVALID_ARG, "pair must satisfy 0 <= qa < qb < n");
            if (used.count(qa) || used.count(qb))
                fail(TN_ERR_INVALID_ARG, "a qubit appears twice in one two-qubit layer");
            used.insert(qa);
            used.insert(qb);
            int ia = cur[qa], ib = cur[qb];
            if (hyper) {
                // fSim(pi/2, phi) |x_a x_b> = d(x_a, x_b) |x_b x_a>: the rank-2
                // diagonal d on the two wire indices, then the wires exchange
                // them. value[x_a + 2 x_b] = F[(x_b x_a)][(x_a x_b)].
                Leaf L{LEAF_DIAG, qa, qb, 0, {ia, ib}, std::vector<cd>(4)};
                for (int xa = 0; xa < 2; ++xa)
                    for (int xb = 0; xb < 2; ++xb) L.vals[xa + 2 * xb] = f[(xb * 2 + xa) * 4 + (xa * 2 + xb)];
                add_leaf(L);
                cur[qa] = ib;
                cur[qb] = ia;
                continue;
            }
            int oa = new_edge(qa, ++seg[qa]);
            int ob = new_edge(qb, ++seg[qb]);
            // bits (ia, ib, oa, ob): value[ia + 2 ib + 4 oa + 8 ob] = F[(oa ob)][(ia ib)]
            Leaf L{LEAF_2Q, qa, qb, 0, {ia, ib, oa, ob}, std::vector<cd>(16)};
            for (int idx = 0; idx < 16; ++idx) {
                int xa = idx & 1, xb = (idx >> 1) & 1, ya = (idx >> 2) & 1, yb = (idx >> 3) & 1;
                L.vals[idx] = f[(ya * 2 + yb) * 4 + (xa * 2 + xb)];
            }
            add_leaf(L);
            cur[qa] = oa;
            cur[qb] = ob;
        }
    }
    for (size_t i = 0; i < net.closed_qubits.size(); ++i) {
        int q = net.closed_qubits[i];
        int b = net.closed_bits[i];
        Leaf L{LEAF_PROJ, q, -1, (int)i, {cur[q]}, {b == 0 ? 1.0 : 0.0, b == 1 ? 1.0 : 0.0}};
        net.proj_leaf.push_back(add_leaf(L));
    }
    for (int q : net.open_qubits) {
        net.edges[cur[q]].open = true;
        net.open_edges.push_back(cur[q]);
    }
    for (auto &e : net.edges)
        if (!e.open && (hyper ? e.n_ends < 2 : e.n_ends != 2))
            fail(TN_ERR_INVALID_ARG, "internal: dangling edge");
    return net;
}

void set_prefix(Network &net, const uint8_t *closed_bits) {
    if (!net.closed_qubits.empty() && !closed_bits) fail(TN_ERR_INVALID_ARG, "closed_bits is null");
    for (size_t i = 0; i < net.closed_qubits.size(); ++i)
        if (closed_bits[i] > 1) fail(TN_ERR_INVALID_ARG, "closed bits must be 0 or 1");
    for (size_t i = 0; i < net.closed_qubits.size(); ++i) {
        const int b = closed_bits[i];
        net.closed_bits[i] = (uint8_t)b;
        Leaf &L = net.leaves[(size_t)net.proj_leaf[i]];
        L.vals[0] = b == 0 ? 1.0 : 0.0;
        L.vals[1] = b == 1 ? 1.0 : 0.0;
    }
}

}  // namespace tn
