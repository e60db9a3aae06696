/*
 * Oracle: plain, slow, FP64 CPU reference for the stem contraction.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library. It shares no code,
 * header, table or constant with the GPU library and includes none of it.
 *
 * What it computes (paper sections cited per function):
 *   orc_gate_1q / orc_fsim  -- the gate matrices printed in Sec. 2.
 *   orc_statevector         -- Schroedinger evolution of the circuit of Sec. 2
 *                              (optionally with |v><v| inserted on chosen wire
 *                              segments, which is what fixing a sliced edge
 *                              means, Supp. A.1 "Slicing").
 *   orc_contract            -- one pairwise contraction step, Supp. A.1: the
 *                              sum over the edges of E_AB outside E*_AB of
 *                              the product of entries, for every assignment
 *                              of the output edges E*_AB (shared edges that
 *                              stay in E*_AB, hyperedges, are not summed).
 *   orc_feynman             -- the tensor-network value T_H[b] of Supp. A.1 as
 *                              the literal sum of Feynman path values F(a).
 *
 * Conventions: complex numbers are C99 double complex (interleaved re, im).
 * A tensor with edge list e[0..r-1] stores entry (a_e0, ..., a_e(r-1)) at
 * linear index sum_j a_ej * 2^(r-1-j) (first edge = most significant bit).
 * A state vector over n qubits stores basis state x at index
 * sum_q x_q * 2^(n-1-q) (qubit 0 = most significant bit).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* Sec. 2: sqrt(X), sqrt(Y), sqrt(W) with sqrt(i) = e^{i pi/4} and
 * sqrt(-i) = e^{-i pi/4}. Row-major [out][in]. id 0, 1, 2 respectively. */
int orc_gate_1q(int id, cplx *g)
{
    const double s = 1.0 / sqrt(2.0);
    switch (id) {
    case 0: /* sqrt(X) = [[1, -i], [-i, 1]] / sqrt2 */
        g[0] = s; g[1] = -I * s; g[2] = -I * s; g[3] = s;
        return 0;
    case 1: /* sqrt(Y) = [[1, -1], [1, 1]] / sqrt2 */
        g[0] = s; g[1] = -s; g[2] = s; g[3] = s;
        return 0;
    case 2: /* sqrt(W) = [[1, -sqrt(i)], [sqrt(-i), 1]] / sqrt2 */
        g[0] = s;
        g[1] = -cexp(I * M_PI / 4.0) * s;
        g[2] = cexp(-I * M_PI / 4.0) * s;
        g[3] = s;
        return 0;
    default:
        return -1;
    }
}

/* Sec. 2: fSim(theta, phi) in the basis |00>,|01>,|10>,|11> of (qa, qb),
 * qa being the high bit. Row-major [out][in]. */
void orc_fsim(double theta, double phi, cplx *f)
{
    for (int i = 0; i < 16; ++i) f[i] = 0.0;
    f[0 * 4 + 0] = 1.0;
    f[1 * 4 + 1] = cos(theta);
    f[1 * 4 + 2] = -I * sin(theta);
    f[2 * 4 + 1] = -I * sin(theta);
    f[2 * 4 + 2] = cos(theta);
    f[3 * 4 + 3] = cexp(-I * phi);
}

static void apply_1q(cplx *psi, int n, int q, const cplx *g)
{
    const int64_t dim = (int64_t)1 << n;
    const int64_t bit = (int64_t)1 << (n - 1 - q);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < dim; ++i) {
        if (i & bit) continue;
        cplx a0 = psi[i], a1 = psi[i | bit];
        psi[i] = g[0] * a0 + g[1] * a1;
        psi[i | bit] = g[2] * a0 + g[3] * a1;
    }
}

static void apply_2q(cplx *psi, int n, int qa, int qb, const cplx *f)
{
    const int64_t dim = (int64_t)1 << n;
    const int64_t ba = (int64_t)1 << (n - 1 - qa);
    const int64_t bb = (int64_t)1 << (n - 1 - qb);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < dim; ++i) {
        if ((i & ba) || (i & bb)) continue;
        const int64_t idx[4] = {i, i | bb, i | ba, i | ba | bb};
        cplx in[4], out[4];
        for (int r = 0; r < 4; ++r) in[r] = psi[idx[r]];
        for (int r = 0; r < 4; ++r) {
            out[r] = 0.0;
            for (int c = 0; c < 4; ++c) out[r] += f[r * 4 + c] * in[c];
        }
        for (int r = 0; r < 4; ++r) psi[idx[r]] = out[r];
    }
}

/* Keep only the component of qubit q equal to v (the projector |v><v|). */
static void apply_projector(cplx *psi, int n, int q, int v)
{
    const int64_t dim = (int64_t)1 << n;
    const int64_t bit = (int64_t)1 << (n - 1 - q);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < dim; ++i) {
        int x = (i & bit) ? 1 : 0;
        if (x != v) psi[i] = 0.0;
    }
}

static void project_segment(cplx *psi, int n, int q, int seg, const int32_t *pq,
                            const int32_t *ps, const int8_t *pv, int n_proj)
{
    for (int k = 0; k < n_proj; ++k)
        if (pq[k] == q && ps[k] == seg) apply_projector(psi, n, q, pv[k]);
}

/*
 * Sec. 2 circuit, Schroedinger method (Sec. 3): start from |0...0>, apply for
 * each cycle t < m the single-qubit layer g1q[t][*] then the two-qubit layer
 * pairs[pair_off[t] .. pair_off[t+1]), then the final single-qubit layer
 * g1q[m][*]. Wire segment s of qubit q is the wire after the s-th gate acting
 * on q (segment 0 lies between |0> and the first gate). For every listed
 * (proj_q[k], proj_seg[k]) the projector |proj_val[k]><proj_val[k]| is applied
 * on that segment. psi must hold 2^n entries. Returns 0, or -1 on bad input.
 */
int orc_statevector(int n, int m, const int8_t *g1q, const int32_t *pair_off,
                    const int32_t *pairs, double theta, double phi,
                    const int32_t *proj_q, const int32_t *proj_seg,
                    const int8_t *proj_val, int n_proj, cplx *psi)
{
    if (n <= 0 || n > 34 || m < 0) return -1;
    const int64_t dim = (int64_t)1 << n;
    memset(psi, 0, sizeof(cplx) * (size_t)dim);
    psi[0] = 1.0;
    int *count = (int *)calloc((size_t)n, sizeof(int));
    if (!count) return -1;
    cplx f[16];
    orc_fsim(theta, phi, f);
    for (int q = 0; q < n; ++q) project_segment(psi, n, q, 0, proj_q, proj_seg, proj_val, n_proj);
    for (int t = 0; t <= m; ++t) {
        for (int q = 0; q < n; ++q) {
            cplx g[4];
            if (orc_gate_1q(g1q[(int64_t)t * n + q], g) != 0) { free(count); return -1; }
            apply_1q(psi, n, q, g);
            count[q] += 1;
            project_segment(psi, n, q, count[q], proj_q, proj_seg, proj_val, n_proj);
        }
        if (t == m) break;
        for (int p = pair_off[t]; p < pair_off[t + 1]; ++p) {
            int qa = pairs[2 * p], qb = pairs[2 * p + 1];
            if (qa < 0 || qb < 0 || qa >= n || qb >= n || qa == qb) { free(count); return -1; }
            apply_2q(psi, n, qa, qb, f);
            count[qa] += 1;
            count[qb] += 1;
            project_segment(psi, n, qa, count[qa], proj_q, proj_seg, proj_val, n_proj);
            project_segment(psi, n, qb, count[qb], proj_q, proj_seg, proj_val, n_proj);
        }
    }
    free(count);
    return 0;
}

static int find_edge(const int64_t *e, int r, int64_t x)
{
    for (int j = 0; j < r; ++j)
        if (e[j] == x) return j;
    return -1;
}

/*
 * One pairwise contraction step (Supp. A.1, "Contraction trees"): the step
 * enumerates the assignments of E_AB, the edges of A or B, and sums the
 * products of entries of those that agree on E*_AB, the output edges:
 *   C[b] = sum over assignments c of the edges in E_AB but not in E*_AB of
 *          A[(b, c) restricted to A's edges] * B[(b, c) restricted to B's].
 * In a graph an edge of both A and B is summed and every other edge is an
 * output edge; in a hypergraph an edge of both A and B that other tensors
 * (or the open edges) still hold is an output edge, taken at the same value
 * in A and B and not summed. ec must list distinct edges of A or B. Returns
 * 0, or -1 when the edge lists do not fit (a repeated edge, an output edge in
 * neither input, more than 30 summed edges).
 */
int orc_contract(const cplx *A, int ra, const int64_t *ea,
                 const cplx *B, int rb, const int64_t *eb,
                 cplx *C, int rc, const int64_t *ec)
{
    if (ra < 0 || rb < 0 || rc < 0 || ra > 40 || rb > 40 || rc > 40) return -1;
    for (int i = 0; i < ra; ++i)
        if (find_edge(ea, i, ea[i]) >= 0) return -1;
    for (int i = 0; i < rb; ++i)
        if (find_edge(eb, i, eb[i]) >= 0) return -1;
    for (int i = 0; i < rc; ++i)
        if (find_edge(ec, i, ec[i]) >= 0) return -1;
    for (int i = 0; i < rc; ++i)
        if (find_edge(ea, ra, ec[i]) < 0 && find_edge(eb, rb, ec[i]) < 0) return -1;
    /* summed edges: the edges of A or B that are not output edges */
    int64_t summed[80];
    int k = 0;
    for (int i = 0; i < ra; ++i)
        if (find_edge(ec, rc, ea[i]) < 0) summed[k++] = ea[i];
    for (int i = 0; i < rb; ++i)
        if (find_edge(ec, rc, eb[i]) < 0 && find_edge(ea, ra, eb[i]) < 0) summed[k++] = eb[i];
    if (k > 30) return -1;

    /* stride of each output bit inside A and inside B (0 if absent) */
    int64_t outA[64], outB[64];
    for (int i = 0; i < rc; ++i) {
        int ja = find_edge(ea, ra, ec[i]), jb = find_edge(eb, rb, ec[i]);
        outA[i] = ja >= 0 ? ((int64_t)1 << (ra - 1 - ja)) : 0;
        outB[i] = jb >= 0 ? ((int64_t)1 << (rb - 1 - jb)) : 0;
    }
    const int64_t nsum = (int64_t)1 << k;
    int64_t *offA = (int64_t *)malloc(sizeof(int64_t) * (size_t)nsum);
    int64_t *offB = (int64_t *)malloc(sizeof(int64_t) * (size_t)nsum);
    if (!offA || !offB) { free(offA); free(offB); return -1; }
    for (int64_t c = 0; c < nsum; ++c) {
        int64_t oa = 0, ob = 0;
        for (int j = 0; j < k; ++j) {
            if (!((c >> (k - 1 - j)) & 1)) continue;
            int ja = find_edge(ea, ra, summed[j]), jb = find_edge(eb, rb, summed[j]);
            if (ja >= 0) oa += (int64_t)1 << (ra - 1 - ja);
            if (jb >= 0) ob += (int64_t)1 << (rb - 1 - jb);
        }
        offA[c] = oa;
        offB[c] = ob;
    }
    const int64_t nout = (int64_t)1 << rc;
#pragma omp parallel for schedule(static)
    for (int64_t o = 0; o < nout; ++o) {
        int64_t ba = 0, bb = 0;
        for (int i = 0; i < rc; ++i) {
            if ((o >> (rc - 1 - i)) & 1) {
                ba += outA[i];
                bb += outB[i];
            }
        }
        cplx acc = 0.0;
        for (int64_t c = 0; c < nsum; ++c) acc += A[ba + offA[c]] * B[bb + offB[c]];
        C[o] = acc;
    }
    free(offA);
    free(offB);
    return 0;
}

/*
 * Tensor-network value by the Feynman method (Supp. A.1, "Tensor networks"):
 *   T_H[b] = sum over all edge assignments a that agree with b on the open
 *            edges of F(a) = prod_v T_v[a restricted to v's edges].
 * Edges are numbered 0..n_edges-1; edges[off[v] .. off[v]+rank[v]) is the
 * ordered edge list of tensor v, whose entries start at vals + voff[v].
 * open[0..n_open) lists the open edges; out (2^n_open entries) is indexed by
 * the open assignment with open[0] as the most significant bit.
 * Returns 0, or -1 for more than 30 edges or bad edge numbers.
 */
int orc_feynman(int n_tensors, const int32_t *rank, const int32_t *off,
                const int32_t *edges, const int64_t *voff, const cplx *vals,
                int n_edges, const int32_t *open, int n_open, cplx *out)
{
    if (n_edges > 30 || n_edges < 0) return -1;
    for (int v = 0; v < n_tensors; ++v)
        for (int j = 0; j < rank[v]; ++j)
            if (edges[off[v] + j] < 0 || edges[off[v] + j] >= n_edges) return -1;
    for (int i = 0; i < n_open; ++i)
        if (open[i] < 0 || open[i] >= n_edges) return -1;
    const int64_t nb = (int64_t)1 << n_open;
    for (int64_t b = 0; b < nb; ++b) out[b] = 0.0;
    const int64_t npaths = (int64_t)1 << n_edges;
    for (int64_t a = 0; a < npaths; ++a) { /* a: bit e = value of edge e */
        cplx f = 1.0;
        for (int v = 0; v < n_tensors && f != 0.0; ++v) {
            int64_t idx = 0;
            for (int j = 0; j < rank[v]; ++j) idx = 2 * idx + ((a >> edges[off[v] + j]) & 1);
            f *= vals[voff[v] + idx];
        }
        int64_t b = 0;
        for (int i = 0; i < n_open; ++i) b = 2 * b + ((a >> open[i]) & 1);
        out[b] += f;
    }
    return 0;
}
