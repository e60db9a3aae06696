"""GPU parity: the CUDA stem path (through the C interface) against the FP64
oracle, element by element, on seeded inputs.

Tolerance: relative L2 error <= 1e-5 for the FP32 path (the stated bound for
the FP32-accurate path). Data movement (permutation) must be bit-exact.
"""

import json
import math
import os

import numpy as np
import pytest

import oracle
import paper_2005_06787_gb300 as P
from synthetic.circuits import (CONFIGS, Circuit, config_circuit, grid_layout, random_bits,
                                random_circuit, random_complex, random_uniform)

pytestmark = pytest.mark.gpu
TOL = 1e-5
GOLD = os.path.join(os.path.dirname(__file__), "golden")

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    P.build()
    P.load()
    torch.cuda.set_device(0)


@pytest.fixture(autouse=True)
def _device_waits_completed():
    # every bounded device-side wait of the test (tensor-core GEMM) must have
    # completed
    yield
    P.tn_device_status()


def rel_l2(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run(plan, s0, s1, mode="fused", prec="fp32", device=True, accumulate=False, out=None):
    info = P.tn_plan_info(plan)
    n = max(info["n_prefixes"], 1) << info["n_open"]
    if out is None:
        out = torch.zeros(2 * n, dtype=torch.float64, device="cuda" if device else "cpu")
    P.tn_contract_stem(plan, s0, s1, out, prec=prec, mode=mode, accumulate=accumulate)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.complex128).reshape(max(info["n_prefixes"], 1), -1)


# ------------------------------------------------------------------ kernels

@pytest.mark.parametrize("rank,seed,offset", [(1, 1, 0), (4, 6, 0), (5, 2, 0), (11, 3, 0), (12, 7, 0),
                                              (17, 4, 0), (20, 5, 0), (24, 8, 0), (13, 9, 1)])
def test_permute_bit_exact(rank, seed, offset):
    # rank >= 4 on 16-byte aligned tensors runs tiled through shared memory;
    # an 8-byte offset (offset = 1 entry) takes the element-wise kernel
    rng = np.random.default_rng(seed)
    perm = rng.permutation(rank).astype(np.int32)
    x = random_complex((1 << rank,), seed, np.complex64)
    buf_in = torch.zeros(2 * ((1 << rank) + offset), dtype=torch.float32, device="cuda")
    buf_out = torch.zeros_like(buf_in)
    xin = buf_in[2 * offset:]
    xin.copy_(torch.from_numpy(x.view(np.float32).copy()))
    xout = buf_out[2 * offset:]
    P.tn_permute(xin, xout, rank, perm)
    torch.cuda.synchronize()
    got = xout.cpu().numpy().view(np.complex64)
    # input bit j -> output bit perm[j]; numpy axes are MSB first
    t = x.reshape((2,) * rank)
    axes_in_bit = list(range(rank))  # bit j <-> axis rank-1-j
    out_axes = [0] * rank
    for j in axes_in_bit:
        out_axes[rank - 1 - perm[j]] = rank - 1 - j
    ref = np.transpose(t, out_axes).reshape(-1)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("M,K,N,batch", [(1000, 4, 4, 1), (4096, 16, 16, 2), (777, 3, 5, 3),
                                         (65, 64, 300, 1), (1, 1, 1, 1), (5000, 2, 1, 1)])
def test_cgemm_simt_matches_fp64(M, K, N, batch):
    A = random_complex((batch, M, K), 11, np.complex64)
    B = random_complex((batch, K, N), 12, np.complex64)
    dA = torch.from_numpy(A.view(np.float32).copy()).cuda()
    dB = torch.from_numpy(B.view(np.float32).copy()).cuda()
    dC = torch.zeros(batch * M * N * 2, dtype=torch.float32, device="cuda")
    P.tn_cgemm(dA, dB, dC, M, K, N, batch, M * K, K * N, M * N)
    torch.cuda.synchronize()
    got = dC.cpu().numpy().view(np.complex64).reshape(batch, M, N)
    ref = np.matmul(A.astype(np.complex128), B.astype(np.complex128))
    assert rel_l2(got, ref) < TOL


# relative L2 bounds per precision: 3xTF32 carries ~21 mantissa bits per
# product (gated at the FP32-path tolerance); 3xBF16 ~16 bits; 1xBF16 8 bits
TC_TOL = {"tf32x3": 1e-5, "bf16x3": 1e-4, "bf16x1": 1e-2}


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "bf16x1"])
@pytest.mark.parametrize("M,K,N,batch", [(128, 16, 8, 1), (1000, 4, 8, 1), (4096, 16, 16, 2),
                                         (777, 64, 64, 1), (333, 3, 5, 3), (300, 128, 128, 1),
                                         (256, 32, 200, 1), (1, 1, 1, 1), (100000, 32, 96, 1),
                                         (50000, 8, 4, 3), (70001, 2, 2, 2), (9999, 16, 9, 1)])
def test_cgemm_tensor_core_matches_fp64(prec, M, K, N, batch):
    A = random_complex((batch, M, K), 21, np.complex64)
    B = random_complex((batch, K, N), 22, np.complex64)
    dA = torch.from_numpy(A.view(np.float32).copy()).cuda()
    dB = torch.from_numpy(B.view(np.float32).copy()).cuda()
    dC = torch.full((batch * M * N * 2,), float("nan"), dtype=torch.float32, device="cuda")
    P.tn_cgemm(dA, dB, dC, M, K, N, batch, M * K, K * N, M * N, prec=prec)
    torch.cuda.synchronize()
    got = dC.cpu().numpy().view(np.complex64).reshape(batch, M, N)
    ref = np.matmul(A.astype(np.complex128), B.astype(np.complex128))
    assert rel_l2(got, ref) < TC_TOL[prec], rel_l2(got, ref)


# Shapes of the TMA-pipelined tcgen05 kernels (K >= 16, 2N a multiple of 32,
# M >= 128), including ragged M (partial last tile, rows past M read as zero
# and not stored), batches (one launch per item) and the large benchmark
# shape, whose reference is checked on sampled rows (every row must be
# written: C starts as NaN).
@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "bf16x1"])
# (38000, 64, 512) and (65536, 512, 512) fill enough waves of the GPU that
# 3xBF16 takes its 256-column kernel (the others take the 128-column one);
# N = 16 and 32 take 32- and 64-column tiles, and K = 16 a k-block that the
# copy pads with zeros past 2K (BF16 stages hold 64 real K).
@pytest.mark.parametrize("M,K,N,batch", [(128, 32, 128, 1), (1000, 64, 128, 1), (130, 32, 256, 2),
                                         (4096, 256, 64, 1), (2048, 128, 512, 1), (16384, 512, 512, 1),
                                         (38000, 64, 512, 1), (65536, 512, 512, 1), (4096, 16, 16, 1),
                                         (1000, 32, 16, 1), (3000, 16, 32, 2), (65536, 32, 32, 1)])
def test_cgemm_large_tensor_core_matches_fp64(prec, M, K, N, batch):
    A = random_complex((batch, M, K), 31, np.complex64)
    B = random_complex((batch, K, N), 32, np.complex64)
    dA = torch.from_numpy(A.view(np.float32).copy()).cuda()
    dB = torch.from_numpy(B.view(np.float32).copy()).cuda()
    dC = torch.full((batch * M * N * 2,), float("nan"), dtype=torch.float32, device="cuda")
    P.tn_cgemm(dA, dB, dC, M, K, N, batch, M * K, K * N, M * N, prec=prec)
    torch.cuda.synchronize()
    got = dC.cpu().numpy().view(np.complex64).reshape(batch, M, N)
    assert np.isfinite(got.view(np.float32)).all()
    rows = np.arange(M) if M <= 4096 else np.unique(np.r_[0, M - 1, np.random.default_rng(3).integers(0, M, 512)])
    ref = np.matmul(A[:, rows].astype(np.complex128), B.astype(np.complex128))
    assert rel_l2(got[:, rows], ref) < TC_TOL[prec], rel_l2(got[:, rows], ref)


@pytest.mark.parametrize("prec,tol", [("fp32", TOL), ("tf32x3", TOL), ("bf16x3", 1e-4)])
def test_cgemm_chain_of_61_unitary_steps(prec, tol, capsys):
    # 61 stem-like GEMM steps (4 x 4 complex unitaries, magnitudes kept) applied
    # one after another through tn_cgemm; the error against FP64 and its
    # component along the exact result (negative: the magnitude shrinks, the
    # signature of truncating accumulation) are printed. The FP32-accurate
    # paths must stay within 1e-5 after all steps.
    rng = np.random.default_rng(61)
    M, steps = 1 << 16, 61

    def rnd(*shape):
        return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)

    def dev(x):
        return torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64)).view(np.float32).reshape(-1).copy()).cuda()

    x = rnd(M, 4).astype(np.complex64).astype(np.complex128)
    ref = x.copy()
    dX, dY = dev(x), torch.zeros(2 * M * 4, dtype=torch.float32, device="cuda")
    for _ in range(steps):
        q, r = np.linalg.qr(rnd(4, 4))
        U = (q * (np.diag(r) / np.abs(np.diag(r)))).astype(np.complex64).astype(np.complex128)
        P.tn_cgemm(dX, dev(U), dY, M, 4, 4, prec=prec)
        dX, dY = dY, dX
        ref = ref @ U
    torch.cuda.synchronize()
    got = dX.cpu().numpy().view(np.complex64).astype(np.complex128).reshape(M, 4)
    e = got - ref
    nr = np.vdot(ref, ref).real
    rel = float(np.sqrt(np.vdot(e, e).real / nr))
    bias = float(np.vdot(ref, e).real / nr)
    with capsys.disabled():
        print(f"\n61-step unitary chain, {prec}: rel L2 {rel:.3e}, bias along the exact value {bias:.3e}")
    assert rel < tol


def test_fp32_fma_peak_is_sane():
    # the fused pass's roofline denominator: independent FMA chains on every
    # SM; it must see every SM and land between a quarter of and just above
    # the unit-count bound (SMs x 128 lanes x 2 flops x 2.07 GHz)
    tflops, sms = P.tn_fp32_fma_peak()
    props = torch.cuda.get_device_properties(0)
    assert sms == props.multi_processor_count
    nominal = sms * 128 * 2 * 2.07e9 / 1e12
    assert 0.25 * nominal < tflops < 1.05 * nominal, (tflops, nominal)


def test_linear_xeb_kernel():
    a = random_complex((4096,), 3) / 64.0
    d = torch.from_numpy(a.view(np.float64).copy()).cuda()
    got = P.tn_linear_xeb(d, 12)
    ref = oracle.linear_xeb(np.abs(a) ** 2, 12)
    assert got == pytest.approx(ref, rel=1e-12)


# ------------------------------------------------------------ stem, small

def _plan(c, oq, closed, **kw):
    net = P.tn_build_network(c, oq, closed)
    plan = P.tn_plan_create(net, **kw)
    return net, plan


@pytest.mark.parametrize("mode", ["fused", "plain"])
def test_grid4x4_m8_closed_amplitudes(mode):
    # 16 qubits, 8 cycles, 64 seeded bitstrings as 64 closed prefixes
    name = "grid4x4_m8"
    cfg = CONFIGS[name]
    c = config_circuit(name)
    bits = [list(random_bits(16, cfg["bit_seed"] + i)) for i in range(cfg["bitstrings"])]
    net, plan = _plan(c, [], bits[0], cw_limit=30, restarts=4)
    P.tn_plan_prepare(plan, np.asarray(bits, dtype=np.uint8))
    got = run(plan, 0, 1, mode=mode)[:, 0]
    psi = oracle.statevector(c)
    ref = np.array([oracle.sv_amplitudes(c, [], b, psi)[0] for b in bits])
    assert rel_l2(got, ref) < TOL


@pytest.mark.parametrize("mode", ["fused", "plain"])
@pytest.mark.parametrize("rows,cols,m,cw,n_open,seed", [(3, 4, 8, 7, 3, 1), (4, 4, 10, 9, 6, 2),
                                                        (3, 3, 6, 5, 0, 3), (2, 3, 4, 6, 6, 4)])
def test_sliced_partials_and_sum(mode, rows, cols, m, cw, n_open, seed):
    c = random_circuit(grid_layout(rows, cols), m, 50 + seed)
    oq = list(range(n_open))
    cb = list(random_bits(c.n_qubits - n_open, seed))
    net, plan = _plan(c, oq, cb, cw_limit=cw, restarts=3, min_sliced=2 if n_open < c.n_qubits else 0)
    P.tn_plan_prepare(plan)
    info = P.tn_plan_info(plan)
    nsl = info["n_sliced"]
    _, sl = P.tn_plan_export(plan)
    _, _, q, s = net.info()
    sliced = [(int(q[e]), int(s[e])) for e in sl]
    psi = oracle.statevector(c)
    ref = oracle.sv_amplitudes(c, oq, cb, psi)
    tot = run(plan, 0, 1 << nsl, mode=mode)[0]
    assert rel_l2(tot, ref) < TOL
    for sid in sorted({0, (1 << nsl) - 1, (1 << nsl) // 3}):
        part = run(plan, sid, sid + 1, mode=mode)[0]
        pref = oracle.sv_amplitudes(c, oq, cb, projectors=oracle.slice_assignment(sliced, sid))
        if np.linalg.norm(pref) > 1e-12:
            assert rel_l2(part, pref) < TOL
        else:
            assert np.linalg.norm(part) < 1e-6


def test_ranges_add_and_host_output():
    c = random_circuit(grid_layout(3, 4), 8, 71)
    oq = [0, 1, 2, 3]
    cb = list(random_bits(8, 9))
    net, plan = _plan(c, oq, cb, cw_limit=7, restarts=3, min_sliced=3)
    P.tn_plan_prepare(plan)
    nsl = P.tn_plan_info(plan)["n_sliced"]
    full = run(plan, 0, 1 << nsl)
    out = torch.zeros(2 * 16, dtype=torch.float64, device="cuda")
    P.tn_contract_stem(plan, 0, 3, out)
    P.tn_contract_stem(plan, 3, 1 << nsl, out, accumulate=True)
    torch.cuda.synchronize()
    acc = out.cpu().numpy().view(np.complex128)
    assert rel_l2(acc, full[0]) < 1e-12
    host = np.zeros(32)
    P.tn_contract_stem(plan, 0, 1 << nsl, host)
    assert rel_l2(host.view(np.complex128), full[0]) < 1e-12
    empty = run(plan, 2, 2)
    assert np.all(empty == 0)
    with pytest.raises(P.TnError):
        P.tn_contract_stem(plan, 0, (1 << nsl) + 1, out)
    with pytest.raises(P.TnError):
        P.tn_contract_stem(plan, 3, 2, out)


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3", "bf16x1"])
def test_stem_gemm_steps_per_precision(prec):
    # gemm_min_kn = 2 routes every step with two or more contracted or new
    # bits through a GEMM (SIMT for fp32, tcgen05 otherwise)
    c = random_circuit(grid_layout(4, 4), 10, 93)
    oq = [0, 1, 2, 3, 4, 5]
    cb = list(random_bits(10, 4))
    net, plan = _plan(c, oq, cb, cw_limit=9, restarts=3, min_sliced=2, gemm_min_kn=2)
    assert P.tn_plan_info(plan)["n_gemm_steps"] > 0
    P.tn_plan_prepare(plan)
    nsl = P.tn_plan_info(plan)["n_sliced"]
    got = run(plan, 0, 1 << nsl, prec=prec)[0]
    ref = oracle.sv_amplitudes(c, oq, cb)
    # a single BF16 product per step is reported, not gated: ~2^-9 per step
    # over tens of steps; here it only has to stay a sane approximation
    tol = {"fp32": TOL, "tf32x3": TOL, "bf16x3": 1e-4, "bf16x1": 0.1}[prec]
    assert rel_l2(got, ref) < tol, rel_l2(got, ref)


def test_all_qubits_open_is_statevector():
    c = random_circuit(grid_layout(2, 3), 6, 5)
    oq = list(range(6))
    net, plan = _plan(c, oq, [], cw_limit=8, restarts=2)
    P.tn_plan_prepare(plan)
    got = run(plan, 0, 1 << P.tn_plan_info(plan)["n_sliced"])[0]
    assert rel_l2(got, oracle.statevector(c)) < TOL


def test_prefix_batch_equals_single_prefixes():
    c = random_circuit(grid_layout(3, 4), 8, 77)
    oq = [0, 5]
    pres = [list(random_bits(10, 300 + i)) for i in range(5)]
    net, plan = _plan(c, oq, pres[0], cw_limit=6, restarts=2, slice_batch=3)
    P.tn_plan_prepare(plan, np.asarray(pres, dtype=np.uint8))
    nsl = P.tn_plan_info(plan)["n_sliced"]
    got = run(plan, 0, 1 << nsl)
    psi = oracle.statevector(c)
    for i, p in enumerate(pres):
        assert rel_l2(got[i], oracle.sv_amplitudes(c, oq, p, psi)) < TOL


def test_set_prefix_revalues_projectors_and_short_names():
    # a plan made after tn_set_prefix contracts the new prefix; one made before
    # keeps the old one; tn_destroy_* free handles at once
    c = random_circuit(grid_layout(3, 4), 8, 78)
    oq = [1, 6]
    a, b = list(random_bits(10, 401)), list(random_bits(10, 402))
    net = P.tn_build_network(c, oq, a)
    plan_a = P.tn_plan_create(net, cw_limit=6, restarts=2)
    P.tn_set_prefix(net, b)
    plan_b = P.tn_plan_create(net, cw_limit=6, restarts=2)
    psi = oracle.statevector(c)
    for plan, bits in ((plan_a, a), (plan_b, b)):
        P.tn_plan_prepare(plan)
        got = run(plan, 0, 1 << P.tn_plan_info(plan)["n_sliced"])[0]
        assert rel_l2(got, oracle.sv_amplitudes(c, oq, bits, psi)) < TOL
    P.tn_destroy_plan(plan_a)
    P.tn_destroy_plan(plan_b)
    P.tn_destroy_network(net)


# ------------------------------------------------------- frugal sampling

def _sample_gpu(amps, n, M, u, key):
    B, K = amps.shape
    d_a = torch.from_numpy(np.ascontiguousarray(amps).view(np.float64).copy()).cuda()
    d_u = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    d_k = torch.from_numpy(np.ascontiguousarray(key)).cuda()
    idx = torch.empty(B, dtype=torch.int32, device="cuda")
    cnt = torch.empty(B, dtype=torch.int32, device="cuda")
    picked = torch.empty(2 * B, dtype=torch.float64, device="cuda")
    P.tn_frugal_sample(d_a, d_u, d_k, B, K, n, M, idx, cnt, picked)
    torch.cuda.synchronize()
    pk = picked.cpu().numpy()
    return idx.cpu().numpy(), cnt.cpu().numpy(), pk[0::2] + 1j * pk[1::2]


@pytest.mark.parametrize("B,K,n,M", [(300, 64, 12, 10.0), (7, 256, 20, 3.0), (1000, 1, 5, 0.5),
                                     (64, 100, 9, 40.0)])
def test_frugal_sample_matches_oracle(B, K, n, M):
    amps = random_complex((B, K), 40 + K) / math.sqrt(2.0 * 2 ** n)
    u = random_uniform((B, K), 500 + K)
    key = random_uniform((B, K), 600 + K)
    idx, cnt, picked = _sample_gpu(amps, n, M, u, key)
    ridx, rcnt = oracle.frugal_sample(amps, n, M, u, key)
    assert (idx == ridx).all() and (cnt == rcnt).all()
    ok = ridx >= 0
    assert np.array_equal(picked[ok], amps[ok, ridx[ok]]) and (picked[~ok] == 0).all()


def test_frugal_sampling_of_contracted_batches():
    # 30 qubits, 16 prefixes x 64 open amplitudes contracted over all slices,
    # then one sample per prefix batch; decisions match the oracle on the
    # same amplitudes exactly, and the state vector's amplitudes wherever no
    # candidate sits within 1e-4 of its threshold
    name = "grid5x6_m14"
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "grid5x6_m14_amps.json")))
    c = config_circuit(name)
    oq = g["open_qubits"]
    pres = np.asarray(g["prefixes"], dtype=np.uint8)
    net, plan = _plan(c, oq, list(pres[0]), cw_limit=30, restarts=2)
    P.tn_plan_prepare(plan, pres)
    amps = run(plan, 0, 1 << P.tn_plan_info(plan)["n_sliced"])
    n, M = c.n_qubits, 10.0
    u = random_uniform(amps.shape, 7001)
    key = random_uniform(amps.shape, 7002)
    idx, cnt, _ = _sample_gpu(amps, n, M, u, key)
    ridx, rcnt = oracle.frugal_sample(amps, n, M, u, key)
    assert (idx == ridx).all() and (cnt == rcnt).all()
    ref = np.asarray(g["amps_re"]) + 1j * np.asarray(g["amps_im"])
    sidx, _ = oracle.frugal_sample(ref, n, M, u, key)
    thr = np.abs(ref) ** 2 * 2.0 ** n / M
    clear = (np.abs(u - thr) > 1e-4 * np.maximum(thr, 1e-300)).all(axis=1)
    assert clear.sum() >= 12
    assert (idx[clear] == sidx[clear]).all()


# ------------------------------------------------------------ 30-qubit grid

def test_grid5x6_m14_against_stored_statevector():
    path = os.path.join(GOLD, "grid5x6_m14_amps.json")
    g = json.load(open(path))
    name = g["workload"]
    c = config_circuit(name)
    oq = g["open_qubits"]
    pres = np.asarray(g["prefixes"], dtype=np.uint8)
    net, plan = _plan(c, oq, list(pres[0]), cw_limit=30, min_sliced=CONFIGS[name]["n_sliced"],
                      restarts=4)
    P.tn_plan_prepare(plan, pres)
    info = P.tn_plan_info(plan)
    assert info["n_sliced"] == CONFIGS[name]["n_sliced"]
    got = run(plan, 0, 1 << info["n_sliced"])
    ref = np.asarray(g["amps_re"]) + 1j * np.asarray(g["amps_im"])
    assert rel_l2(got, ref) < TOL


# ----------------------------------------------- full size, closed form
# With fSim(0, 0) = identity the network keeps its structure (the planner
# sees only structure, so the plan and every launch are the full-size ones)
# but its value factorises over qubits: a partial amplitude is the product
# over qubits of <x_q| ... P_v ... |0>, the projectors P_v sitting on the
# sliced wire segments of that qubit. Single-qubit sequences made only of
# sqrt(X) and sqrt(Y) end in exact basis states, so a factor can be zero up to
# rounding; the test therefore picks, per closed qubit, the prefix bit with the
# larger factor, and measures the error against the product of the per-qubit
# vector norms (the scale the FP32 rounding is relative to).

def _qubit_vectors(c, sliced_by_wire, slice_id):
    n = c.n_qubits
    events = [[] for _ in range(n)]
    for t in range(c.n_cycles + 1):
        for q in range(n):
            events[q].append(oracle.gate_1q(c.gates_1q[t][q]))
        if t == c.n_cycles:
            break
        for (a, b) in c.pairs[t]:
            events[a].append(np.eye(2))
            events[b].append(np.eye(2))
    vec = {}
    for q in range(n):
        v = np.array([1.0, 0.0], dtype=complex)
        for s_idx, G in enumerate(events[q]):
            key = (q, s_idx)
            if key in sliced_by_wire:
                v = v * (np.arange(2) == ((slice_id >> sliced_by_wire[key]) & 1))
            v = G @ v
        key = (q, len(events[q]))
        if key in sliced_by_wire:
            v = v * (np.arange(2) == ((slice_id >> sliced_by_wire[key]) & 1))
        vec[q] = v
    return vec


ZERO = 1e-9  # a per-qubit factor below this is zero up to FP64 rounding


def _closed_form(c, oq, closed_bits, sliced_by_wire, slice_id):
    """Partial amplitudes and their scale: the product of the per-qubit
    factors' magnitudes with numerically-zero factors counted as 1 (the FP32
    rounding of such a factor is relative to its unit-norm chain)."""
    vec = _qubit_vectors(c, sliced_by_wire, slice_id)
    closed = [q for q in range(c.n_qubits) if q not in set(oq)]
    scal = 1.0 + 0j
    scale = 1.0
    for q, b in zip(closed, closed_bits):
        f = vec[q][int(b)]
        scal *= f
        scale *= abs(f) if abs(f) > ZERO else 1.0
    out = np.ones(1, dtype=complex)
    for q in oq:
        out = np.kron(out, vec[q])
        nv = np.linalg.norm(vec[q])
        scale *= nv if nv > ZERO else 1.0
    return scal * out, scale


@pytest.mark.parametrize("name,n_open,extra", [("diag53_m14", None, {}),
                                               ("diag53_m14", None, {"tile_bits": 12, "max_pass_steps": 8}),
                                               ("diag53_m12", None, {}), ("diag53_m12", 0, {}),
                                               ("diag53_m12", 4, {}), ("diag53_m12", 8, {})])
def test_full_size_plan_identity_fsim_closed_form(name, n_open, extra):
    # the 53-qubit 12-cycle workload is also run at 1, 16 and 256 amplitudes
    # per batch (0, 4, 8 open qubits) beside its 64-amplitude default; the
    # 14-cycle one also with the tile and steps per pass its bench launch
    # configuration uses (the learned search's pick)
    from bench import plan_options, workload_inputs
    cfg = CONFIGS[name]
    c, oq, cb_bench = workload_inputs(name)
    if n_open is not None:
        oq = c.layout.open_qubits(n_open)
        cb_bench = list(random_bits(c.n_qubits - n_open, cfg["bit_seed"]))
    c0 = Circuit(c.n_qubits, c.n_cycles, c.gates_1q, c.pairs, 0.0, 0.0, c.layout)
    closed = [q for q in range(c.n_qubits) if q not in set(oq)]
    v0 = _qubit_vectors(c0, {}, 0)
    cb = [int(np.argmax(np.abs(v0[q]))) for q in closed]
    opts = dict(plan_options(name), **extra)
    net_ref, plan_ref = _plan(c, oq, cb_bench, **opts)
    net, plan = _plan(c0, oq, cb, **opts)
    o1, s1 = P.tn_plan_export(plan_ref)
    o2, s2 = P.tn_plan_export(plan)
    assert np.array_equal(o1, o2) and np.array_equal(s1, s2)
    P.tn_plan_prepare(plan)
    info = P.tn_plan_info(plan)
    _, _, q, s = net.info()
    wires = {(int(q[e]), int(s[e])): j for j, e in enumerate(s2)}
    nsl = info["n_sliced"]
    ids = [0, 1, 2, (1 << nsl) - 1, 12345 % (1 << nsl), 987654 % (1 << nsl)]
    for sid in ids:
        got = run(plan, sid, sid + 1)[0]
        ref, scale = _closed_form(c0, oq, cb, wires, sid)
        err = np.linalg.norm(got - ref) / scale
        assert err < TOL, (sid, err)
        if np.linalg.norm(ref) > 1e-2 * scale:
            assert rel_l2(got, ref) < TOL, (sid, rel_l2(got, ref))
    # a whole batch at the bench's batch size
    sb = info["batch_items"]
    got = run(plan, 0, sb)[0]
    parts = [_closed_form(c0, oq, cb, wires, sid) for sid in range(sb)]
    ref = sum(p[0] for p in parts)
    assert np.linalg.norm(got - ref) / max(p[1] for p in parts) < TOL


# ------------------------------- full size, real gates, stored oracle slices
# tests/golden/<workload>_slices.json holds FP64 oracle values of slices 0
# and 1 of the 53-qubit 12- and 14-cycle workloads (written by
# make_stored_slices.py from the order and sliced wire segments in
# <workload>_scheme.json, which make_scheme.py exports from the planner). The
# plan is rebuilt from that order and those segments, so the comparison is
# always on the same sub-networks.

def _stored_plan(name, **kw):
    from bench import workload_inputs
    sch = json.load(open(os.path.join(GOLD, f"{name}_scheme.json")))
    gold = json.load(open(os.path.join(GOLD, f"{name}_slices.json")))
    assert gold["sliced_wires"] == sch["sliced_wires"]
    c, oq, cb = workload_inputs(name)
    net = P.tn_build_network(c, oq, cb)
    _, _, q, s = net.info()
    eid = {(int(a), int(b)): e for e, (a, b) in enumerate(zip(q, s))}
    sliced = [eid[tuple(w)] for w in sch["sliced_wires"]]
    plan = P.tn_plan_create(net, order=[tuple(x) for x in sch["order"]], sliced_edges=sliced, **kw)
    return plan, gold


def _stored_m12_plan(**kw):
    return _stored_plan("diag53_m12", **kw)


@pytest.mark.parametrize("mode", ["fused", "plain"])
def test_diag53_m12_slices_match_stored_oracle(mode):
    plan, gold = _stored_m12_plan()
    P.tn_plan_prepare(plan)
    for sid, v in gold["slices"].items():
        ref = np.asarray(v["re"]) + 1j * np.asarray(v["im"])
        got = run(plan, int(sid), int(sid) + 1, mode=mode)[0]
        assert rel_l2(got, ref) < TOL, (sid, rel_l2(got, ref))


def test_diag53_m12_per_branch_merges_match_stored_oracle(capsys):
    # merge_group -1: the plain model chooses which consecutive branches to
    # merge; the stored scheme's slices must come out the same
    plan, gold = _stored_m12_plan(merge_group=-1)
    base, _ = _stored_m12_plan()
    info, info0 = P.tn_plan_info(plan), P.tn_plan_info(base)
    assert info["n_branches"] < info0["n_branches"]
    P.tn_plan_prepare(plan)
    errs = []
    for sid, v in gold["slices"].items():
        ref = np.asarray(v["re"]) + 1j * np.asarray(v["im"])
        got = run(plan, int(sid), int(sid) + 1)[0]
        errs.append(rel_l2(got, ref))
    with capsys.disabled():
        print(f"\ndiag53_m12 per-branch merges ({info0['n_branches']} -> {info['n_branches']} branches, "
              f"{info['n_gemm_steps']} GEMM steps): rel L2 vs FP64 oracle per slice {errs}")
    assert max(errs) < TOL


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3", "bf16x1"])
def test_diag53_m12_merged_gemm_steps_per_precision(prec, capsys):
    # branch merging (runs of 3) turns most stem steps into GEMM steps
    plan, gold = _stored_m12_plan(merge_group=3)
    assert P.tn_plan_info(plan)["n_gemm_steps"] > 30
    P.tn_plan_prepare(plan)
    errs = []
    for sid, v in gold["slices"].items():
        ref = np.asarray(v["re"]) + 1j * np.asarray(v["im"])
        got = run(plan, int(sid), int(sid) + 1, prec=prec)[0]
        errs.append(rel_l2(got, ref))
    with capsys.disabled():
        print(f"\ndiag53_m12 merged, {prec}: rel L2 vs FP64 oracle per slice {errs}")
    # The FP32-accurate paths (FP32 SIMT and 3xTF32) are gated at 1e-5. 3xTF32
    # keeps hi*hi and the two correction products in separate tensor-memory
    # accumulators (measured 7.8e-6 and 8.1e-6 here; 2.5e-5 when all three
    # shared one accumulator, whose truncating FP32 adds biased every step).
    # 3xBF16 carries about 16 significand bits per operand (hi + lo), so its
    # error is reported and bounded, as is the single BF16 product's.
    tol = {"fp32": TOL, "tf32x3": TOL, "bf16x3": 1e-4, "bf16x1": 0.1}[prec]
    assert max(errs) < tol


# The bench workload (53 qubits, 14 cycles, cw 30: stem tensors of 2^30
# entries) with real gates, in the bench's launch configuration (tile 12, up
# to 8 steps per pass, one slice per launch), against the stored FP64 oracle
# slices, element by element.
@pytest.mark.parametrize("extra", [{"tile_bits": 12, "max_pass_steps": 8}, {}])
def test_diag53_m14_slices_match_stored_oracle(extra, capsys):
    plan, gold = _stored_plan("diag53_m14", **extra)
    P.tn_plan_prepare(plan)
    info = P.tn_plan_info(plan)
    assert info["cw"] == 30 and info["n_gemm_steps"] == 0
    errs = []
    for sid, v in gold["slices"].items():
        ref = np.asarray(v["re"]) + 1j * np.asarray(v["im"])
        got = run(plan, int(sid), int(sid) + 1)[0]
        errs.append(rel_l2(got, ref))
    with capsys.disabled():
        print(f"\ndiag53_m14 {extra or 'planner defaults'}: rel L2 vs FP64 oracle per slice {errs}")
    assert max(errs) < TOL


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3", "bf16x1"])
def test_diag53_m14_merged_gemm_steps_per_precision(prec, capsys):
    # the bench's precision sweep plan: runs of 3 branches merged, every stem
    # step a GEMM step; FP32-accurate paths gated at 1e-5 (reading of the
    # tolerance: FP32 SIMT and 3xTF32), the BF16 ones bounded
    plan, gold = _stored_plan("diag53_m14", merge_group=3)
    assert P.tn_plan_info(plan)["n_gemm_steps"] > 60
    P.tn_plan_prepare(plan)
    errs = []
    for sid, v in gold["slices"].items():
        ref = np.asarray(v["re"]) + 1j * np.asarray(v["im"])
        got = run(plan, int(sid), int(sid) + 1, prec=prec)[0]
        errs.append(rel_l2(got, ref))
    with capsys.disabled():
        print(f"\ndiag53_m14 merged, {prec}: rel L2 vs FP64 oracle per slice {errs}")
    tol = {"fp32": TOL, "tf32x3": TOL, "bf16x3": 1e-4, "bf16x1": 0.1}[prec]
    assert max(errs) < tol


# The 20-cycle workload with its best plan (total cost 2^61.99: cw 30, 23
# sliced edges; tests/golden/diag53_m20_scheme.json, exported by
# make_scheme.py with the options it records): real gates, the bench's launch
# configuration. Slice 0 against the stored FP64 oracle value; 8 seeded
# slices timed and the whole 64-amplitude batch extrapolated (Supp. A.4:
# per-subtask time x number of subtasks).
def test_diag53_m20_best_plan_slice_and_time(capsys):
    from bench import workload_inputs
    from synthetic.circuits import SplitMix64
    sch = json.load(open(os.path.join(GOLD, "diag53_m20_scheme.json")))
    c, oq, cb = workload_inputs("diag53_m20")
    net = P.tn_build_network(c, oq, cb)
    _, _, q, s = net.info()
    eid = {(int(a), int(b)): e for e, (a, b) in enumerate(zip(q, s))}
    plan = P.tn_plan_create(net, order=[tuple(x) for x in sch["order"]],
                            sliced_edges=[eid[tuple(w)] for w in sch["sliced_wires"]],
                            cw_limit=30, tile_bits=12, max_pass_steps=8)
    P.tn_plan_prepare(plan)
    info = P.tn_plan_info(plan)
    assert info["cw"] == 30 and info["n_sliced"] == 23
    assert abs(info["log2_tc"] - sch["log2_tc"]) < 1e-6
    gold_path = os.path.join(GOLD, "diag53_m20_slices.json")
    err = None
    if os.path.exists(gold_path):
        gold = json.load(open(gold_path))
        assert gold["sliced_wires"] == sch["sliced_wires"]
        for sid, v in gold["slices"].items():
            ref = np.asarray(v["re"]) + 1j * np.asarray(v["im"])
            err = rel_l2(run(plan, int(sid), int(sid) + 1)[0], ref)
            assert err < TOL, (sid, err)
    rng = SplitMix64(CONFIGS["diag53_m20"]["bit_seed"])
    ids = [rng.next() % (1 << info["n_sliced"]) for _ in range(8)]
    out = torch.zeros(2 * 64, dtype=torch.float64, device="cuda")
    P.tn_contract_stem(plan, ids[0], ids[0] + 1, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for sid in ids:
        P.tn_contract_stem(plan, sid, sid + 1, out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / len(ids)
    days = ms * 2.0 ** info["n_sliced"] / 1e3 / 86400
    with capsys.disabled():
        print(f"\ndiag53_m20 plan 2^{info['log2_tc']:.2f} (cw {info['cw']}, {info['n_sliced']} sliced): "
              f"slice 0 rel L2 vs FP64 oracle {err}; {ms:.1f} ms per slice, "
              f"{8 * info['stem_tc_per_slice'] / (ms / 1e3) / 1e12:.1f} TFLOP/s, one 64-amplitude batch "
              f"{days:.2f} days on one GPU")


# ------------------------------------------- hypergraph networks (Sec. 3)
# The circuit as a multi-hypergraph (diagonal part of fSim(pi/2, phi) on two
# hyperedges): greedy scheme, FP64 pairwise steps on the GPU, amplitudes of
# every prepared prefix against the FP64 state vector.
@pytest.mark.parametrize("rows,cols,m,seed,n_open,n_pre", [(4, 4, 8, 1, 0, 64), (3, 4, 8, 71, 4, 3),
                                                          (4, 5, 12, 3, 6, 2)])
def test_hypernetwork_plan_matches_statevector(rows, cols, m, seed, n_open, n_pre):
    c = random_circuit(grid_layout(rows, cols), m, seed)
    oq = list(range(n_open))
    nc = c.n_qubits - n_open
    pres = np.asarray([list(random_bits(nc, 300 + i)) for i in range(n_pre)], dtype=np.uint8)
    hnet = P.tn_build_hypernetwork(c, oq, list(pres[0]))
    plan = P.tn_plan_create(hnet, cw_limit=30, restarts=8)
    P.tn_plan_prepare(plan, pres)
    got = run(plan, 0, 1)
    psi = oracle.statevector(c)
    ref = np.stack([oracle.sv_amplitudes(c, oq, list(pr), psi=psi) for pr in pres])
    assert rel_l2(got, ref) < 1e-11, rel_l2(got, ref)
    # ranges add: empty range then the slice again, accumulated into host memory
    host = np.zeros(2 * got.size)
    P.tn_contract_stem(plan, 0, 0, host)
    P.tn_contract_stem(plan, 0, 1, host, accumulate=True)
    P.tn_contract_stem(plan, 0, 1, host, accumulate=True)
    assert rel_l2(host.view(np.complex128).reshape(got.shape), 2 * ref) < 1e-11
