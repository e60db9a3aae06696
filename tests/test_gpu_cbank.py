"""Branch matrices in the constant bank: a fused pass launched with one batch
item (one prefix, one slice) takes the branch matrices of its (2,2) steps and
paired (2,1), (1,3), (1,2) steps from a constant-bank copy staged on the
launch's stream; launches with several items read them from shared memory. Both paths against the FP64 oracle
(relative L2 error <= 1e-5), against each other, per slice, and with two
plans running on two streams at once.
"""

import numpy as np
import pytest

import oracle
import paper_2005_06787_gb300 as P
from synthetic.circuits import grid_layout, random_bits, random_circuit

pytestmark = pytest.mark.gpu
TOL = 1e-5

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    P.build()
    P.load()
    torch.cuda.set_device(0)


@pytest.fixture(autouse=True)
def _device_waits_completed():
    yield
    P.tn_device_status()


def rel_l2(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def contract(plan, s0, s1, stream=None, out=None):
    info = P.tn_plan_info(plan)
    if out is None:
        out = torch.zeros(2 << info["n_open"], dtype=torch.float64, device="cuda")
    P.tn_contract_stem(plan, s0, s1, out, stream=stream)
    return out


def amps(out):
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.complex128)


def is_22(s, pair):
    return s["pass_"] >= 0 and not s["gemm"] and s["k"] == 2 and s["n"] == 2 and s["pair"] == pair


# a 3x4 grid, 6 cycles, seed 1: its plans hold (2,2) steps whose contracted
# bits include tile position 0 (rest indices taken one at a time)
@pytest.mark.parametrize("n_open,tile", [(0, 6), (4, 6), (4, 10)])
def test_unpaired_22_steps_from_constant_bank(n_open, tile):
    lay = grid_layout(3, 4)
    c = random_circuit(lay, 6, 1)
    oq = lay.open_qubits(n_open) if n_open else []
    cb = list(random_bits(c.n_qubits - len(oq), 7))
    net = P.tn_build_network(c, oq, cb)
    plan = P.tn_plan_create(net, cw_limit=30, restarts=1, seed=1, tile_bits=tile, slice_batch=1)
    assert any(is_22(s, 0) for s in P.tn_plan_steps(plan))
    P.tn_plan_prepare(plan)
    info = P.tn_plan_info(plan)
    assert info["batch_items"] == 1 and info["n_passes_cbank"] > 0
    got = amps(contract(plan, 0, 1 << info["n_sliced"]))
    assert rel_l2(got, oracle.sv_amplitudes(c, oq, cb)) < TOL


def _sliced_case(slice_batch):
    lay = grid_layout(4, 4)
    c = random_circuit(lay, 10, 52)
    oq = list(range(6))
    cb = list(random_bits(c.n_qubits - 6, 2))
    net = P.tn_build_network(c, oq, cb)
    plan = P.tn_plan_create(net, cw_limit=9, restarts=3, min_sliced=3, slice_batch=slice_batch)
    P.tn_plan_prepare(plan)
    return c, oq, cb, net, plan


def test_constant_bank_and_shared_memory_paths_agree_per_slice():
    c, oq, cb, net, plan1 = _sliced_case(1)
    _, _, _, _, plan4 = _sliced_case(4)
    i1, i4 = P.tn_plan_info(plan1), P.tn_plan_info(plan4)
    steps = P.tn_plan_steps(plan1)
    assert any(is_22(s, 1) for s in steps) and any(is_22(s, 0) for s in steps)
    # the other shapes taken from the constant bank when paired
    paired = {(s["k"], s["n"]) for s in steps if s["pass_"] >= 0 and not s["gemm"] and s["pair"]}
    assert {(2, 1), (1, 3), (1, 2)} <= paired
    # the same scheme (the planner is seeded); only the launch batching differs
    assert P.tn_plan_steps(plan1) == P.tn_plan_steps(plan4)
    assert i1["batch_items"] == 1 and i1["n_passes_cbank"] > 0
    assert i4["batch_items"] == 4 and i4["n_passes_cbank"] == 0
    nsl = i1["n_sliced"]
    assert nsl >= 3
    _, sl = P.tn_plan_export(plan1)
    _, _, q, s = net.info()
    sliced = [(int(q[e]), int(s[e])) for e in sl]
    psi = oracle.statevector(c)
    tot1 = amps(contract(plan1, 0, 1 << nsl))
    tot4 = amps(contract(plan4, 0, 1 << nsl))
    assert rel_l2(tot1, oracle.sv_amplitudes(c, oq, cb, psi)) < TOL
    # identical FP32 partials; only the FP64 summation order may differ
    assert rel_l2(tot1, tot4) < 1e-9
    for sid in sorted({0, 1, (1 << nsl) - 1, (1 << nsl) // 3}):
        part = amps(contract(plan1, sid, sid + 1))
        pref = oracle.sv_amplitudes(c, oq, cb, projectors=oracle.slice_assignment(sliced, sid))
        if np.linalg.norm(pref) > 1e-12:
            assert rel_l2(part, pref) < TOL
        else:
            assert np.linalg.norm(part) < 1e-6


def test_constant_bank_calls_on_two_streams():
    # two plans with different branch matrices; calls on two streams must give
    # what they give one after the other
    plans = []
    for seed, bits in ((61, 3), (62, 4)):
        lay = grid_layout(4, 5)
        c = random_circuit(lay, 10, seed)
        oq = lay.open_qubits(4)
        cb = list(random_bits(c.n_qubits - 4, bits))
        net = P.tn_build_network(c, oq, cb)
        plan = P.tn_plan_create(net, cw_limit=11, restarts=2, min_sliced=4, slice_batch=1)
        P.tn_plan_prepare(plan)
        info = P.tn_plan_info(plan)
        assert info["n_passes_cbank"] > 0
        plans.append((plan, 1 << info["n_sliced"], oracle.sv_amplitudes(c, oq, cb)))
    seq = [amps(contract(p, 0, n)) for p, n, _ in plans]
    for (_, _, ref), got in zip(plans, seq):
        assert rel_l2(got, ref) < TOL
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = [torch.zeros(2 << 4, dtype=torch.float64, device="cuda") for _ in plans]
    torch.cuda.synchronize()
    for _ in range(3):
        for (p, n, _), st, o in zip(plans, streams, outs):
            contract(p, 0, n, stream=st, out=o)
        torch.cuda.synchronize()
        for o, ref in zip(outs, seq):
            assert np.array_equal(amps(o), ref)
