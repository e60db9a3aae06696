"""GPU test of tn_contract_stem_noalloc, the allocation-free entry point for
callers that must not allocate device memory while contracting (cudaMalloc
synchronises the device and can fail under a memory budget owned by someone
else). It must give the same amplitudes as tn_contract_stem, on two calls in
a row (the shared static scratch keeps the last call's contents, so the
second call checks that nothing leaks from the first).

This file is named to be collected last, so a run that stops at the first
failure has already run every other test; it also passes when run alone.
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _amps(fn, plan, s0, s1, n):
    out = torch.full((2 * n,), float("nan"), dtype=torch.float64, device="cuda")
    fn(plan, s0, s1, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.complex128)


@pytest.mark.parametrize("n_prefixes", [1, 3])
def test_noalloc_matches_contract_stem_twice(n_prefixes):
    c = random_circuit(grid_layout(3, 4), 8, 71)
    oq = [0, 1, 2, 3]
    pres = np.asarray([list(random_bits(8, 40 + i)) for i in range(n_prefixes)], dtype=np.uint8)
    net = P.tn_build_network(c, oq, list(pres[0]))
    plan = P.tn_plan_create(net, cw_limit=7, restarts=3, min_sliced=3)
    P.tn_plan_prepare(plan, pres)
    nsl = P.tn_plan_info(plan)["n_sliced"]
    n = n_prefixes * 16
    ref = _amps(lambda *a: P.tn_contract_stem(*a, mode="fused"), plan, 0, 1 << nsl, n)
    for _ in range(2):
        got = _amps(P.tn_contract_stem_noalloc, plan, 0, 1 << nsl, n)
        assert _rel(got, ref) < TOL
    # a partial range, then the rest accumulated, in two calls
    part = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
    P.tn_contract_stem_noalloc(plan, 0, 3, part)
    P.tn_contract_stem_noalloc(plan, 3, 1 << nsl, part, accumulate=True)
    torch.cuda.synchronize()
    assert _rel(part.cpu().numpy().view(np.complex128), ref) < TOL


def test_noalloc_rejects_oversize_plan_and_host_output():
    c = random_circuit(grid_layout(4, 6), 6, 5)
    oq = list(range(22))  # 22 open qubits: the final tensor alone exceeds 2^20 entries
    net = P.tn_build_network(c, oq, list(random_bits(2, 1)))
    plan = P.tn_plan_create(net, cw_limit=24, restarts=1)
    P.tn_plan_prepare(plan)
    out = torch.zeros(2 << 22, dtype=torch.float64, device="cuda")
    with pytest.raises(P.TnError) as e:
        P.tn_contract_stem_noalloc(plan, 0, 1, out)
    assert e.value.status == 6
    small = random_circuit(grid_layout(2, 3), 4, 2)
    snet = P.tn_build_network(small, [0, 1], list(random_bits(4, 3)))
    splan = P.tn_plan_create(snet, cw_limit=8)
    P.tn_plan_prepare(splan)
    with pytest.raises(P.TnError) as e:
        P.tn_contract_stem_noalloc(splan, 0, 1, np.zeros(8))
    assert e.value.status == 1


# The three ways the allocation-free call differs from tn_contract_stem's
# graph path, each checked against tn_contract_stem and against the FP64
# oracle's state vector (the sum over all slices is the amplitude itself):
#   shrink  - the plan's slices per launch do not fit the static buffers
#             (slice_batch * 2^max_rank > 2^20), so the call runs fewer per launch;
#   cbank   - one batch item per launch: passes read their branch matrices
#             from the constant bank (staging kernel + device copy);
#   gemm    - a branch-merged plan whose stem has GEMM steps.
# After a first call has loaded every kernel, further calls must leave the
# device's free memory unchanged: the call allocates nothing.
CASES = {
    "shrink": dict(grid=(4, 5), cycles=12, seed=72, opts=dict(cw_limit=14, restarts=2, min_sliced=8,
                                                               slice_batch=1024)),
    "cbank": dict(grid=(3, 4), cycles=8, seed=71, opts=dict(cw_limit=7, restarts=3, min_sliced=3,
                                                             slice_batch=1)),
    "gemm": dict(grid=(3, 4), cycles=8, seed=71, opts=dict(cw_limit=7, restarts=3, min_sliced=3,
                                                            merge_group=3)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_paths_match_oracle_without_allocating(case):
    cfg = CASES[case]
    c = random_circuit(grid_layout(*cfg["grid"]), cfg["cycles"], cfg["seed"])
    oq = [0, 1, 2, 3]
    cb = list(random_bits(c.n_qubits - len(oq), 40))
    net = P.tn_build_network(c, oq, cb)
    plan = P.tn_plan_create(net, **cfg["opts"])
    P.tn_plan_prepare(plan)
    info = P.tn_plan_info(plan)
    nsl = info["n_sliced"]
    if case == "shrink":
        assert info["batch_items"] * info["max_stem_elems"] > (1 << 20)
    elif case == "cbank":
        assert info["batch_items"] == 1 and info["n_passes_cbank"] > 0
    else:
        assert info["n_gemm_steps"] > 0
    ref_sv = oracle.sv_amplitudes(c, oq, cb)
    ref = _amps(lambda *a: P.tn_contract_stem(*a, mode="fused"), plan, 0, 1 << nsl, 16)
    assert _rel(ref, ref_sv) < TOL
    # every output buffer exists before the free-memory reading
    outs = [torch.full((32,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(4)]
    P.tn_contract_stem_noalloc(plan, 0, 1 << nsl, outs[3])  # loads every kernel it uses
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    P.tn_contract_stem_noalloc(plan, 0, 1 << nsl, outs[0])
    P.tn_contract_stem_noalloc(plan, 0, 1 << nsl, outs[1])
    half = (1 << nsl) // 2 + 1
    P.tn_contract_stem_noalloc(plan, 0, half, outs[2])
    P.tn_contract_stem_noalloc(plan, half, 1 << nsl, outs[2], accumulate=True)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    for o in outs[:3]:
        got = o.cpu().numpy().view(np.complex128)
        assert _rel(got, ref) < TOL and _rel(got, ref_sv) < TOL
    assert free1 == free0
