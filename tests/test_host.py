"""Host-side tests of libtnstem (no GPU): the C interface loads and exports
every declared symbol, the planner's schemes are valid contraction trees whose
value (computed by the oracle) equals the state-vector amplitudes, reported
costs equal the oracle's tc/cw, and bad input is rejected with a status."""

import math
import os
import re

import numpy as np
import pytest

import oracle
import paper_2005_06787_gb300 as P
from synthetic.circuits import (CONFIGS, config_circuit, grid_layout, random_bits,
                                random_circuit)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    P.build()
    P.load()


def test_library_exports_every_header_symbol():
    hdr = open(os.path.join(ROOT, "include", "tnstem.h")).read()
    declared = set(re.findall(r"\b(tn_[a-z0-9_]+)\s*\(", hdr))
    assert declared, "no declarations parsed"
    lib = P.load()
    for name in sorted(declared):
        assert hasattr(lib, name), f"libtnstem.so lacks {name}"
    assert set(P.EXPORTED) <= declared


def test_set_prefix_rejects_bad_bits():
    c = random_circuit(grid_layout(2, 3), 4, 9)
    net = P.tn_build_network(c, [0], [0, 1, 0, 1, 1])
    with pytest.raises(P.TnError):
        P.tn_set_prefix(net, [0, 1, 2, 1, 1])
    with pytest.raises(ValueError):
        P.tn_set_prefix(net, [0, 1])
    P.tn_set_prefix(net, [1, 1, 0, 0, 1])
    plan = P.tn_plan_create(net, cw_limit=6, restarts=1)
    assert P.tn_plan_info(plan)["cw"] <= 6
    P.tn_destroy_plan(plan)
    P.tn_destroy_network(net)


def _net(c, oq, seed):
    cb = list(random_bits(c.n_qubits - len(oq), seed))
    return P.tn_build_network(c, oq, cb), cb


def _oracle_edges(net):
    _, _, q, s = net.info()
    return [(int(a), int(b)) for a, b in zip(q, s)]


@pytest.mark.parametrize("rows,cols,m,cw,n_open", [(3, 4, 8, 7, 3), (3, 3, 6, 5, 2),
                                                    (2, 4, 5, 4, 0), (4, 4, 8, 9, 4)])
def test_planned_scheme_value_equals_statevector(rows, cols, m, cw, n_open):
    c = random_circuit(grid_layout(rows, cols), m, rows * 100 + m)
    oq = list(range(n_open))
    net, cb = _net(c, oq, 17)
    plan = P.tn_plan_create(net, cw_limit=cw, restarts=4)
    info = P.tn_plan_info(plan)
    assert info["cw"] <= cw
    order, sl = P.tn_plan_export(plan)
    edges = _oracle_edges(net)
    sliced = [edges[e] for e in sl]
    onet = oracle.build_network(c, oq, cb)
    tot = oracle.contract_sliced_sum(onet, sliced, [tuple(x) for x in order])
    ref = oracle.sv_amplitudes(c, oq, cb)
    np.testing.assert_allclose(tot.reshape(-1), ref, atol=1e-13)
    tc, ocw = oracle.tree_cost(onet.edges, onet.open_edges, [tuple(x) for x in order], sliced)
    assert ocw == info["cw"]
    assert math.log2(tc) == pytest.approx(info["log2_tc"], abs=1e-9)


@pytest.mark.parametrize("rows,cols,m,cw,n_open,joins", [(3, 4, 10, 8, 2, True), (3, 3, 6, 5, 2, False)])
def test_per_branch_merges_keep_the_value_and_lower_the_predicted_time(rows, cols, m, cw, n_open, joins):
    # merge_group -1: branch merges chosen one by one along the stem by the
    # plain FLOP-and-memory model; the merged scheme (merged branches are
    # subtrees of the exported order) still equals the state vector, and its
    # tc/cw are the oracle's for that order
    c = random_circuit(grid_layout(rows, cols), m, rows * 100 + m)
    oq = list(range(n_open))
    net, cb = _net(c, oq, 17)
    plan = P.tn_plan_create(net, cw_limit=cw, restarts=4, merge_group=-1)
    info = P.tn_plan_info(plan)
    base = P.tn_plan_info(P.tn_plan_create(net, cw_limit=cw, restarts=4))
    assert info["cw"] <= cw
    # the 3 x 4 circuit gets at least one merge, the 3 x 3 one none
    assert (info["n_branches"] < base["n_branches"]) == joins
    assert info["log2_tc"] <= base["log2_tc"] + 1e-9
    order, sl = P.tn_plan_export(plan)
    edges = _oracle_edges(net)
    sliced = [edges[e] for e in sl]
    onet = oracle.build_network(c, oq, cb)
    tot = oracle.contract_sliced_sum(onet, sliced, [tuple(x) for x in order])
    np.testing.assert_allclose(tot.reshape(-1), oracle.sv_amplitudes(c, oq, cb), atol=1e-13)
    tc, ocw = oracle.tree_cost(onet.edges, onet.open_edges, [tuple(x) for x in order], sliced)
    assert ocw == info["cw"]
    assert math.log2(tc) == pytest.approx(info["log2_tc"], abs=1e-9)


def test_per_branch_merges_on_the_12_cycle_workload():
    # the plain model joins only branches whose merge it predicts faster:
    # far fewer than the uniform runs of merge_group 3, never more stem cost
    name = "diag53_m12"
    cfg = CONFIGS[name]
    c = config_circuit(name)
    oq = c.layout.open_qubits(cfg["n_open"])
    net, _ = _net(c, oq, cfg["bit_seed"])
    kw = dict(cw_limit=cfg["cw_limit"], restarts=1, anneal_iters=20000)
    i0 = P.tn_plan_info(P.tn_plan_create(net, **kw))
    i1 = P.tn_plan_info(P.tn_plan_create(net, merge_group=-1, **kw))
    i3 = P.tn_plan_info(P.tn_plan_create(net, merge_group=3, **kw))
    assert i3["n_branches"] < i1["n_branches"] <= i0["n_branches"]
    assert i1["log2_tc"] <= i0["log2_tc"] + 1e-9
    assert i1["n_gemm_steps"] < i3["n_gemm_steps"]


def test_given_order_round_trip():
    c = random_circuit(grid_layout(3, 4), 8, 3)
    net, _ = _net(c, [0, 1], 5)
    p1 = P.tn_plan_create(net, cw_limit=7, restarts=3)
    order, sl = P.tn_plan_export(p1)
    p2 = P.tn_plan_create(net, order=[tuple(x) for x in order], sliced_edges=list(sl))
    i1, i2 = P.tn_plan_info(p1), P.tn_plan_info(p2)
    assert i1["log2_tc"] == pytest.approx(i2["log2_tc"])
    assert i1["cw"] == i2["cw"]
    o2, s2 = P.tn_plan_export(p2)
    onet = oracle.build_network(c, [0, 1], list(random_bits(10, 5)))
    edges = _oracle_edges(net)
    v = oracle.contract_sliced_sum(onet, [edges[e] for e in s2], [tuple(x) for x in o2])
    np.testing.assert_allclose(v.reshape(-1), oracle.sv_amplitudes(c, [0, 1], list(random_bits(10, 5))),
                               atol=1e-13)


def test_plan_shapes_of_paper_workloads():
    # 53-qubit, 12-cycle stand-in: the stem fits the width limit by slicing
    name = "diag53_m12"
    cfg = CONFIGS[name]
    c = config_circuit(name)
    oq = c.layout.open_qubits(cfg["n_open"])
    net, _ = _net(c, oq, cfg["bit_seed"])
    plan = P.tn_plan_create(net, cw_limit=cfg["cw_limit"], restarts=2)
    info = P.tn_plan_info(plan)
    assert info["cw"] <= cfg["cw_limit"]
    assert info["n_sliced"] >= 1
    steps = P.tn_plan_steps(plan)
    assert len(steps) == info["n_stem_steps"]
    # every step is a (k, n) absorption that keeps ranks consistent
    for a, b in zip(steps, steps[1:]):
        assert a["r_out"] == b["r_in"]
    for s in steps:
        assert s["r_out"] == s["r_in"] - s["k"] + s["n"]
    assert steps[-1]["r_out"] == cfg["n_open"]
    # fused passes read and write each stem tensor once per group of steps
    assert info["stem_bytes_fused"] < info["stem_bytes_plain"] / 4


def test_annealing_planner_cost_on_12_cycles():
    # Supp. A.2 local optimisation + dynamic slicing: the annealed search must
    # keep the 53-qubit 12-cycle batch (64 amplitudes) within width 30 at a
    # total cost near the paper's 1.09e13 = 2^43.3 (Table 1, Sycamore), and
    # well below the greedy stem growth alone
    name = "diag53_m12"
    cfg = CONFIGS[name]
    c = config_circuit(name)
    oq = c.layout.open_qubits(cfg["n_open"])
    net, _ = _net(c, oq, cfg["bit_seed"])
    greedy = P.tn_plan_info(P.tn_plan_create(net, cw_limit=30, restarts=2, anneal_iters=-1))
    annealed = P.tn_plan_info(P.tn_plan_create(net, cw_limit=30, restarts=2, anneal_iters=300000))
    assert annealed["cw"] <= 30 and greedy["cw"] <= 30
    assert annealed["log2_tc"] <= 44.5, annealed["log2_tc"]
    assert annealed["log2_tc"] < greedy["log2_tc"] - 2.0


def test_two_phase_restarts_give_valid_schemes():
    # slice_restarts: every restart's stem is annealed unsliced, only the best
    # ones are sliced; the scheme must still meet the width and its value
    # must equal the state vector's
    c = random_circuit(grid_layout(3, 4), 8, 91)
    oq = [0, 7]
    net, cb = _net(c, oq, 23)
    plan = P.tn_plan_create(net, cw_limit=6, restarts=4, slice_restarts=1, anneal_iters=20000)
    info = P.tn_plan_info(plan)
    assert info["cw"] <= 6
    order, sl = P.tn_plan_export(plan)
    edges = _oracle_edges(net)
    onet = oracle.build_network(c, oq, cb)
    sliced = [edges[e] for e in sl]
    tot = oracle.contract_sliced_sum(onet, sliced, [tuple(x) for x in order])
    np.testing.assert_allclose(tot.reshape(-1), oracle.sv_amplitudes(c, oq, cb), atol=1e-13)
    tc, ocw = oracle.tree_cost(onet.edges, onet.open_edges, [tuple(x) for x in order], sliced)
    assert ocw == info["cw"]
    assert math.log2(tc) == pytest.approx(info["log2_tc"], abs=1e-9)


def _check_scheme_value(c, oq, cb, net, plan, limit):
    info = P.tn_plan_info(plan)
    assert info["cw"] <= limit
    order, sl = P.tn_plan_export(plan)
    edges = _oracle_edges(net)
    onet = oracle.build_network(c, oq, cb)
    sliced = [edges[e] for e in sl]
    tot = oracle.contract_sliced_sum(onet, sliced, [tuple(x) for x in order])
    np.testing.assert_allclose(tot.reshape(-1), oracle.sv_amplitudes(c, oq, cb), atol=1e-13)
    tc, ocw = oracle.tree_cost(onet.edges, onet.open_edges, [tuple(x) for x in order], sliced)
    assert ocw == info["cw"]
    assert math.log2(tc) == pytest.approx(info["log2_tc"], abs=1e-9)
    return order, sl, info


def test_start_cluster_and_stem_start_sweep():
    # start_cluster picks the first restart's stem seed; stem_starts grows
    # stems from spread start clusters on the host's threads. Every scheme
    # must meet the width and equal the state vector; the sweep must not
    # depend on scheduling (two runs agree).
    c = random_circuit(grid_layout(3, 4), 8, 91)
    oq = [0, 7]
    net, cb = _net(c, oq, 23)
    exports = set()
    for start in (0, 5, 11):
        plan = P.tn_plan_create(net, cw_limit=6, restarts=1, start_cluster=start, anneal_iters=5000)
        order, sl, _ = _check_scheme_value(c, oq, cb, net, plan, 6)
        exports.add((order.tobytes(), sl.tobytes()))
    assert len(exports) > 1  # different start clusters, different stems
    runs = []
    for _ in range(2):
        plan = P.tn_plan_create(net, cw_limit=6, stem_starts=12, anneal_iters=5000)
        order, sl, info = _check_scheme_value(c, oq, cb, net, plan, 6)
        runs.append((order.tobytes(), sl.tobytes(), info["log2_tc"]))
    assert runs[0] == runs[1]


def test_width_area_weight_gives_valid_schemes():
    # the unsliced anneal's excess-width term changes the stems it prefers;
    # the schemes must still meet the width and equal the state vector
    c = random_circuit(grid_layout(3, 4), 8, 91)
    oq = [0, 7]
    net, cb = _net(c, oq, 23)
    for w in (0.05, 0.5):
        plan = P.tn_plan_create(net, cw_limit=5, restarts=3, anneal_iters=5000, width_area_weight=w)
        _check_scheme_value(c, oq, cb, net, plan, 5)


def test_network_info_wire_segments():
    c = random_circuit(grid_layout(2, 2), 2, 9)
    net, _ = _net(c, [1], 3)
    nl, ne, q, s = net.info()
    onet = oracle.build_network(c, [1], list(random_bits(3, 3)))
    assert nl == len(onet.tensors)
    assert sorted(zip(q.tolist(), s.tolist())) == sorted(onet.all_edges())


def test_bad_inputs_are_rejected():
    c = random_circuit(grid_layout(2, 2), 2, 9)
    with pytest.raises(P.TnError) as e:
        P.tn_build_network(c, [7], [0, 0, 0])
    assert e.value.status == 1
    with pytest.raises(P.TnError):
        P.tn_build_network(c, [0, 0], [0, 0])
    with pytest.raises(P.TnError):
        P.tn_build_network(c, [0], [0, 2, 0])
    net, _ = _net(c, [0], 1)
    nl = net.info()[0]
    with pytest.raises(P.TnError):
        P.tn_plan_create(net, order=[(0, 0)] * (nl - 1))
    with pytest.raises(P.TnError):
        P.tn_plan_create(net, order=[(0, 1)])
    _, _, q, s = net.info()
    open_edge = [e for e in range(len(q)) if (q[e], s[e]) == (0, max(s[q == 0]))][0]
    good = P.tn_plan_create(net, cw_limit=8)
    order, _ = P.tn_plan_export(good)
    with pytest.raises(P.TnError):
        P.tn_plan_create(net, order=[tuple(x) for x in order], sliced_edges=[open_edge])
    out = np.zeros(4)
    with pytest.raises(P.TnError):  # not prepared
        P.tn_contract_stem(good, 0, 1, out)


def test_infeasible_width_reports_status():
    c = random_circuit(grid_layout(3, 3), 6, 4)
    net, _ = _net(c, list(range(9)), 0)  # all open: width >= 9 with no slicing allowed
    with pytest.raises(P.TnError) as e:
        P.tn_plan_create(net, cw_limit=6, max_sliced=1)
    assert e.value.status == 4


def test_hypernetwork_plan_cost_matches_oracle_and_is_cheaper():
    # Supp. A.1 cost on the multi-hypergraph (Sec. 3 hyperedges for the
    # diagonal part of fSim(pi/2, phi)): the library's greedy scheme, exported,
    # has the tc / cw the oracle computes for the oracle's own hypergraph of
    # the circuit, and contracting that network in that order gives the state
    # vector; it costs less than the graph network's stem plan
    import math
    from synthetic.circuits import config_circuit
    c = config_circuit("grid4x4_m8")
    oq, cb = [0, 1, 2], list(random_bits(13, 5))
    hnet = P.tn_build_hypernetwork(c, oq, cb)
    plan = P.tn_plan_create(hnet, cw_limit=30, restarts=8)
    info = P.tn_plan_info(plan)
    order, sl = P.tn_plan_export(plan)
    assert len(sl) == 0
    onet = oracle.build_hypernetwork(c, oq, cb)
    nl, ne, q, s = hnet.info()
    assert nl == len(onet.tensors)
    labels = sorted({e for el in onet.edges for e in el})
    assert sorted(zip(q.tolist(), s.tolist())) == labels
    tc, cw = oracle.tree_cost(onet.edges, onet.open_edges, [tuple(x) for x in order])
    assert math.isclose(math.log2(tc), info["log2_tc"], rel_tol=0, abs_tol=1e-9) and cw == info["cw"]
    val = oracle.contract(onet, [tuple(x) for x in order]).reshape(-1)
    np.testing.assert_allclose(val, oracle.sv_amplitudes(c, oq, cb), atol=1e-13)
    gplan = P.tn_plan_create(P.tn_build_network(c, oq, cb), cw_limit=30, restarts=2)
    assert info["log2_tc"] < P.tn_plan_info(gplan)["log2_tc"] - 2


def test_hypernetwork_needs_swap_times_diagonal_fsim_and_unsliced_plans():
    from synthetic.circuits import grid_layout, random_circuit
    c = random_circuit(grid_layout(2, 3), 3, 4, theta=1.0)
    with pytest.raises(P.TnError) as e:
        P.tn_build_hypernetwork(c, [0], list(random_bits(5, 1)))
    assert e.value.status == 6
    c = random_circuit(grid_layout(2, 3), 3, 4)
    hnet = P.tn_build_hypernetwork(c, [0], list(random_bits(5, 1)))
    with pytest.raises(P.TnError) as e:
        P.tn_plan_create(hnet, sliced_edges=[3], order=None)
    assert e.value.status in (1, 6)
    plan = P.tn_plan_create(hnet, cw_limit=30)
    with pytest.raises(P.TnError) as e:
        P.tn_plan_steps(plan)
    assert e.value.status == 6
