"""GPU tests of the learned step-time cost model.

The library's forward/backward kernels are checked against the FP64 oracle
MLP (oracle/mlp.py) on the same parameters and rows; training must fit a known
function; and the search scored by the trained network, with the plain
FLOP-and-memory model as fallback and check, must pick a plan at least as fast
(measured on the GPU) as the plain model's own pick, on the 53-qubit 12-cycle
workload with the network trained on that method's own step timings.
"""

import time

import numpy as np
import pytest

import oracle.mlp as om
import paper_2005_06787_gb300 as P
from paper_2005_06787_gb300 import learned

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    P.build()
    P.load()
    torch.cuda.set_device(0)


def test_mlp_gradient_matches_oracle():
    n_in, h1, h2 = P.N_FEATURES, 64, 64
    m = P.Mlp(n_in, h1, h2, seed=5)
    rng = np.random.default_rng(11)
    p = (rng.standard_normal(m.n_params()) * 0.2).astype(np.float32)
    m.set_params(p)
    X = rng.standard_normal((300, n_in)).astype(np.float32)
    t = rng.standard_normal(300).astype(np.float32)
    loss, g = m.loss_grad(X, t)
    ref_loss, ref_g = om.loss_grad(p.astype(np.float64), X, t, n_in, h1, h2)
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    assert np.linalg.norm(g - ref_g) / np.linalg.norm(ref_g) < 1e-5
    y = m.predict(X)
    ref_y, _ = om.forward(p.astype(np.float64), X, n_in, h1, h2)
    assert np.abs(y - ref_y).max() < 1e-5 * max(1.0, np.abs(ref_y).max())


def test_mlp_training_fits_known_function():
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, (2048, P.N_FEATURES)).astype(np.float32)
    t = (np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2] + 0.5 * np.abs(X[:, 3])).astype(np.float32)
    m = P.Mlp(P.N_FEATURES, 64, 64, seed=3)
    l0, _ = m.loss_grad(X, t)
    m.train(X, t, epochs=300, batch=256, lr=3e-3)
    l1, _ = m.loss_grad(X, t)
    assert l1 < 0.02 * l0, (l0, l1)


def _time_plan(plan, n_slices, stream):
    out = torch.zeros(2 * 64, dtype=torch.float64, device="cuda")
    P.tn_contract_stem(plan, 0, 1, out, stream=stream)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P.tn_contract_stem(plan, 0, n_slices, out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best / n_slices


def test_learned_search_gain_diag53_m12(capsys):
    from bench import plan_options, workload_inputs
    name = "diag53_m12"
    c, oq, cb = workload_inputs(name)
    net = P.tn_build_network(c, oq, cb)
    # the search's own planner effort is trimmed: this test is about the cost model
    base = dict(plan_options(name), anneal_iters=100000)
    stream = torch.cuda.current_stream()
    # training rows: the method's own timings over the knobs the search varies
    rows = []
    # (plans for training rows skip the annealing search: only their launch
    # shapes and timings matter)
    for plan in learned.plan_variants(net, dict(base, anneal_iters=-1), tiles=(10, 11, 12),
                                      steps=(2, 4, 6, 8), merges=(0, 3)):
        P.tn_plan_prepare(plan, stream=stream)
        rows.append((plan, "fp32", "fused"))
    X, y, flop = learned.gather(rows, repeats=2)
    del rows
    torch.cuda.empty_cache()
    mlp = learned.train_cost_model(X, y, epochs=600)
    pred = mlp.predict(X)
    corr = np.corrcoef(pred, y)[0, 1]
    assert corr > 0.9, corr
    t0 = time.perf_counter()
    plan_m, rep = P.tn_plan_search(net, mlp=mlp, n_seeds=2, **base)
    search_s = time.perf_counter() - t0
    plan_f, rep_f = P.tn_plan_search(net, mlp=None, n_seeds=2, **base)
    # compare whole-job time: per-slice time x slice count of each plan
    P.tn_plan_prepare(plan_m, stream=stream)
    ms_m = _time_plan(plan_m, 4, stream)
    tot_m = ms_m * 2.0 ** P.tn_plan_info(plan_m)["n_sliced"]
    del plan_m
    P.tn_plan_prepare(plan_f, stream=stream)
    ms_f = _time_plan(plan_f, 4, stream)
    tot_f = ms_f * 2.0 ** P.tn_plan_info(plan_f)["n_sliced"]
    with capsys.disabled():
        print(f"\nlearned search: {rep['n_candidates']} candidates, {rep['n_launch_rows']} launch "
              f"rows scored in {search_s:.1f} s; train rows {len(y)}, fit corr {corr:.3f}; "
              f"MLP pick {rep['mlp_pick']['tile_bits']}/{rep['mlp_pick']['max_pass_steps']}/"
              f"{rep['mlp_pick']['merge_group']} seed {rep['mlp_pick']['seed']} measured "
              f"{ms_m:.2f} ms/slice, {tot_m / 1e3:.1f} s all slices; plain-model pick "
              f"{rep_f['flop_pick']['tile_bits']}/{rep_f['flop_pick']['max_pass_steps']}/"
              f"{rep_f['flop_pick']['merge_group']} seed {rep_f['flop_pick']['seed']} measured "
              f"{ms_f:.2f} ms/slice, {tot_f / 1e3:.1f} s all slices; gain {tot_f / tot_m:.3f}x; "
              f"predicted {rep['mlp_pick_mlp_ms'] / 1e3:.1f} s (MLP) vs "
              f"{rep['mlp_pick_flop_ms'] / 1e3:.1f} s (plain model); used_mlp={rep['used_mlp']}")
    assert rep["n_candidates"] >= 60
    assert tot_m <= 1.05 * tot_f, (tot_m, tot_f)
    # held-out plans (another stem-growth seed): predicted vs measured batch time
    meas, p_mlp, p_flop = [], [], []
    held = dict(base, seed=base["seed"] + 104729, anneal_iters=-1)
    for tb, ms, mg in [(12, 8, 0), (12, 4, 0), (11, 8, 0), (10, 6, 0), (12, 2, 0), (12, 8, 3)]:
        plan = P.tn_plan_create(net, **dict(held, tile_bits=tb, max_pass_steps=ms, merge_group=mg))
        P.tn_plan_prepare(plan, stream=stream)
        Xh, flop_ms = P.tn_plan_features(plan)
        meas.append(_time_plan(plan, 2, stream))
        p_mlp.append(float(np.exp(mlp.predict(Xh).astype(np.float64)).sum()))
        p_flop.append(float(flop_ms.sum()))
        del plan
    meas, p_mlp, p_flop = map(np.asarray, (meas, p_mlp, p_flop))
    err_mlp = np.abs(np.log(p_mlp / meas)).mean()
    err_flop = np.abs(np.log(p_flop / meas)).mean()
    rank = lambda a: np.argsort(np.argsort(a))
    rho_mlp = np.corrcoef(rank(p_mlp), rank(meas))[0, 1]
    rho_flop = np.corrcoef(rank(p_flop), rank(meas))[0, 1]
    with capsys.disabled():
        print(f"held-out plans: measured ms/batch {np.round(meas, 2).tolist()}; MLP "
              f"{np.round(p_mlp, 2).tolist()} (mean |log err| {err_mlp:.3f}, rank corr "
              f"{rho_mlp:.2f}); plain model {np.round(p_flop, 2).tolist()} (mean |log err| "
              f"{err_flop:.3f}, rank corr {rho_flop:.2f})")
    assert err_mlp < err_flop


def _stored_scheme_plan(name, **kw):
    """Plan of a workload rebuilt from its stored order and sliced wire
    segments (tests/golden), with other launch options."""
    import json
    import os
    from bench import plan_options, workload_inputs
    gold = os.path.join(os.path.dirname(__file__), "golden")
    sch = json.load(open(os.path.join(gold, f"{name}_scheme.json")))
    c, oq, cb = workload_inputs(name)
    net = P.tn_build_network(c, oq, cb)
    _, _, q, s = net.info()
    eid = {(int(a), int(b)): e for e, (a, b) in enumerate(zip(q, s))}
    return P.tn_plan_create(net, order=[tuple(x) for x in sch["order"]],
                            sliced_edges=[eid[tuple(w)] for w in sch["sliced_wires"]],
                            **dict(plan_options(name), **kw))


def test_learned_pick_beats_plain_model_pick_diag53_m14(capsys):
    # The network is trained on launch timings of the 53-qubit 12-cycle
    # workload only; it then scores launch configurations (tile size x steps
    # per pass) of the held-out 14-cycle bench workload beside the plain
    # FLOP-and-memory model. Where the two picks differ, the learned pick must
    # run strictly faster on the GPU; where they agree the gain is 1.
    stream = torch.cuda.current_stream()
    rows = []
    for tb in (10, 11, 12):
        for ms in (2, 4, 6, 8):
            plan = _stored_scheme_plan("diag53_m12", tile_bits=tb, max_pass_steps=ms)
            P.tn_plan_prepare(plan, stream=stream)
            rows.append((plan, "fp32", "fused"))
    X, y, _ = learned.gather(rows, repeats=2)
    del rows
    torch.cuda.empty_cache()
    mlp = learned.train_cost_model(X, y, epochs=600)
    cands = [(tb, ms) for tb in (11, 12) for ms in (2, 4, 6, 8)]
    pm, pf = {}, {}
    for cand in cands:
        plan = _stored_scheme_plan("diag53_m14", tile_bits=cand[0], max_pass_steps=cand[1])
        Xc, flop_ms = P.tn_plan_features(plan)
        pm[cand] = float(np.exp(mlp.predict(Xc).astype(np.float64)).sum())
        pf[cand] = float(flop_ms.sum())
        del plan
    pick_m = min(cands, key=lambda k: pm[k])
    pick_f = min(cands, key=lambda k: pf[k])
    measured = {}
    for cand in {pick_m, pick_f}:
        plan = _stored_scheme_plan("diag53_m14", tile_bits=cand[0], max_pass_steps=cand[1])
        P.tn_plan_prepare(plan, stream=stream)
        measured[cand] = _time_plan(plan, 3, stream)
        del plan
        torch.cuda.empty_cache()
    gain = measured[pick_f] / measured[pick_m]
    with capsys.disabled():
        print(f"\ndiag53_m14 launch options (tile bits, steps per pass): learned pick {pick_m} "
              f"(predicted {pm[pick_m]:.1f} ms/slice, measured {measured[pick_m]:.1f}), plain-model "
              f"pick {pick_f} (predicted {pf[pick_f]:.1f} ms/slice, measured {measured[pick_f]:.1f}); "
              f"measured gain {gain:.3f}x; trained on {len(y)} launches of diag53_m12")
    if pick_m != pick_f:
        assert gain > 1.0, (pick_m, pick_f, measured)
    else:
        assert gain == 1.0
