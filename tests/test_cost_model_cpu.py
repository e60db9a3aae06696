"""CPU tests of the learned cost model's oracle and of the plain cost model.

The FP64 oracle MLP (oracle/mlp.py) is pinned by the definition of the
derivative (central finite differences in FP64), by closed forms (a network
whose hidden weights vanish outputs b3 and has gradient 2 mean(b3 - t) in b3
only; a purely linear regime), and by a planted mistake (a dropped ReLU mask)
that the finite-difference pin catches. The per-launch features and the plain
FLOP-and-memory model are checked against the plan they describe.
"""

import numpy as np
import pytest

import oracle.mlp as om
import paper_2005_06787_gb300 as P
from synthetic.circuits import grid_layout, random_bits, random_circuit


def _rand(n_in=5, h1=7, h2=6, rows=11, seed=3):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(om.n_params(n_in, h1, h2)) * 0.5
    X = rng.standard_normal((rows, n_in))
    t = rng.standard_normal(rows)
    return p, X, t


def test_oracle_mlp_gradient_matches_finite_differences():
    n_in, h1, h2 = 5, 7, 6
    p, X, t = _rand(n_in, h1, h2)
    loss, g = om.loss_grad(p, X, t, n_in, h1, h2)
    eps = 1e-6
    for i in range(0, p.size, 3):
        q = p.copy()
        q[i] += eps
        lp, _ = om.loss_grad(q, X, t, n_in, h1, h2)
        q[i] -= 2 * eps
        lm, _ = om.loss_grad(q, X, t, n_in, h1, h2)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(fd)), i


def test_oracle_mlp_closed_forms():
    n_in, h1, h2 = 4, 3, 5
    p = np.zeros(om.n_params(n_in, h1, h2))
    p[-1] = 0.7  # b3
    X = np.arange(12.0).reshape(3, 4)
    t = np.array([1.0, 0.0, -1.0])
    y, _ = om.forward(p, X, n_in, h1, h2)
    assert np.allclose(y, 0.7)
    loss, g = om.loss_grad(p, X, t, n_in, h1, h2)
    assert loss == pytest.approx(np.mean((0.7 - t) ** 2))
    assert g[-1] == pytest.approx(2 * np.mean(0.7 - t))
    assert np.all(g[:-1] == 0)


def test_oracle_mlp_linear_regime():
    # positive inputs and weights keep every ReLU open: y = W3 W2 W1 x + ...
    n_in, h1, h2 = 3, 4, 2
    rng = np.random.default_rng(1)
    p = np.abs(rng.standard_normal(om.n_params(n_in, h1, h2)))
    X = np.abs(rng.standard_normal((5, n_in)))
    W1, b1, W2, b2, W3, b3 = om.unpack(p, n_in, h1, h2)
    ref = (X @ W1.T + b1) @ W2.T @ W3 + b2 @ W3 + b3[0]
    y, _ = om.forward(p, X, n_in, h1, h2)
    assert np.allclose(y, ref)


def test_planted_missing_relu_mask_fails_fd_pin():
    n_in, h1, h2 = 5, 7, 6
    p, X, t = _rand(n_in, h1, h2, seed=9)

    def bad_grad(p):
        W1, b1, W2, b2, W3, b3 = om.unpack(p, n_in, h1, h2)
        y, (Xd, z1, a1, z2, a2) = om.forward(p, X, n_in, h1, h2)
        dy = 2.0 * (y - t) / len(t)
        dz2 = np.outer(dy, W3)  # mask dropped
        return dz2.sum(axis=0)  # gradient of b2 without the ReLU mask

    _, g = om.loss_grad(p, X, t, n_in, h1, h2)
    off_b2 = h1 * n_in + h1 + h2 * h1
    assert np.abs(bad_grad(p) - g[off_b2:off_b2 + h2]).max() > 1e-6


@pytest.fixture(scope="module")
def built():
    P.build()
    P.load()


def test_features_match_plan(built):
    c = random_circuit(grid_layout(3, 4), 8, 3)
    net = P.tn_build_network(c, [0, 1, 2], list(random_bits(9, 5)))
    plan = P.tn_plan_create(net, cw_limit=7, restarts=2)
    info = P.tn_plan_info(plan)
    X, ms = P.tn_plan_features(plan, mode="fused")
    assert len(X) == info["n_passes_fused"] + info["n_gemm_steps"]
    assert np.all(ms > 0)
    steps = P.tn_plan_steps(plan)
    assert X[:, 6].sum() * 8 == pytest.approx(len(steps))      # every step in one launch
    Xp, msp = P.tn_plan_features(plan, mode="plain")
    assert len(Xp) == 2 * len(steps)
    assert Xp[0::2, 2].sum() == len(steps) and Xp[1::2, 1].sum() == len(steps)
    # the plain model charges the plain path more HBM time than the fused one
    assert msp.sum() > ms.sum()
