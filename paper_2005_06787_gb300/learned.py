"""Training data and training loop of the learned step-time cost model.

Rows come from the method's own stem runs: for a prepared plan, the
per-launch features of one batch (``tn_plan_features``) are paired, in launch
order, with the CUDA-event times of the same launches (``tn_plan_profile``).
The target is ln(ms). Training and inference run in the library's GPU MLP
kernels (``Mlp``); this module only gathers rows and calls them.
"""

from __future__ import annotations

from typing import Iterable, List, Optional, Sequence, Tuple

import numpy as np

from . import binding as B


def profile_rows(plan: B.Plan, prec: str = "fp32", mode: str = "fused", slice_begin: int = 0,
                 repeats: int = 2) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(features [rows, 16], ln measured ms [rows], plain-model ms [rows]) for
    one batch of a prepared plan; the measured time is the minimum over
    ``repeats`` profiled runs."""
    X, flop_ms = B.tn_plan_features(plan, prec=prec, mode=mode)
    best = None
    for _ in range(max(1, repeats)):
        recs = [r for r in B.tn_plan_profile(plan, slice_begin, prec=prec, mode=mode)
                if r["kind"] in (0, 1, 2)]
        if len(recs) != len(X):
            raise RuntimeError("profile records and features disagree on the launch count")
        ms = np.array([r["ms"] for r in recs])
        best = ms if best is None else np.minimum(best, ms)
    return X, np.log(np.maximum(best, 1e-4)).astype(np.float32), flop_ms


def gather(plans: Iterable[Tuple[B.Plan, str, str]], repeats: int = 2):
    """Stack rows of several (plan, precision, mode) runs."""
    xs, ys, fs = [], [], []
    for plan, prec, mode in plans:
        X, y, f = profile_rows(plan, prec, mode, repeats=repeats)
        xs.append(X)
        ys.append(y)
        fs.append(f)
    return np.concatenate(xs), np.concatenate(ys), np.concatenate(fs)


def train_cost_model(X: np.ndarray, y: np.ndarray, epochs: int = 400, lr: float = 3e-3,
                     batch: int = 128, seed: int = 7, mlp: Optional[B.Mlp] = None) -> B.Mlp:
    """Fit an MLP (16 -> 64 -> 64 -> 1) to ln(ms) on the GPU."""
    if mlp is None:
        mlp = B.Mlp(B.N_FEATURES, 64, 64, seed)
    mlp.train(X, y, epochs=epochs, batch=min(batch, len(y)), lr=lr, seed=seed)
    return mlp


def plan_variants(net: B.Network, base: dict, tiles: Sequence[int] = (10, 11, 12),
                  steps: Sequence[int] = (2, 4, 6, 8), merges: Sequence[int] = (0, 3)) -> List[B.Plan]:
    """Plans of one network that differ in the knobs the search varies."""
    out = []
    for mg in merges:
        for tb in tiles:
            for ms in steps:
                o = dict(base)
                o.update(tile_bits=tb, max_pass_steps=ms, merge_group=mg)
                try:
                    out.append(B.tn_plan_create(net, **o))
                except B.TnError:
                    pass
    return out
