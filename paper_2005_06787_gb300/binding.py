"""ctypes binding of libtnstem.so: the C entry points under the same names.

Argument marshalling only; every step of the stem runs in the library's CUDA
kernels. Loading fails loudly when the library has not been built.
PyTorch supplies device memory (tensors) and streams.
"""

from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libtnstem.so")

TN_OK = 0
STATUS_NAMES = {0: "TN_OK", 1: "TN_ERR_INVALID_ARG", 2: "TN_ERR_OOM", 3: "TN_ERR_CUDA",
                4: "TN_ERR_PLAN_INFEASIBLE", 5: "TN_ERR_TIMEOUT", 6: "TN_ERR_UNSUPPORTED"}

PREC = {"fp32": 0, "tf32x3": 1, "bf16x3": 2, "bf16x1": 3}
MODE = {"plain": 0, "fused": 1}

EXPORTED = [
    "tn_build_network", "tn_network_info", "tn_plan_create", "tn_plan_prepare", "tn_plan_info",
    "tn_plan_export", "tn_plan_steps", "tn_contract_stem", "tn_contract_stem_noalloc",
    "tn_plan_profile", "tn_plan_destroy",
    "tn_network_destroy", "tn_linear_xeb", "tn_permute", "tn_cgemm", "tn_last_error",
    "tn_version", "tn_plan_features", "tn_mlp_create", "tn_mlp_n_params", "tn_mlp_set_params",
    "tn_mlp_get_params", "tn_mlp_loss_grad", "tn_mlp_train", "tn_mlp_predict", "tn_mlp_destroy",
    "tn_plan_search", "tn_set_prefix", "tn_destroy_plan", "tn_destroy_network", "tn_frugal_sample",
    "tn_device_status", "tn_fp32_fma_peak", "tn_build_hypernetwork",
]
N_FEATURES = 16


class TnError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class tn_circuit(C.Structure):
    _fields_ = [("n_qubits", C.c_int32), ("n_cycles", C.c_int32),
                ("gates_1q", C.POINTER(C.c_int8)), ("pair_offsets", C.POINTER(C.c_int32)),
                ("pairs", C.POINTER(C.c_int32)), ("theta", C.c_double), ("phi", C.c_double)]


class tn_plan_opts(C.Structure):
    _fields_ = [("cw_limit", C.c_int32), ("min_sliced", C.c_int32), ("max_sliced", C.c_int32),
                ("restarts", C.c_int32), ("local_opt_iters", C.c_int32),
                ("branch_rank", C.c_int32), ("slice_batch", C.c_int32),
                ("tile_bits", C.c_int32), ("max_pass_steps", C.c_int32),
                ("gemm_min_kn", C.c_int32), ("merge_group", C.c_int32),
                ("merge_rank_cap", C.c_int32), ("anneal_iters", C.c_int32),
                ("slice_restarts", C.c_int32), ("seed", C.c_uint64),
                ("start_cluster", C.c_int32), ("stem_starts", C.c_int32),
                ("width_area_weight", C.c_double)]


class tn_plan_stats(C.Structure):
    _fields_ = [("log2_tc", C.c_double), ("stem_tc_per_slice", C.c_double),
                ("branch_tc", C.c_double), ("cw", C.c_int32), ("n_sliced", C.c_int32),
                ("n_stem_steps", C.c_int32), ("n_branches", C.c_int32),
                ("n_passes_fused", C.c_int32), ("n_gemm_steps", C.c_int32),
                ("n_open", C.c_int32), ("n_prefixes", C.c_int32), ("batch_items", C.c_int32),
                ("stem_bytes_plain", C.c_double), ("stem_bytes_fused", C.c_double),
                ("max_stem_elems", C.c_double), ("device_bytes", C.c_int64),
                ("n_passes_cbank", C.c_int32), ("pad_", C.c_int32)]


class tn_step_info(C.Structure):
    _fields_ = [("r_in", C.c_int32), ("r_out", C.c_int32), ("k", C.c_int32), ("n", C.c_int32),
                ("pass_", C.c_int32), ("gemm", C.c_int32), ("pair", C.c_int32)]


class tn_launch_record(C.Structure):
    _fields_ = [("kind", C.c_int32), ("index", C.c_int32), ("r_in", C.c_int32),
                ("r_out", C.c_int32), ("n_steps", C.c_int32), ("k", C.c_int32), ("n", C.c_int32),
                ("items", C.c_int32), ("ms", C.c_double), ("bytes", C.c_double),
                ("flops", C.c_double)]


class tn_search_opts(C.Structure):
    _fields_ = [("n_seeds", C.c_int32), ("fallback_factor", C.c_double)]


class tn_search_report(C.Structure):
    _fields_ = [("n_candidates", C.c_int32), ("n_launch_rows", C.c_int32), ("used_mlp", C.c_int32),
                ("chosen", tn_plan_opts), ("mlp_pick", tn_plan_opts), ("flop_pick", tn_plan_opts),
                ("mlp_pick_mlp_ms", C.c_double), ("mlp_pick_flop_ms", C.c_double),
                ("flop_pick_mlp_ms", C.c_double), ("flop_pick_flop_ms", C.c_double)]


_lib = None


def load():
    """Load libtnstem.so; raise if it was not built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libtnstem.so not built at {LIB_PATH}: run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
    L.tn_build_network.argtypes = [C.POINTER(tn_circuit), vp, i32, vp, C.POINTER(vp)]
    L.tn_build_hypernetwork.argtypes = [C.POINTER(tn_circuit), vp, i32, vp, C.POINTER(vp)]
    L.tn_network_info.argtypes = [vp, vp, vp, vp, vp]
    L.tn_plan_create.argtypes = [vp, vp, i32, vp, i32, C.POINTER(tn_plan_opts), C.POINTER(vp)]
    L.tn_plan_prepare.argtypes = [vp, vp, i32, vp]
    L.tn_plan_info.argtypes = [vp, C.POINTER(tn_plan_stats)]
    L.tn_plan_export.argtypes = [vp, vp, vp]
    L.tn_plan_steps.argtypes = [vp, vp, i32, vp]
    L.tn_contract_stem.argtypes = [vp, u64, u64, C.c_int, C.c_int, vp, vp, i32]
    L.tn_contract_stem_noalloc.argtypes = [vp, u64, u64, vp, vp, i32]
    L.tn_plan_destroy.argtypes = [vp]
    L.tn_plan_destroy.restype = None
    L.tn_network_destroy.argtypes = [vp]
    L.tn_destroy_plan.argtypes = [vp]
    L.tn_destroy_plan.restype = None
    L.tn_destroy_network.argtypes = [vp]
    L.tn_destroy_network.restype = None
    L.tn_set_prefix.argtypes = [vp, vp]
    L.tn_network_destroy.restype = None
    L.tn_plan_profile.argtypes = [vp, u64, C.c_int, C.c_int, vp, vp, i32, vp]
    L.tn_linear_xeb.argtypes = [vp, i64, i32, vp, C.POINTER(C.c_double)]
    L.tn_frugal_sample.argtypes = [vp, vp, vp, i64, i32, i32, C.c_double, vp, vp, vp, vp]
    L.tn_device_status.argtypes = []
    L.tn_fp32_fma_peak.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(i32)]
    L.tn_permute.argtypes = [vp, vp, i32, vp, vp]
    L.tn_cgemm.argtypes = [vp, vp, vp, i64, i64, i64, i64, i64, i64, i64, C.c_int, vp]
    L.tn_plan_features.argtypes = [vp, C.c_int, C.c_int, vp, vp, i32, vp]
    L.tn_mlp_create.argtypes = [i32, i32, i32, u64, C.POINTER(vp)]
    L.tn_mlp_n_params.argtypes = [vp, C.POINTER(i64)]
    L.tn_mlp_set_params.argtypes = [vp, vp, i64]
    L.tn_mlp_get_params.argtypes = [vp, vp, i64]
    L.tn_mlp_loss_grad.argtypes = [vp, vp, vp, i32, C.POINTER(C.c_double), vp]
    L.tn_mlp_train.argtypes = [vp, vp, vp, i32, i32, i32, C.c_float, u64, C.POINTER(C.c_double)]
    L.tn_mlp_predict.argtypes = [vp, vp, i32, vp]
    L.tn_mlp_destroy.argtypes = [vp]
    L.tn_mlp_destroy.restype = None
    L.tn_plan_search.argtypes = [vp, C.POINTER(tn_plan_opts), C.POINTER(tn_search_opts), vp, C.c_int,
                                 C.POINTER(vp), C.POINTER(tn_search_report)]
    L.tn_last_error.restype = C.c_char_p
    L.tn_last_error.argtypes = []
    L.tn_version.restype = C.c_char_p
    L.tn_version.argtypes = []
    for name in EXPORTED:
        if name not in ("tn_plan_destroy", "tn_network_destroy", "tn_last_error", "tn_version",
                        "tn_mlp_destroy", "tn_destroy_plan", "tn_destroy_network"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(status: int):
    if status != TN_OK:
        raise TnError(status, load().tn_last_error().decode())


def _ptr(a) -> int:
    """Address of a torch tensor or numpy array (None -> 0)."""
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _stream(stream) -> int:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# --------------------------------------------------------------------- network

class Network:
    def __init__(self, handle, n_open: int, n_closed: int, keep):
        self.handle = handle
        self.n_open = n_open
        self.n_closed = n_closed
        self._keep = keep

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tn_network_destroy(self.handle)
            self.handle = None

    def info(self) -> Tuple[int, int, np.ndarray, np.ndarray]:
        L = load()
        nl, ne = C.c_int32(), C.c_int32()
        _check(L.tn_network_info(self.handle, C.byref(nl), C.byref(ne), None, None))
        q = np.zeros(ne.value, dtype=np.int32)
        s = np.zeros(ne.value, dtype=np.int32)
        _check(L.tn_network_info(self.handle, None, None, q.ctypes.data, s.ctypes.data))
        return nl.value, ne.value, q, s


def tn_build_network(circuit, open_qubits: Sequence[int], closed_bits: Sequence[int],
                     hyper: bool = False) -> Network:
    """The circuit's network; hyper=True: tn_build_hypernetwork (diagonal
    parts of fSim(pi/2, phi) on hyperedges)."""
    L = load()
    g, offs, pairs = circuit.flat()
    g = np.ascontiguousarray(g.reshape(-1), dtype=np.int8)
    c = tn_circuit(circuit.n_qubits, circuit.n_cycles,
                   g.ctypes.data_as(C.POINTER(C.c_int8)),
                   offs.ctypes.data_as(C.POINTER(C.c_int32)),
                   pairs.ctypes.data_as(C.POINTER(C.c_int32)), circuit.theta, circuit.phi)
    oq = np.asarray(list(open_qubits) or [0], dtype=np.int32)
    cb = np.asarray(list(closed_bits) or [0], dtype=np.uint8)
    h = C.c_void_p()
    build = L.tn_build_hypernetwork if hyper else L.tn_build_network
    _check(build(C.byref(c), oq.ctypes.data, len(open_qubits), cb.ctypes.data, C.byref(h)))
    return Network(h, len(open_qubits), circuit.n_qubits - len(open_qubits), (g, offs, pairs))


def tn_build_hypernetwork(circuit, open_qubits: Sequence[int], closed_bits: Sequence[int]) -> Network:
    return tn_build_network(circuit, open_qubits, closed_bits, hyper=True)


def tn_set_prefix(net: Network, closed_bits: Sequence[int]) -> None:
    """Re-value the network's closed-qubit projectors with a new prefix."""
    L = load()
    cb = np.asarray(list(closed_bits), dtype=np.uint8)
    if cb.size != net.n_closed:
        raise ValueError(f"expected {net.n_closed} closed bits, got {cb.size}")
    cb = np.ascontiguousarray(cb if cb.size else np.zeros(1, np.uint8))
    _check(L.tn_set_prefix(net.handle, cb.ctypes.data))


# ------------------------------------------------------------------------ plan

def make_opts(**kw) -> tn_plan_opts:
    o = tn_plan_opts()
    defaults = dict(cw_limit=30, min_sliced=0, max_sliced=40, restarts=8, local_opt_iters=4,
                    branch_rank=4, slice_batch=0, tile_bits=0, max_pass_steps=0, gemm_min_kn=0,
                    merge_group=0, merge_rank_cap=0, anneal_iters=0, slice_restarts=0, seed=0x5EED,
                    start_cluster=0, stem_starts=0, width_area_weight=0.0)
    defaults.update(kw)
    for k, v in defaults.items():
        setattr(o, k, float(v) if k == "width_area_weight" else int(v))
    return o


class Plan:
    def __init__(self, handle, net: Network):
        self.handle = handle
        self.net = net

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tn_plan_destroy(self.handle)
            self.handle = None

    def info(self) -> dict:
        return tn_plan_info(self)


def tn_plan_create(net: Network, order: Optional[Sequence[Tuple[int, int]]] = None,
                   sliced_edges: Optional[Sequence[int]] = None, **opts) -> Plan:
    L = load()
    o = make_opts(**opts)
    ordp, n_pairs = None, 0
    if order is not None:
        ordp = np.ascontiguousarray(np.asarray(order, dtype=np.int32).reshape(-1))
        n_pairs = len(order)
    slp, nsl = None, 0
    if sliced_edges is not None and len(sliced_edges):
        slp = np.ascontiguousarray(np.asarray(sliced_edges, dtype=np.int32))
        nsl = len(sliced_edges)
    h = C.c_void_p()
    _check(L.tn_plan_create(net.handle, _ptr(ordp) or None, n_pairs, _ptr(slp) or None, nsl,
                            C.byref(o), C.byref(h)))
    return Plan(h, net)


def tn_destroy_plan(plan: Plan) -> None:
    """Free a plan now (otherwise it is freed when garbage-collected)."""
    if plan.handle:
        load().tn_destroy_plan(plan.handle)
        plan.handle = None


def tn_destroy_network(net: Network) -> None:
    """Free a network now (plans made from it hold their own copy)."""
    if net.handle:
        load().tn_destroy_network(net.handle)
        net.handle = None


def tn_plan_prepare(plan: Plan, prefixes: Optional[np.ndarray] = None, stream=None):
    L = load()
    if prefixes is None:
        _check(L.tn_plan_prepare(plan.handle, None, 0, _stream(stream)))
        return
    pre = np.ascontiguousarray(np.asarray(prefixes, dtype=np.uint8))
    if pre.ndim == 1:
        pre = pre[None, :]
    _check(L.tn_plan_prepare(plan.handle, pre.ctypes.data, pre.shape[0], _stream(stream)))


def tn_plan_info(plan: Plan) -> dict:
    L = load()
    s = tn_plan_stats()
    _check(L.tn_plan_info(plan.handle, C.byref(s)))
    return {f: getattr(s, f) for f, _ in tn_plan_stats._fields_}


def tn_plan_export(plan: Plan) -> Tuple[np.ndarray, np.ndarray]:
    L = load()
    nl, _, _, _ = plan.net.info()
    info = tn_plan_info(plan)
    order = np.zeros(2 * (nl - 1), dtype=np.int32)
    sl = np.zeros(max(info["n_sliced"], 1), dtype=np.int32)
    _check(L.tn_plan_export(plan.handle, order.ctypes.data, sl.ctypes.data))
    return order.reshape(-1, 2), sl[:info["n_sliced"]]


def tn_plan_steps(plan: Plan):
    L = load()
    n = C.c_int32()
    _check(L.tn_plan_steps(plan.handle, None, 0, C.byref(n)))
    arr = (tn_step_info * max(n.value, 1))()
    w = C.c_int32()
    _check(L.tn_plan_steps(plan.handle, arr, n.value, C.byref(w)))
    return [dict(r_in=a.r_in, r_out=a.r_out, k=a.k, n=a.n, pass_=a.pass_, gemm=a.gemm, pair=a.pair)
            for a in arr[:w.value]]


def tn_contract_stem(plan: Plan, slice_begin: int, slice_end: int, out, prec: str = "fp32",
                     mode: str = "fused", stream=None, accumulate: bool = False):
    """out: float64 tensor/array of n_prefixes * 2^n_open * 2 (re, im)."""
    L = load()
    _check(L.tn_contract_stem(plan.handle, int(slice_begin), int(slice_end), PREC[prec],
                              MODE[mode], _stream(stream), _ptr(out), int(bool(accumulate))))
    return out


def tn_contract_stem_noalloc(plan: Plan, slice_begin: int, slice_end: int, out, stream=None,
                             accumulate: bool = False):
    """Allocation-free fused contraction; out must be a CUDA float64 tensor."""
    L = load()
    _check(L.tn_contract_stem_noalloc(plan.handle, int(slice_begin), int(slice_end),
                                      _stream(stream), _ptr(out), int(bool(accumulate))))
    return out


def tn_plan_profile(plan: Plan, slice_begin: int = 0, prec: str = "fp32", mode: str = "fused",
                    stream=None):
    """Per-launch CUDA-event timings of one batch (list of dicts)."""
    L = load()
    n = C.c_int32()
    arr = (tn_launch_record * 4096)()
    _check(L.tn_plan_profile(plan.handle, int(slice_begin), PREC[prec], MODE[mode], _stream(stream),
                             arr, 4096, C.byref(n)))
    return [{f: getattr(a, f) for f, _ in tn_launch_record._fields_} for a in arr[:n.value]]


def tn_linear_xeb(amps_dev, n_qubits: int, stream=None) -> float:
    L = load()
    out = C.c_double()
    count = amps_dev.numel() // 2
    _check(L.tn_linear_xeb(_ptr(amps_dev), count, n_qubits, _stream(stream), C.byref(out)))
    return out.value


def tn_frugal_sample(amps_dev, u_dev, key_dev, n_batches: int, batch_size: int, n_qubits: int,
                     M: float, index_dev, accepted_dev, picked_dev, stream=None):
    """Frugal rejection sampling of n_batches amplitude batches (device
    buffers: FP64 complex amplitudes and uniforms u, key of n_batches x
    batch_size; outputs int32 index and accepted count per batch and the
    sampled FP64 complex amplitude)."""
    L = load()
    _check(L.tn_frugal_sample(_ptr(amps_dev), _ptr(u_dev), _ptr(key_dev), n_batches, batch_size,
                              n_qubits, float(M), _stream(stream), _ptr(index_dev),
                              _ptr(accepted_dev), _ptr(picked_dev)))


def tn_device_status() -> None:
    """Raise TnError(TN_ERR_TIMEOUT) if a bounded device-side wait gave up."""
    _check(load().tn_device_status())


def tn_fp32_fma_peak(stream=None) -> Tuple[float, int]:
    """Measured FP32 FMA rate of the current GPU (TFLOP/s) and its SM count."""
    L = load()
    tf = C.c_double()
    sms = C.c_int32()
    _check(L.tn_fp32_fma_peak(_stream(stream), C.byref(tf), C.byref(sms)))
    return float(tf.value), int(sms.value)


def tn_permute(inp, out, rank: int, perm: Sequence[int], stream=None):
    L = load()
    p = np.ascontiguousarray(np.asarray(perm, dtype=np.int32))
    _check(L.tn_permute(_ptr(inp), _ptr(out), rank, p.ctypes.data, _stream(stream)))
    return out


def tn_cgemm(A, B, Cm, M: int, K: int, N: int, batch: int = 1, strideA: int = 0,
             strideB: int = 0, strideC: int = 0, prec: str = "fp32", stream=None):
    L = load()
    _check(L.tn_cgemm(_ptr(A), _ptr(B), _ptr(Cm), M, K, N, batch, strideA, strideB, strideC,
                      PREC[prec], _stream(stream)))
    return Cm


def tn_version() -> str:
    return load().tn_version().decode()


# ------------------------------------------------------------ cost models

def tn_plan_features(plan: Plan, prec: str = "fp32", mode: str = "fused"):
    """Per-launch features [rows, 16] and plain-model times [rows] (ms)."""
    L = load()
    n = C.c_int32()
    _check(L.tn_plan_features(plan.handle, PREC[prec], MODE[mode], None, None, 0, C.byref(n)))
    X = np.zeros((max(n.value, 1), N_FEATURES), dtype=np.float32)
    ms = np.zeros(max(n.value, 1), dtype=np.float64)
    w = C.c_int32()
    _check(L.tn_plan_features(plan.handle, PREC[prec], MODE[mode], X.ctypes.data, ms.ctypes.data,
                              n.value, C.byref(w)))
    return X[:w.value], ms[:w.value]


class Mlp:
    """Handle of the library's GPU MLP cost model."""

    def __init__(self, n_in: int = N_FEATURES, h1: int = 64, h2: int = 64, seed: int = 1):
        L = load()
        h = C.c_void_p()
        _check(L.tn_mlp_create(n_in, h1, h2, seed, C.byref(h)))
        self.handle = h
        self.n_in, self.h1, self.h2 = n_in, h1, h2

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tn_mlp_destroy(self.handle)
            self.handle = None

    def n_params(self) -> int:
        n = C.c_int64()
        _check(load().tn_mlp_n_params(self.handle, C.byref(n)))
        return n.value

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.n_params(), dtype=np.float32)
        _check(load().tn_mlp_get_params(self.handle, p.ctypes.data, p.size))
        return p

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(load().tn_mlp_set_params(self.handle, p.ctypes.data, p.size))

    def loss_grad(self, X, t):
        X = np.ascontiguousarray(X, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        loss = C.c_double()
        g = np.zeros(self.n_params(), dtype=np.float32)
        _check(load().tn_mlp_loss_grad(self.handle, X.ctypes.data, t.ctypes.data, len(t),
                                       C.byref(loss), g.ctypes.data))
        return loss.value, g

    def train(self, X, t, epochs=200, batch=256, lr=1e-3, seed=1) -> float:
        X = np.ascontiguousarray(X, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        loss = C.c_double()
        _check(load().tn_mlp_train(self.handle, X.ctypes.data, t.ctypes.data, len(t), epochs, batch,
                                   lr, seed, C.byref(loss)))
        return loss.value

    def predict(self, X) -> np.ndarray:
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.zeros(len(X), dtype=np.float32)
        _check(load().tn_mlp_predict(self.handle, X.ctypes.data, len(X), y.ctypes.data))
        return y


def tn_plan_search(net: Network, mlp: Optional[Mlp] = None, prec: str = "fp32", n_seeds: int = 3,
                   fallback_factor: float = 4.0, **opts):
    """Search candidate plans; returns (plan, report dict)."""
    L = load()
    o = make_opts(**opts)
    so = tn_search_opts(n_seeds, fallback_factor)
    rep = tn_search_report()
    h = C.c_void_p()
    _check(L.tn_plan_search(net.handle, C.byref(o), C.byref(so), mlp.handle if mlp else None,
                            PREC[prec], C.byref(h), C.byref(rep)))

    def od(x):
        return {f: getattr(x, f) for f, _ in tn_plan_opts._fields_}
    report = {"n_candidates": rep.n_candidates, "n_launch_rows": rep.n_launch_rows,
              "used_mlp": bool(rep.used_mlp), "chosen": od(rep.chosen), "mlp_pick": od(rep.mlp_pick),
              "flop_pick": od(rep.flop_pick), "mlp_pick_mlp_ms": rep.mlp_pick_mlp_ms,
              "mlp_pick_flop_ms": rep.mlp_pick_flop_ms, "flop_pick_mlp_ms": rep.flop_pick_mlp_ms,
              "flop_pick_flop_ms": rep.flop_pick_flop_ms}
    return Plan(h, net), report
