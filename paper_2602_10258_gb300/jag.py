"""Thin ctypes binding of the C ABI in ``include/jag.h``.

Argument marshalling only: every step of index build and search runs in the
CUDA library ``libjag.so``.  Device buffers and streams come from PyTorch
(``torch.Tensor.data_ptr()``, ``torch.cuda.Stream.cuda_stream``).  If the
library cannot be loaded, every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import numpy as np

from . import build_ext
from .datagen import FILTER_DTYPE

JAG_OK, JAG_EINVAL, JAG_ENOMEM, JAG_ECUDA, JAG_ETIMEOUT, JAG_EUNSUPPORTED = range(6)
JAG_F_NONE, JAG_F_LABEL, JAG_F_RANGE_I32, JAG_F_RANGE_F32, JAG_F_SUBSET, JAG_F_BOOL = range(6)
JAG_VEC_F32, JAG_VEC_BF16, JAG_VEC_FP8 = range(3)
JAG_SEARCH_SCAN_ALL = 0x1
JAG_POLICY_PLAIN, JAG_POLICY_LEARNED, JAG_POLICY_FORCED = range(3)
MLP_FEATURES, MLP_HIDDEN = 12, 64

_STATUS = {1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EUNSUPPORTED"}


class JagError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("jag status %s (%d): %s" % (_STATUS.get(status, "?"), status, msg))
        self.status = status


class BuildParams(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int64), ("x", C.c_void_p), ("attr_i32", C.c_void_p),
                ("attr_f32", C.c_void_p), ("attr_mask", C.c_void_p), ("dist_a", C.c_int32),
                ("R", C.c_int32), ("l_b", C.c_int32), ("alpha", C.c_float),
                ("n_thresholds", C.c_int32), ("threshold_pct", C.c_int32 * 4),
                ("sample_size", C.c_int32), ("seed", C.c_uint64), ("storage", C.c_int32),
                ("device", C.c_int32), ("graph", C.c_void_p), ("entry", C.c_int64),
                ("n_weights", C.c_int32), ("reserved", C.c_int32), ("weight_mult", C.c_double * 8)]


class SearchArgs(C.Structure):
    _fields_ = [("queries", C.c_void_p), ("filters", C.c_void_p), ("filter_aux", C.c_void_p),
                ("aux_bytes", C.c_int64), ("nq", C.c_int64), ("k", C.c_int32), ("beam", C.c_int32),
                ("out_ids", C.c_void_p), ("out_dist", C.c_void_p), ("stream", C.c_void_p),
                ("s0", C.c_int64), ("scan_cap", C.c_int64), ("counters", C.c_void_p),
                ("flags", C.c_int32), ("hash_bits", C.c_int32), ("ev_graph_begin", C.c_void_p),
                ("ev_graph_end", C.c_void_p), ("policy", C.c_void_p)]


class PolicyStruct(C.Structure):
    """Mirror of jag_policy."""
    _fields_ = [("mode", C.c_int32), ("h0", C.c_int32), ("w_bf16", C.c_void_p), ("b_f32", C.c_void_p),
                ("tau", C.c_float), ("stop_scale", C.c_float), ("n_ladder", C.c_int32),
                ("ladder", C.c_int32 * 16), ("forced", C.c_void_p), ("features", C.c_void_p),
                ("decisions", C.c_void_p)]


class ServeParams(C.Structure):
    """Mirror of jag_serve_params."""
    _fields_ = [("k", C.c_int32), ("beam", C.c_int32), ("s0", C.c_int64), ("scan_cap", C.c_int64),
                ("hash_bits", C.c_int32), ("max_requests", C.c_int32), ("max_queries", C.c_int64),
                ("arena_bytes", C.c_int64), ("lut_bytes", C.c_int64), ("ctas", C.c_int32),
                ("reserved", C.c_int32), ("idle_exit_s", C.c_double), ("policy", C.c_void_p)]


class ServeTiming(C.Structure):
    """Mirror of jag_serve_timing."""
    _fields_ = [("submit_s", C.c_double), ("done_s", C.c_double), ("device_s", C.c_double),
                ("status", C.c_uint32), ("reserved", C.c_uint32)]


class Info(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int64), ("R", C.c_int32), ("storage", C.c_int32),
                ("entry", C.c_int64), ("device_bytes", C.c_int64), ("build_seconds", C.c_double),
                ("n_thresholds", C.c_int32), ("dist_a", C.c_int32), ("weighted", C.c_int32),
                ("reserved", C.c_int32)]


EXPORTED = ["jag_build", "jag_search", "jag_query", "jag_search_host", "jag_search_noalloc", "jag_get_info",
            "jag_get_graph", "jag_get_thresholds", "jag_get_stored_rows", "jag_free", "jag_last_error",
            "jag_version", "jag_mlp_loss_grad", "jag_mlp_train", "jag_mlp_export", "jag_serve_start",
            "jag_serve_submit", "jag_serve_wait", "jag_serve_replay", "jag_serve_info", "jag_serve_stop"]

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return build_ext.LIB


def load(build_if_missing: bool = True):
    """Load libjag.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = build_ext.LIB
            if build_if_missing and build_ext.stale():
                build_ext.build()
            if not os.path.exists(path):
                raise RuntimeError("libjag.so is missing; build it with paper_2602_10258_gb300.build_ext")
            L = C.CDLL(path)
            P = C.c_void_p
            L.jag_build.argtypes = [C.POINTER(BuildParams), C.POINTER(P)]
            L.jag_build.restype = C.c_int
            L.jag_search.argtypes = [P, C.POINTER(SearchArgs)]
            L.jag_search.restype = C.c_int
            L.jag_query.argtypes = [P, P, P, P, C.c_int64, C.c_int64, C.c_int32, C.c_int32, P, P, P]
            L.jag_query.restype = C.c_int
            L.jag_search_host.argtypes = [P, C.POINTER(SearchArgs)]
            L.jag_search_host.restype = C.c_int
            L.jag_search_noalloc.argtypes = [P, C.POINTER(SearchArgs)]
            L.jag_search_noalloc.restype = C.c_int
            L.jag_get_info.argtypes = [P, C.POINTER(Info)]
            L.jag_get_info.restype = C.c_int
            L.jag_get_graph.argtypes = [P, P]
            L.jag_get_graph.restype = C.c_int
            L.jag_get_thresholds.argtypes = [P, P]
            L.jag_get_thresholds.restype = C.c_int
            L.jag_get_stored_rows.argtypes = [P, P, P, C.POINTER(C.c_int32)]
            L.jag_get_stored_rows.restype = C.c_int
            L.jag_free.argtypes = [P]
            L.jag_free.restype = None
            L.jag_last_error.argtypes = []
            L.jag_last_error.restype = C.c_char_p
            L.jag_version.argtypes = []
            L.jag_version.restype = C.c_char_p
            I32, I64, F = C.c_int32, C.c_int64, C.c_float
            L.jag_mlp_loss_grad.argtypes = [I32, P, P, P, P, I64, F, P, P, P]
            L.jag_mlp_loss_grad.restype = C.c_int
            L.jag_mlp_train.argtypes = [I32, P, P, P, C.POINTER(C.c_int64), P, P, P, I64, I32, I32, F, F, P, P]
            L.jag_mlp_train.restype = C.c_int
            L.jag_mlp_export.argtypes = [I32, P, P, P, P]
            L.jag_mlp_export.restype = C.c_int
            D = C.c_double
            L.jag_serve_start.argtypes = [P, P, C.POINTER(C.c_void_p)]
            L.jag_serve_start.restype = C.c_int
            L.jag_serve_submit.argtypes = [P, P, P, P, I64, I32, D, C.POINTER(C.c_uint64)]
            L.jag_serve_submit.restype = C.c_int
            L.jag_serve_wait.argtypes = [P, C.c_uint64, P, P, P, D]
            L.jag_serve_wait.restype = C.c_int
            L.jag_serve_replay.argtypes = [P, I64, P, P, P, P, P, P, I64, P, P, P, P, D]
            L.jag_serve_replay.restype = C.c_int
            L.jag_serve_info.argtypes = [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
            L.jag_serve_info.restype = C.c_int
            L.jag_serve_stop.argtypes = [P]
            L.jag_serve_stop.restype = C.c_int
            _lib = L
    return _lib


def _check(rc):
    if rc != JAG_OK:
        raise JagError(rc, load().jag_last_error().decode())


def _np_ptr(a):
    return None if a is None else a.ctypes.data


def jag_build(x, attr_i32=None, attr_f32=None, attr_mask=None, dist_a=JAG_F_RANGE_I32, R=32,
              l_b=64, alpha=1.2, thresholds=(100, 1, 0), sample_size=500, seed=0,
              storage=JAG_VEC_F32, device=0, graph=None, entry=0, weights=None):
    """Build (or upload) an index from host arrays; returns an opaque handle.
    weights: multipliers of h for a Weight-JAG build (None: Threshold-JAG)."""
    L = load()
    x = np.ascontiguousarray(x, np.float32)
    keep = [x]

    def arr(a, dt):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dt)
        keep.append(a)
        return a

    ai, af, am = arr(attr_i32, np.int32), arr(attr_f32, np.float32), arr(attr_mask, np.uint64)
    g = arr(graph, np.int32)
    p = BuildParams()
    p.n, p.d = x.shape
    p.x = _np_ptr(x)
    p.attr_i32, p.attr_f32, p.attr_mask = _np_ptr(ai), _np_ptr(af), _np_ptr(am)
    p.dist_a, p.R, p.l_b, p.alpha = int(dist_a), int(R), int(l_b), float(alpha)
    th = list(thresholds)
    p.n_thresholds = len(th)
    for i in range(min(4, len(th))):
        p.threshold_pct[i] = int(th[i])
    p.sample_size, p.seed, p.storage, p.device = int(sample_size), int(seed), int(storage), int(device)
    p.graph = _np_ptr(g)
    p.entry = int(entry)
    if weights is not None:
        p.n_weights = len(weights)
        for i, c in enumerate(weights):
            p.weight_mult[i] = float(c)
    h = C.c_void_p()
    _check(L.jag_build(C.byref(p), C.byref(h)))
    return h


def jag_free(h):
    if h:
        load().jag_free(h)


def jag_get_info(h) -> dict:
    i = Info()
    _check(load().jag_get_info(h, C.byref(i)))
    return {f: getattr(i, f) for f, _ in Info._fields_}


def jag_get_graph(h) -> np.ndarray:
    info = jag_get_info(h)
    out = np.empty((info["n"], info["R"]), np.int32)
    _check(load().jag_get_graph(h, _np_ptr(out)))
    return out


def jag_get_thresholds(h) -> np.ndarray:
    info = jag_get_info(h)
    out = np.empty((info["n"], info["n_thresholds"]), np.uint32)
    _check(load().jag_get_thresholds(h, _np_ptr(out)))
    return out


def jag_get_stored_rows(h):
    """(rows [n][row_bytes] uint8, scales [n] float32) of a BF16 / FP8 index."""
    info = jag_get_info(h)
    rb = C.c_int32(0)
    _check(load().jag_get_stored_rows(h, None, None, C.byref(rb)))
    rows = np.empty((info["n"], rb.value), np.uint8)
    sc = np.empty(info["n"], np.float32)
    _check(load().jag_get_stored_rows(h, _np_ptr(rows), _np_ptr(sc), C.byref(rb)))
    return rows, sc


def _args(nq, k, beam, s0, scan_cap, flags, hash_bits, aux_bytes):
    a = SearchArgs()
    a.nq, a.k, a.beam = int(nq), int(k), int(beam)
    a.s0, a.scan_cap, a.flags, a.hash_bits = int(s0), int(scan_cap), int(flags), int(hash_bits)
    a.aux_bytes = int(aux_bytes)
    return a


def jag_search(h, queries, filters, aux, k, beam, out_ids, out_dist, counters=None, stream=None,
               s0=-1, scan_cap=0, flags=0, hash_bits=0, ev_begin=None, ev_end=None, policy=None):
    """Device-pointer search: every tensor argument is a CUDA tensor (queries
    float32 [nq, d], filters uint8 [nq*16], aux uint8, out_ids int32 [nq, k],
    out_dist float32 [nq, k], counters int32 [nq, 4] or None).  Asynchronous
    on ``stream`` (a torch.cuda.Stream or None for the current stream)."""
    import torch
    L = load()
    nq = queries.shape[0]
    a = _args(nq, k, beam, s0, scan_cap, flags, hash_bits, 0 if aux is None else aux.numel())
    a.queries = queries.data_ptr()
    a.filters = filters.data_ptr()
    a.filter_aux = None if aux is None or aux.numel() == 0 else aux.data_ptr()
    a.out_ids, a.out_dist = out_ids.data_ptr(), out_dist.data_ptr()
    a.counters = None if counters is None else counters.data_ptr()
    st = stream if stream is not None else torch.cuda.current_stream(queries.device)
    a.stream = st.cuda_stream
    a.ev_graph_begin = None if ev_begin is None else ev_begin.cuda_event
    a.ev_graph_end = None if ev_end is None else ev_end.cuda_event
    ps = None if policy is None else policy.struct()
    a.policy = None if ps is None else C.addressof(ps)
    _check(L.jag_search(h, C.byref(a)))


def jag_query(h, queries, filters, aux, k, beam, out_ids, out_dist, stream=None):
    """The flat Query call (Algorithm 2) with the library's defaults: CUDA
    tensors as in jag_search; asynchronous on ``stream``."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream(queries.device)
    nb = 0 if aux is None else aux.numel()
    _check(load().jag_query(h, queries.data_ptr(), filters.data_ptr(), None if nb == 0 else aux.data_ptr(), nb,
                            queries.shape[0], int(k), int(beam), out_ids.data_ptr(), out_dist.data_ptr(),
                            st.cuda_stream))


def jag_search_noalloc(h, queries, filters, aux, k, beam, out_ids, out_dist, counters=None, stream=None,
                       s0=-1, scan_cap=0, flags=0, hash_bits=0, policy=None):
    """jag_search without any device allocation: the library's fixed scratch
    area is used instead (for callers that cannot allocate while searching).
    Calls share that area, so calls whose device work overlaps race; a call
    needing more than the area holds raises JagError (EINVAL)."""
    import torch
    L = load()
    nq = queries.shape[0]
    a = _args(nq, k, beam, s0, scan_cap, flags, hash_bits, 0 if aux is None else aux.numel())
    a.queries = queries.data_ptr()
    a.filters = filters.data_ptr()
    a.filter_aux = None if aux is None or aux.numel() == 0 else aux.data_ptr()
    a.out_ids, a.out_dist = out_ids.data_ptr(), out_dist.data_ptr()
    a.counters = None if counters is None else counters.data_ptr()
    st = stream if stream is not None else torch.cuda.current_stream(queries.device)
    a.stream = st.cuda_stream
    ps = None if policy is None else policy.struct()
    a.policy = None if ps is None else C.addressof(ps)
    _check(L.jag_search_noalloc(h, C.byref(a)))


def jag_search_host(h, queries, filters, aux, k, beam, counters=False, s0=-1, scan_cap=0, flags=0,
                    hash_bits=0, out_ids=None, out_dist=None, out_counters=None):
    """Host-buffer search: numpy (or pinned torch CPU) inputs and outputs; the
    call copies to and from the device and returns when answers are in host
    memory.  Returns (ids, dist, counters)."""
    L = load()
    q = np.ascontiguousarray(queries, np.float32) if isinstance(queries, np.ndarray) else queries
    nq = q.shape[0]
    f = np.ascontiguousarray(filters) if isinstance(filters, np.ndarray) else filters
    ax = aux
    if isinstance(aux, np.ndarray):
        ax = np.ascontiguousarray(aux, np.uint8)
    nb = 0 if ax is None else (ax.nbytes if isinstance(ax, np.ndarray) else ax.numel())

    def ptr(t):
        if t is None:
            return None
        return t.ctypes.data if isinstance(t, np.ndarray) else t.data_ptr()

    if out_ids is None:
        out_ids = np.empty((nq, k), np.int32)
    if out_dist is None:
        out_dist = np.empty((nq, k), np.float32)
    cnt = out_counters
    if counters and cnt is None:
        cnt = np.empty((nq, 4), np.int32)
    a = _args(nq, k, beam, s0, scan_cap, flags, hash_bits, nb)
    a.queries, a.filters, a.filter_aux = ptr(q), ptr(f), (ptr(ax) if nb else None)
    a.out_ids, a.out_dist, a.counters = ptr(out_ids), ptr(out_dist), ptr(cnt) if counters else None
    a.stream = None
    _check(L.jag_search_host(h, C.byref(a)))
    return out_ids, out_dist, (cnt if counters else None)


class Index:
    """Convenience owner of a built index (frees it on close/deletion)."""

    def __init__(self, x, attr_i32=None, attr_f32=None, attr_mask=None, dist_a=JAG_F_RANGE_I32, R=32,
                 l_b=64, alpha=1.2, thresholds=(100, 1, 0), sample_size=500, seed=0,
                 storage=JAG_VEC_F32, device=0, graph=None, entry=0, weights=None):
        self.h = jag_build(x, attr_i32, attr_f32, attr_mask, dist_a, R, l_b, alpha, thresholds,
                           sample_size, seed, storage, device, graph, entry, weights)
        self.d = int(np.asarray(x).shape[1])

    @classmethod
    def from_workload(cls, w, **kw):
        return cls(w.x, w.attr_i32, w.attr_f32, w.attr_mask, w.dist_a, **kw)

    def info(self):
        return jag_get_info(self.h)

    def graph(self):
        return jag_get_graph(self.h)

    def thresholds(self):
        return jag_get_thresholds(self.h)

    def stored_rows(self):
        return jag_get_stored_rows(self.h)

    def search(self, queries, filters, aux, k, beam, counters=False, stream=None, s0=-1, scan_cap=0,
               flags=0, hash_bits=0, ev_begin=None, ev_end=None, policy=None):
        """Search with device tensors; filters/aux may be numpy (copied to the
        device).  Returns CUDA tensors (ids, dist, counters or None)."""
        import torch
        dev = queries.device
        ft = filters_to_device(filters, dev)
        at = aux_to_device(aux, dev)
        nq = queries.shape[0]
        ids = torch.empty((nq, k), dtype=torch.int32, device=dev)
        dist = torch.empty((nq, k), dtype=torch.float32, device=dev)
        cnt = torch.empty((nq, 4), dtype=torch.int32, device=dev) if counters else None
        jag_search(self.h, queries, ft, at, k, beam, ids, dist, cnt, stream, s0, scan_cap, flags,
                   hash_bits, ev_begin, ev_end, policy)
        return ids, dist, cnt

    def search_host(self, queries, filters, aux, k, beam, **kw):
        return jag_search_host(self.h, queries, filters, aux, k, beam, **kw)

    def close(self):
        if getattr(self, "h", None):
            jag_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def filters_to_device(filters, device):
    import torch
    if isinstance(filters, torch.Tensor):
        return filters.to(device)
    f = np.ascontiguousarray(filters, dtype=FILTER_DTYPE)
    return torch.from_numpy(f.view(np.uint8).copy()).to(device)


def aux_to_device(aux, device):
    import torch
    if aux is None:
        return None
    if isinstance(aux, torch.Tensor):
        return aux.to(device)
    return torch.from_numpy(np.ascontiguousarray(aux, np.uint8).copy()).to(device)


# ---------------------------------------------------------------------------
# learned beam width / stop hop
# ---------------------------------------------------------------------------

LADDER = (16, 24, 32, 48, 64, 96, 128, 192, 256)


def mlp_n_params(nl):
    h, f = MLP_HIDDEN, MLP_FEATURES
    return h * f + h + h * h + h + (nl + 1) * h + nl + 1


class Policy:
    """Search policy passed to jag_search (``policy=``): device tensors for the
    BF16 weights / fp32 biases (LEARNED), the per-query (beam, stop) pairs
    (FORCED) and the optional feature / decision outputs."""

    def __init__(self, mode, h0=8, w_bf16=None, b_f32=None, tau=0.0, stop_scale=64.0, ladder=LADDER,
                 forced=None, features=None, decisions=None):
        self.mode, self.h0, self.tau, self.stop_scale = int(mode), int(h0), float(tau), float(stop_scale)
        self.ladder = tuple(int(v) for v in ladder)
        self.w_bf16, self.b_f32, self.forced = w_bf16, b_f32, forced
        self.features, self.decisions = features, decisions

    @staticmethod
    def _ptr(t):
        return None if t is None else t.data_ptr()

    def struct(self):
        p = PolicyStruct()
        p.mode, p.h0, p.tau, p.stop_scale = self.mode, self.h0, self.tau, self.stop_scale
        p.n_ladder = len(self.ladder)
        for i, v in enumerate(self.ladder):
            p.ladder[i] = v
        p.w_bf16, p.b_f32 = self._ptr(self.w_bf16), self._ptr(self.b_f32)
        p.forced, p.features, p.decisions = self._ptr(self.forced), self._ptr(self.features), self._ptr(self.decisions)
        self._s = p
        return p

    @classmethod
    def learned(cls, params, ladder=LADDER, h0=8, tau=0.0, stop_scale=64.0, stream=None, **kw):
        """Policy from a flat fp32 parameter tensor (CUDA): the weights are
        exported to BF16 by jag_mlp_export."""
        import torch
        nl = len(ladder)
        nw = MLP_HIDDEN * MLP_FEATURES + MLP_HIDDEN * MLP_HIDDEN + (nl + 1) * MLP_HIDDEN
        w = torch.empty(nw, dtype=torch.int16, device=params.device)
        b = torch.empty(2 * MLP_HIDDEN + nl + 1, dtype=torch.float32, device=params.device)
        mlp_export(nl, params, w, b, stream)
        return cls(JAG_POLICY_LEARNED, h0=h0, w_bf16=w, b_f32=b, tau=tau, stop_scale=stop_scale, ladder=ladder, **kw)


def _stream_ptr(stream, device):
    import torch
    st = stream if stream is not None else torch.cuda.current_stream(device)
    return st.cuda_stream


def mlp_loss_grad(nl, params, X, y, t, lam, stream=None):
    """(loss, grad) of the network over all rows (CUDA tensors)."""
    import torch
    g = torch.empty_like(params)
    loss = torch.empty(1, dtype=torch.float32, device=params.device)
    _check(load().jag_mlp_loss_grad(int(nl), params.data_ptr(), X.data_ptr(), y.data_ptr(), t.data_ptr(),
                                    int(X.shape[0]), float(lam), g.data_ptr(), loss.data_ptr(),
                                    _stream_ptr(stream, params.device)))
    return loss, g


class Trainer:
    """Adam state of one parameter tensor; ``run`` trains in place."""

    def __init__(self, nl, params):
        import torch
        self.nl, self.params = int(nl), params
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.step = C.c_int64(0)

    def run(self, X, y, t, epochs, batch, lr, lam, stream=None):
        trace = np.zeros(max(int(epochs), 1), np.float32)
        _check(load().jag_mlp_train(self.nl, self.params.data_ptr(), self.m.data_ptr(), self.v.data_ptr(),
                                    C.byref(self.step), X.data_ptr(), y.data_ptr(), t.data_ptr(), int(X.shape[0]),
                                    int(epochs), int(batch), float(lr), float(lam), trace.ctypes.data,
                                    _stream_ptr(stream, self.params.device)))
        return trace[:int(epochs)]


def mlp_export(nl, params, w_bf16, b_f32, stream=None):
    _check(load().jag_mlp_export(int(nl), params.data_ptr(), w_bf16.data_ptr(), b_f32.data_ptr(),
                                 _stream_ptr(stream, params.device)))


# ---------------------------------------------------------------------------
# serving: device-resident request loop
# ---------------------------------------------------------------------------

class Server:
    """A jag_server on an index: submit requests from host arrays, wait for
    their answers, or replay an arrival schedule.  Stop (or close) to drain
    and release it."""

    def __init__(self, index, k, beam, s0=-1, scan_cap=0, hash_bits=0, max_requests=0, max_queries=0,
                 arena_bytes=0, lut_bytes=0, ctas=0, idle_exit_s=0.0, policy=None):
        self.index = index
        self.k = int(k)
        self.d = index.d
        p = ServeParams()
        p.k, p.beam, p.s0, p.scan_cap, p.hash_bits = int(k), int(beam), int(s0), int(scan_cap), int(hash_bits)
        p.max_requests, p.max_queries, p.arena_bytes = int(max_requests), int(max_queries), int(arena_bytes)
        p.lut_bytes, p.ctas, p.idle_exit_s = int(lut_bytes), int(ctas), float(idle_exit_s)
        self._pol = None if policy is None else policy.struct()
        p.policy = None if self._pol is None else C.addressof(self._pol)
        self.h = C.c_void_p()
        _check(load().jag_serve_start(index.h, C.byref(p), C.byref(self.h)))
        self._nq = {}

    def submit(self, queries, filters, aux=None, timeout_s=10.0):
        q = np.ascontiguousarray(queries, np.float32)
        f = np.ascontiguousarray(filters)
        a = None if aux is None else np.ascontiguousarray(aux, np.uint8)
        t = C.c_uint64(0)
        _check(load().jag_serve_submit(self.h, q.ctypes.data, f.ctypes.data, None if a is None else a.ctypes.data,
                                       0 if a is None else a.nbytes, len(q), float(timeout_s), C.byref(t)))
        self._nq[t.value] = len(q)
        return t.value

    def wait(self, ticket, timeout_s=10.0):
        """(ids [nq][k], dist [nq][k], timing dict) of a submitted request."""
        nq = self._nq[ticket]
        ids = np.empty((nq, self.k), np.int32)
        dist = np.empty((nq, self.k), np.float32)
        tm = ServeTiming()
        _check(load().jag_serve_wait(self.h, C.c_uint64(ticket), ids.ctypes.data, dist.ctypes.data, C.byref(tm),
                                     float(timeout_s)))
        del self._nq[ticket]
        return ids, dist, {f: getattr(tm, f) for f, _ in ServeTiming._fields_}

    def replay(self, arrival_s, sizes, first, queries, filters, aux=None, timeout_s=120.0):
        """Open-loop replay: returns (ids, dist, latency_s [n_req], device_s [n_req])."""
        arr = np.ascontiguousarray(arrival_s, np.float64)
        sz = np.ascontiguousarray(sizes, np.int32)
        fi = np.ascontiguousarray(first, np.int64)
        q = np.ascontiguousarray(queries, np.float32)
        f = np.ascontiguousarray(filters)
        a = None if aux is None else np.ascontiguousarray(aux, np.uint8)
        ids = np.full((len(q), self.k), -1, np.int32)
        dist = np.full((len(q), self.k), np.inf, np.float32)
        lat = np.zeros(len(arr))
        dev = np.zeros(len(arr))
        _check(load().jag_serve_replay(self.h, len(arr), arr.ctypes.data, sz.ctypes.data, fi.ctypes.data,
                                       q.ctypes.data, f.ctypes.data, None if a is None else a.ctypes.data,
                                       0 if a is None else a.nbytes, ids.ctypes.data, dist.ctypes.data,
                                       lat.ctypes.data, dev.ctypes.data, float(timeout_s)))
        return ids, dist, lat, dev

    def info(self):
        la, qd = C.c_int64(0), C.c_int64(0)
        _check(load().jag_serve_info(self.h, C.byref(la), C.byref(qd)))
        return {"launches": la.value, "queries_done": qd.value}

    def stop(self):
        if self.h:
            _check(load().jag_serve_stop(self.h))
            self.h = None

    close = stop

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
