"""Python handle on the plain C oracle (``jag_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  Nothing here imports the
CUDA package; arrays come from the seeded generators and are passed as plain
numpy buffers.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jag_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libjag_oracle.so")
_lock = threading.Lock()
_lib = None

K_NONE, K_LABEL, K_RANGE_I32, K_RANGE_F32, K_SUBSET, K_BOOL = range(6)

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-pthread", "-Wall", "-Wno-unused-function"]


def compile_lib(force: bool = False) -> str:
    """Compile the oracle with gcc (no CUDA, no shared headers)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


FMT_F32, FMT_BF16, FMT_FP8 = 0, 1, 2


class _Index(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int64), ("x", C.c_void_p),
                ("a_i32", C.c_void_p), ("a_f32", C.c_void_p), ("a_mask", C.c_void_p),
                ("dist_a", C.c_int32), ("R", C.c_int32), ("graph", C.c_void_p),
                ("entry", C.c_int64), ("fmt", C.c_int32), ("qbytes", C.c_int32),
                ("xq", C.c_void_p), ("qscale", C.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(compile_lib())
            P, I64, I32, F32, U64 = C.c_void_p, C.c_int64, C.c_int, C.c_float, C.c_uint64
            sig = {
                "orc_dist_canon": (F32, [P, P, I64]),
                "orc_dist_f64": (C.c_double, [P, P, I64]),
                "orc_bool_lut": (I32, [U64, P, P]),
                "orc_brute_force": (None, [P, P, P, P, I64, I32, P, P, P, P, I32]),
                "orc_query": (I32, [P, P, P, P, I64, I32, I32, I32, I64, I64, P, P, P, I32]),
                "orc_query_lists": (None, [P, P, P, P, I64, I32, P, P, P, P, I32]),
                "orc_medoid": (I64, [P, I64, I64]),
                "orc_sm64": (U64, [U64, U64]),
                "orc_thresholds": (None, [P, P, I32, I32, U64, P, I32]),
                "orc_build": (I32, [P, P, I32, I32, F32, I32]),
                "orc_build_weighted": (I32, [P, P, I32, I32, F32, I32]),
                "orc_joint_prune_weighted": (I32, [P, I64, P, P, I32, P, I32, F32, P]),
                "orc_weights": (None, [P, P, I32, I32, U64, P, P, I32]),
                "orc_dist_A_value": (F32, [P, I64, I64]),
                "orc_joint_prune": (I32, [P, I64, P, P, I32, P, I32, F32, P]),
                "orc_build_search": (I64, [P, I64, C.c_uint32, I32, P, P, I64]),
                "orc_dist_F_batch": (None, [P, P, P, P, I64, P]),
                "orc_g_batch": (None, [P, P, P, P, I64, P]),
                "orc_dist_canon_batch": (None, [P, P, I64, I64, P]),
                "orc_route": (I32, [P, P, P, I64, I64, P]),
                "orc_count_passing": (I64, [P, P, P]),
                "orc_dist_A": (C.c_uint32, [P, I64, I64]),
                "orc_capped": (C.c_uint32, [I32, C.c_uint32, C.c_uint32]),
                "orc_row_bytes": (I32, [I32, I64]),
                "orc_quantize": (None, [P, I64, I64, I32, P, P]),
                "orc_bf16_encode_batch": (None, [P, I64, P]),
                "orc_fp8_encode_batch": (None, [P, I64, P]),
                "orc_fp8_decode_batch": (None, [P, I64, P]),
                "orc_dist_canon_q_batch": (None, [P, P, P, I32, I64, I64, I64, P]),
                "orc_query_policy": (I32, [P, P, P, P, I64, I32, I32, I64, I64, P, P, P, P, I32]),
                "orc_mlp_infer_batch": (None, [P, P, I64, P]),
                "orc_policy_features": (None, [P, P, P, I32, I32, I64, I32, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def alpha2_of(alpha: float) -> float:
    """alpha^2 as the pruning test uses it: alpha is an fp32 parameter, its
    square is formed in double and rounded once to fp32."""
    a = float(np.float32(alpha))
    return float(np.float32(a * a))


class Index:
    """Base vectors, attributes and (optionally) a graph, as the oracle sees them."""

    def __init__(self, x, attr_i32=None, attr_f32=None, attr_mask=None, dist_a=K_RANGE_I32,
                 R=32, graph=None, entry=0, storage=FMT_F32):
        self.x = _c(x, np.float32)
        self.attr_i32 = _c(attr_i32, np.int32)
        self.attr_f32 = _c(attr_f32, np.float32)
        self.attr_mask = _c(attr_mask, np.uint64)
        n, d = self.x.shape
        self.R = int(R)
        self.graph = (np.full((n, self.R), -1, np.int32) if graph is None
                      else np.ascontiguousarray(graph, dtype=np.int32))
        self.xq, self.qscale, qb = None, None, 0
        if storage != FMT_F32:
            self.xq, self.qscale = quantize(self.x, storage)
            qb = self.xq.shape[1]
        self.s = _Index(n, d, _p(self.x), _p(self.attr_i32), _p(self.attr_f32),
                        _p(self.attr_mask), int(dist_a), self.R, _p(self.graph), int(entry),
                        int(storage), qb, _p(self.xq), _p(self.qscale))

    @classmethod
    def from_workload(cls, w, R=32, graph=None, entry=0, storage=FMT_F32):
        return cls(w.x, w.attr_i32, w.attr_f32, w.attr_mask, w.dist_a, R, graph, entry, storage)

    @property
    def n(self):
        return self.s.n

    @property
    def d(self):
        return self.s.d

    @property
    def entry(self):
        return self.s.entry

    @entry.setter
    def entry(self, v):
        self.s.entry = int(v)

    def ref(self):
        return C.byref(self.s)


def default_threads():
    return max(1, os.cpu_count() or 1)


def dist_canon(q, x):
    q = _c(q, np.float32)
    x = _c(x, np.float32)
    return float(lib().orc_dist_canon(_p(q), _p(x), q.shape[-1]))


def dist_canon_rows(q, x):
    q = _c(np.atleast_2d(q), np.float32)
    x = _c(np.atleast_2d(x), np.float32)
    out = np.empty(q.shape[0], np.float32)
    lib().orc_dist_canon_batch(_p(q), _p(x), q.shape[0], q.shape[1], _p(out))
    return out


def dist_f64(q, x):
    q = _c(q, np.float32)
    x = _c(x, np.float32)
    return float(lib().orc_dist_f64(_p(q), _p(x), q.shape[-1]))


def bool_lut(vars_mask: int, table_bytes: np.ndarray):
    m = bin(vars_mask).count("1")
    lut = np.empty(1 << m, np.uint8)
    tb = _c(table_bytes, np.uint8)
    sat = lib().orc_bool_lut(vars_mask, _p(tb), _p(lut))
    return lut, bool(sat)


def brute_force(ix: Index, q, filters, aux, k, with_f64=True, nthreads=None):
    q = _c(q, np.float32)
    nq = q.shape[0]
    f = np.ascontiguousarray(filters)
    aux = _c(aux, np.uint8)
    ids = np.empty((nq, k), np.int32)
    d32 = np.empty((nq, k), np.float32)
    d64 = np.empty((nq, k), np.float64) if with_f64 else None
    npass = np.empty(nq, np.int64)
    lib().orc_brute_force(ix.ref(), _p(q), _p(f), _p(aux), nq, k, _p(ids), _p(d32), _p(d64),
                          _p(npass), nthreads or default_threads())
    return ids, d32, d64, npass


def query(ix: Index, q, filters, aux, k, ls, literal=False, s0=0, scan_cap=32768, nthreads=None):
    """Query (Algorithm 2) for a batch; returns ids, dists, counters[nq,4] =
    (hops, first-seen neighbours, distance computations, routed to scan)."""
    q = _c(q, np.float32)
    nq = q.shape[0]
    f = np.ascontiguousarray(filters)
    aux = _c(aux, np.uint8)
    ids = np.empty((nq, k), np.int32)
    dist = np.empty((nq, k), np.float32)
    cnt = np.zeros((nq, 4), np.int64)
    rc = lib().orc_query(ix.ref(), _p(q), _p(f), _p(aux), nq, k, ls, int(literal), int(s0),
                         int(scan_cap), _p(ids), _p(dist), _p(cnt), nthreads or default_threads())
    if rc:
        raise ValueError("invalid query arguments")
    return ids, dist, cnt


def query_lists(ix: Index, q, filters, aux, ls, nthreads=None):
    q = _c(q, np.float32)
    nq = q.shape[0]
    f = np.ascontiguousarray(filters)
    aux = _c(aux, np.uint8)
    ids = np.empty((nq, ls), np.int32)
    k1 = np.empty((nq, ls), np.uint32)
    dist = np.empty((nq, ls), np.float32)
    ln = np.empty(nq, np.int32)
    lib().orc_query_lists(ix.ref(), _p(q), _p(f), _p(aux), nq, ls, _p(ids), _p(k1), _p(dist),
                          _p(ln), nthreads or default_threads())
    return ids, k1, dist, ln


def route(ix: Index, filt, aux, s0, scan_cap=32768):
    f = np.ascontiguousarray(np.atleast_1d(filt))
    aux = _c(aux, np.uint8)
    cnt = C.c_int64(0)
    r = lib().orc_route(ix.ref(), _p(f), _p(aux), int(s0), int(scan_cap), C.byref(cnt))
    return bool(r), int(cnt.value)


def count_passing(ix: Index, filt, aux):
    f = np.ascontiguousarray(np.atleast_1d(filt))
    aux = _c(aux, np.uint8)
    return int(lib().orc_count_passing(ix.ref(), _p(f), _p(aux)))


def medoid(x):
    x = _c(x, np.float32)
    return int(lib().orc_medoid(_p(x), x.shape[0], x.shape[1]))


def sm64(seed, ctr):
    return int(lib().orc_sm64(seed, ctr))


def thresholds(ix: Index, pct=(100, 1, 0), S=500, seed=0, nthreads=None):
    pct = np.asarray(pct, np.int32)
    out = np.empty((ix.n, len(pct)), np.uint32)
    lib().orc_thresholds(ix.ref(), _p(pct), len(pct), S, seed, _p(out), nthreads or default_threads())
    return out


def build(ix: Index, pct=(100, 1, 0), lb=64, alpha=1.2, S=500, seed=0, nthreads=None):
    """JAG build (Insert + JointRobustPrune over the batch schedule); fills
    ix.graph and ix.entry, returns the per-point thresholds."""
    ix.entry = medoid(ix.x)
    thr = thresholds(ix, pct, S, seed, nthreads)
    rc = lib().orc_build(ix.ref(), _p(thr), thr.shape[1], int(lb), alpha2_of(alpha),
                         nthreads or default_threads())
    if rc:
        raise RuntimeError("oracle build failed")
    return thr


def weights(ix: Index, mult=(0, 1, 10), S=500, seed=0, nthreads=None):
    """Weight-JAG weights: (w [n][len(mult)] float32 = fp32(mult_i * h_p),
    h [n] float64) with h_p = sigma / sigma_A over the threshold sample."""
    mult = np.asarray(mult, np.float64)
    out = np.empty((ix.n, len(mult)), np.float32)
    h = np.empty(ix.n, np.float64)
    lib().orc_weights(ix.ref(), _p(mult), len(mult), S, seed, _p(out), _p(h), nthreads or default_threads())
    return out, h


def build_weighted(ix: Index, mult=(0, 1, 10), lb=64, alpha=1.2, S=500, seed=0, nthreads=None):
    """Weight-JAG build; fills ix.graph and ix.entry, returns (weights, h)."""
    ix.entry = medoid(ix.x)
    w, h = weights(ix, mult, S, seed, nthreads)
    rc = lib().orc_build_weighted(ix.ref(), _p(w), w.shape[1], int(lb), alpha2_of(alpha),
                                  nthreads or default_threads())
    if rc:
        raise RuntimeError("oracle build failed")
    return w, h


def joint_prune_weighted(ix: Index, p, cand, dpc, W, alpha=1.2):
    cand = _c(cand, np.int32)
    dpc = _c(dpc, np.float32)
    W = _c(W, np.float32)
    out = np.empty(ix.R, np.int32)
    m = lib().orc_joint_prune_weighted(ix.ref(), int(p), _p(cand), _p(dpc), len(cand), _p(W), len(W),
                                       alpha2_of(alpha), _p(out))
    return out[:m]


def dist_A_value(ix: Index, i, j):
    return float(lib().orc_dist_A_value(ix.ref(), int(i), int(j)))


def joint_prune(ix: Index, p, cand, dpc, T, alpha=1.2):
    cand = _c(cand, np.int32)
    dpc = _c(dpc, np.float32)
    T = _c(T, np.uint32)
    out = np.empty(ix.R, np.int32)
    m = lib().orc_joint_prune(ix.ref(), int(p), _p(cand), _p(dpc), len(cand), _p(T), len(T),
                              alpha2_of(alpha), _p(out))
    return out[:m]


def build_search(ix: Index, p, t, lb, vcap=1 << 16):
    ids = np.empty(vcap, np.int32)
    d = np.empty(vcap, np.float32)
    nv = lib().orc_build_search(ix.ref(), int(p), int(t), int(lb), _p(ids), _p(d), vcap)
    nv = min(nv, vcap)
    return ids[:nv], d[:nv]


def dist_F(ix: Index, filt, aux, pts):
    f = np.ascontiguousarray(np.atleast_1d(filt))
    aux = _c(aux, np.uint8)
    pts = _c(pts, np.int64)
    out = np.empty(len(pts), np.uint32)
    lib().orc_dist_F_batch(ix.ref(), _p(f), _p(aux), _p(pts), len(pts), _p(out))
    return out


def g(ix: Index, filt, aux, pts):
    f = np.ascontiguousarray(np.atleast_1d(filt))
    aux = _c(aux, np.uint8)
    pts = _c(pts, np.int64)
    out = np.empty(len(pts), np.uint8)
    lib().orc_g_batch(ix.ref(), _p(f), _p(aux), _p(pts), len(pts), _p(out))
    return out.astype(bool)


def dist_A(ix: Index, i, j):
    return int(lib().orc_dist_A(ix.ref(), int(i), int(j)))


def capped(dist_a, da, t):
    return int(lib().orc_capped(int(dist_a), int(da), int(t)))


def row_bytes(fmt, d):
    return int(lib().orc_row_bytes(int(fmt), int(d)))


def quantize(x, fmt):
    """Stored rows [n][row_bytes] (uint8) and per-row scales of BF16 / FP8
    storage, from the format definitions."""
    x = _c(x, np.float32)
    n, d = x.shape
    rb = row_bytes(fmt, d)
    out = np.empty((n, rb), np.uint8)
    scale = np.empty(n, np.float32)
    lib().orc_quantize(_p(x), n, d, int(fmt), _p(out), _p(scale))
    return out, scale


def bf16_encode(x):
    x = _c(np.atleast_1d(x), np.float32)
    out = np.empty(x.shape, np.uint16)
    lib().orc_bf16_encode_batch(_p(x), x.size, _p(out))
    return out


def fp8_encode(x):
    x = _c(np.atleast_1d(x), np.float32)
    out = np.empty(x.shape, np.uint8)
    lib().orc_fp8_encode_batch(_p(x), x.size, _p(out))
    return out


def fp8_decode(c):
    c = _c(np.atleast_1d(c), np.uint8)
    out = np.empty(c.shape, np.float32)
    lib().orc_fp8_decode_batch(_p(c), c.size, _p(out))
    return out


def dist_canon_q_rows(q, rows, scale, fmt):
    q = _c(np.atleast_2d(q), np.float32)
    rows = _c(np.atleast_2d(rows), np.uint8)
    scale = _c(scale, np.float32)
    out = np.empty(q.shape[0], np.float32)
    lib().orc_dist_canon_q_batch(_p(q), _p(rows), _p(scale), int(fmt), q.shape[0], q.shape[1], rows.shape[1],
                                 _p(out))
    return out


POL_PLAIN, POL_LEARNED, POL_FORCED = 0, 1, 2
NFEAT = 12


class _Policy(C.Structure):
    _fields_ = [("mode", C.c_int32), ("h0", C.c_int32), ("w_bf16", C.c_void_p), ("b_f32", C.c_void_p),
                ("tau", C.c_float), ("stop_scale", C.c_float), ("n_ladder", C.c_int32),
                ("ladder", C.c_int32 * 16), ("forced", C.c_void_p), ("features", C.c_void_p),
                ("decisions", C.c_void_p)]


def split_params(theta, nl):
    """BF16 weight codes (W1, W2, W3 concatenated) and fp32 biases (b1, b2,
    b3) of a flat fp32 parameter vector (layout of oracle/jag_mlp.py)."""
    theta = np.asarray(theta, np.float32)
    h, f = 64, 12
    sizes = [h * f, h, h * h, h, (nl + 1) * h, nl + 1]
    parts, off = [], 0
    for sz in sizes:
        parts.append(theta[off:off + sz])
        off += sz
    w = np.concatenate([parts[0], parts[2], parts[4]])
    b = np.concatenate([parts[1], parts[3], parts[5]]).astype(np.float32)
    return bf16_encode(w), b


class Policy:
    """Host-side policy for orc_query_policy."""

    def __init__(self, mode, h0=8, theta=None, ladder=(16, 24, 32, 48, 64, 96, 128, 192, 256), tau=0.0,
                 stop_scale=64.0, forced=None, nq=0, want_features=False, want_decisions=False):
        nl = len(ladder)
        self.nl = nl
        if theta is None:
            theta = np.zeros(64 * 12 + 64 + 64 * 64 + 64 + (nl + 1) * 64 + nl + 1, np.float32)
        self.w, self.b = split_params(theta, nl)
        self.forced = None if forced is None else np.ascontiguousarray(forced, np.int32)
        self.features = np.zeros((nq, NFEAT), np.float32) if want_features else None
        self.decisions = np.zeros((nq, 4), np.int32) if want_decisions else None
        lad = (C.c_int32 * 16)(*([int(v) for v in ladder] + [0] * (16 - nl)))
        self.s = _Policy(int(mode), int(h0), _p(self.w), _p(self.b), float(tau), float(stop_scale), nl, lad,
                         _p(self.forced), _p(self.features), _p(self.decisions))


def query_policy(ix: Index, q, filters, aux, k, ls, pol: Policy, s0=0, scan_cap=8192, nthreads=None):
    q = _c(q, np.float32)
    nq = q.shape[0]
    f = np.ascontiguousarray(filters)
    aux = _c(aux, np.uint8)
    ids = np.empty((nq, k), np.int32)
    dist = np.empty((nq, k), np.float32)
    cnt = np.zeros((nq, 4), np.int64)
    rc = lib().orc_query_policy(ix.ref(), _p(q), _p(f), _p(aux), nq, k, ls, int(s0), int(scan_cap),
                                C.byref(pol.s), _p(ids), _p(dist), _p(cnt), nthreads or default_threads())
    if rc:
        raise ValueError("invalid policy query arguments")
    return ids, dist, cnt


def policy_features(k1, dist, expanded, k, est, kind):
    """The 12 policy features of a list state L given as first keys, fp32
    distances and expanded flags of its entries in order."""
    k1 = _c(k1, np.uint32)
    dist = _c(dist, np.float32)
    ex = _c(expanded, np.uint8)
    f = np.zeros(NFEAT, np.float32)
    lib().orc_policy_features(_p(k1), _p(dist), _p(ex), len(k1), int(k), int(est), int(kind), _p(f))
    return f


def mlp_infer(pol: Policy, X):
    X = _c(np.atleast_2d(X), np.float32)
    out = np.empty((X.shape[0], pol.nl + 1), np.float32)
    lib().orc_mlp_infer_batch(C.byref(pol.s), _p(X), X.shape[0], _p(out))
    return out
