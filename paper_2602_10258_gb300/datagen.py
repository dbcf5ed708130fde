"""Seeded synthetic inputs for filtered nearest-neighbour search.

This module draws base vectors, per-point attributes, query vectors and query
filters.  It holds none of the search method's arithmetic (no distances, no
filter distances, no graph logic): both the CUDA path and the CPU oracle take
its arrays as plain inputs.  Every generator is driven by numpy's PCG64 with
an explicit seed, so the same call yields the same bytes on any machine.

Filter records are 16 bytes, laid out exactly like ``jag_filter`` in
``include/jag.h``: ``kind:int32, aux_off:int32, payload:8 bytes``.  The
payload holds ``label`` (int32), ``(lo, hi)`` (two int32 or two float32) or a
64-bit mask, depending on ``kind``.  Boolean filters keep their truth table in
a separate byte buffer (``aux``) at byte offset ``aux_off``: bit ``s`` of the
table is the value of the predicate for assignment ``s`` of the involved
variables, where bit ``j`` of ``s`` is the value of the ``j``-th lowest set
bit of the variable mask.

Workload recipes (the paper's datasets are not available; these synthetic
stand-ins copy their structure: mixed selectivity, Zipf-like label skew,
Gaussian-mixture embeddings, 100-d vectors as in MSTuring):

* ``range_i32``   -- i.i.d. N(0,1) vectors, int32 attribute uniform in
  [0, 1000), range filters [lo, lo+99] with lo uniform in [0, 900].
* ``label_zipf``  -- Gaussian mixture (centres N(0, 4I), unit covariance),
  label Zipf(s) over L labels, query label from the same law.
* ``subset``      -- Gaussian mixture, 64-bit masks with P(bit j) = 0.5/(j+1);
  queries require 1-3 bits, kept only if the product of their bit
  probabilities lies in [1e-4, 0.5].
* ``mixed``       -- Gaussian mixture, float attribute U[0,1) plus a 32-bit
  mask with Bernoulli(0.3) bits; half the queries are float ranges of width
  10^U(-4,0), half boolean AND/OR forms over 3 of the 32 bits.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

# Filter kinds (values fixed by the C ABI).
F_NONE = 0
F_LABEL = 1
F_RANGE_I32 = 2
F_RANGE_F32 = 3
F_SUBSET = 4
F_BOOL = 5

FILTER_DTYPE = np.dtype([("kind", "<i4"), ("aux_off", "<i4"), ("payload", "<u8")])
assert FILTER_DTYPE.itemsize == 16


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([seed, stream]))


# ---------------------------------------------------------------------------
# filter record constructors
# ---------------------------------------------------------------------------

def filters_empty(n: int) -> np.ndarray:
    return np.zeros(n, dtype=FILTER_DTYPE)


def _pack_i32_pair(lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    lo = np.asarray(lo, dtype="<i4").view("<u4").astype(np.uint64)
    hi = np.asarray(hi, dtype="<i4").view("<u4").astype(np.uint64)
    return lo | (hi << np.uint64(32))


def _pack_f32_pair(lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    lo = np.asarray(lo, dtype="<f4").view("<u4").astype(np.uint64)
    hi = np.asarray(hi, dtype="<f4").view("<u4").astype(np.uint64)
    return lo | (hi << np.uint64(32))


def filters_label(labels) -> np.ndarray:
    labels = np.asarray(labels, dtype=np.int64)
    f = filters_empty(len(labels))
    f["kind"] = F_LABEL
    f["payload"] = _pack_i32_pair(labels.astype("<i4"), np.zeros(len(labels), "<i4"))
    return f


def filters_range_i32(lo, hi) -> np.ndarray:
    lo = np.asarray(lo)
    f = filters_empty(len(lo))
    f["kind"] = F_RANGE_I32
    f["payload"] = _pack_i32_pair(lo, hi)
    return f


def filters_range_f32(lo, hi) -> np.ndarray:
    lo = np.asarray(lo)
    f = filters_empty(len(lo))
    f["kind"] = F_RANGE_F32
    f["payload"] = _pack_f32_pair(lo, hi)
    return f


def filters_subset(masks) -> np.ndarray:
    masks = np.asarray(masks, dtype=np.uint64)
    f = filters_empty(len(masks))
    f["kind"] = F_SUBSET
    f["payload"] = masks
    return f


def filters_none(n: int) -> np.ndarray:
    return filters_empty(n)


def filter_fields(f: np.ndarray):
    """Decode the payload of filter records into (label/lo, hi) int32 views,
    float views and the raw 64-bit word; used by tests and reports only."""
    p = np.asarray(f["payload"], dtype=np.uint64)
    lo_u = (p & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    hi_u = (p >> np.uint64(32)).astype(np.uint32)
    return {
        "i_lo": lo_u.view(np.int32), "i_hi": hi_u.view(np.int32),
        "f_lo": lo_u.view(np.float32), "f_hi": hi_u.view(np.float32),
        "mask": p,
    }


class BoolFilterBuilder:
    """Collects boolean filters: a variable mask (<= 16 set bits) plus a truth
    table over the involved variables, appended to one aux byte buffer."""

    def __init__(self):
        self._aux = bytearray()

    def add(self, vars_mask: int, table_bits) -> tuple:
        """``table_bits[s]`` is the predicate value for assignment ``s``.
        Returns (aux_off, vars_mask).  Tables start on 8-byte boundaries."""
        m = bin(vars_mask).count("1")
        if m > 16:
            raise ValueError("boolean filter over more than 16 variables")
        nbits = 1 << m
        table_bits = np.asarray(table_bits, dtype=np.uint8).reshape(-1)
        if table_bits.size != nbits:
            raise ValueError("truth table must have 2^m entries")
        while len(self._aux) % 8:
            self._aux.append(0)
        off = len(self._aux)
        nbytes = max(1, (nbits + 7) // 8)
        packed = np.packbits(table_bits, bitorder="little")
        buf = bytearray(nbytes)
        buf[: len(packed)] = packed.tobytes()
        self._aux.extend(buf)
        return off, vars_mask

    def aux(self) -> np.ndarray:
        a = bytearray(self._aux)
        while len(a) % 8 or len(a) == 0:
            a.append(0)
        return np.frombuffer(bytes(a), dtype=np.uint8).copy()


def filters_bool(entries) -> np.ndarray:
    """``entries``: list of (aux_off, vars_mask)."""
    f = filters_empty(len(entries))
    f["kind"] = F_BOOL
    f["aux_off"] = [e[0] for e in entries]
    f["payload"] = np.asarray([e[1] for e in entries], dtype=np.uint64)
    return f


# The four monotone 3-variable forms used by the mixed workload, written as
# truth tables over assignment s = (v0 | v1<<1 | v2<<2).
def _form_table(form: int) -> np.ndarray:
    s = np.arange(8)
    a, b, c = (s >> 0) & 1, (s >> 1) & 1, (s >> 2) & 1
    if form == 0:
        t = a & b & c
    elif form == 1:
        t = a | b | c
    elif form == 2:
        t = (a & b) | c
    else:
        t = (a | b) & c
    return t.astype(np.uint8)


# ---------------------------------------------------------------------------
# dataset container
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    x: np.ndarray                      # [N, d] float32 base vectors
    q: np.ndarray                      # [Q, d] float32 query vectors
    filters: np.ndarray                # [Q] FILTER_DTYPE
    aux: np.ndarray                    # uint8 truth-table buffer (>= 8 bytes)
    attr_i32: Optional[np.ndarray] = None    # [N] int32
    attr_f32: Optional[np.ndarray] = None    # [N] float32
    attr_mask: Optional[np.ndarray] = None   # [N] uint64
    dist_a: int = F_RANGE_I32          # which attribute the graph build compares
    params: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self):
        return self.x.shape[0]

    @property
    def d(self):
        return self.x.shape[1]


def gaussian(rng, n, d, chunk=1 << 18) -> np.ndarray:
    out = np.empty((n, d), dtype=np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        out[s:e] = rng.standard_normal((e - s, d), dtype=np.float32)
    return out


def gaussian_mixture(rng, n, d, centres, chunk=1 << 18) -> np.ndarray:
    """Equal-weight mixture, unit covariance around ``centres``."""
    out = np.empty((n, d), dtype=np.float32)
    k = centres.shape[0]
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        comp = rng.integers(0, k, size=e - s)
        out[s:e] = centres[comp] + rng.standard_normal((e - s, d), dtype=np.float32)
    return out


def mixture_centres(rng, k, d) -> np.ndarray:
    return (2.0 * rng.standard_normal((k, d))).astype(np.float32)   # N(0, 4I)


def zipf_labels(rng, n, n_labels, s) -> np.ndarray:
    r = np.arange(1, n_labels + 1, dtype=np.float64)
    p = r ** (-s)
    p /= p.sum()
    return rng.choice(n_labels, size=n, p=p).astype(np.int32)


def make_range_i32(n=10_000, d=32, nq=200, seed=0, width=100, domain=1000) -> Workload:
    x = gaussian(_rng(seed, 1), n, d)
    attr = _rng(seed, 2).integers(0, domain, size=n).astype(np.int32)
    q = gaussian(_rng(seed, 3), nq, d)
    lo = _rng(seed, 4).integers(0, domain - width + 1, size=nq).astype(np.int32)
    hi = (lo + (width - 1)).astype(np.int32)
    return Workload("range_i32", x, q, filters_range_i32(lo, hi), BoolFilterBuilder().aux(),
                    attr_i32=attr, dist_a=F_RANGE_I32,
                    params=dict(n=n, d=d, nq=nq, seed=seed, width=width, domain=domain))


def make_label_zipf(n=1_000_000, d=128, nq=10_000, seed=0, n_labels=1000, s=1.1,
                    n_centres=100, query_seed=None) -> Workload:
    """query_seed: draw the queries from another seed over the same base set
    (held-out or training queries); None = seed."""
    centres = mixture_centres(_rng(seed, 10), n_centres, d)
    x = gaussian_mixture(_rng(seed, 11), n, d, centres)
    labels = zipf_labels(_rng(seed, 12), n, n_labels, s)
    qs = seed if query_seed is None else query_seed
    q = gaussian_mixture(_rng(qs, 13), nq, d, centres)
    ql = zipf_labels(_rng(qs, 14), nq, n_labels, s)
    return Workload("label_zipf", x, q, filters_label(ql), BoolFilterBuilder().aux(),
                    attr_i32=labels, dist_a=F_LABEL,
                    params=dict(n=n, d=d, nq=nq, seed=seed, n_labels=n_labels, s=s,
                                n_centres=n_centres))


def subset_bit_probs(nbits=64) -> np.ndarray:
    return 0.5 / (np.arange(nbits, dtype=np.float64) + 1.0)


def make_subset(n=1_000_000, d=100, nq=10_000, seed=0, n_centres=200,
                sel_lo=1e-4, sel_hi=0.5) -> Workload:
    centres = mixture_centres(_rng(seed, 20), n_centres, d)
    x = gaussian_mixture(_rng(seed, 21), n, d, centres)
    p = subset_bit_probs(64)
    rng = _rng(seed, 22)
    masks = np.zeros(n, dtype=np.uint64)
    for j in range(64):
        bits = rng.random(n) < p[j]
        masks |= bits.astype(np.uint64) << np.uint64(j)
    q = gaussian_mixture(_rng(seed, 23), nq, d, centres)
    rq = _rng(seed, 24)
    pw = p / p.sum()
    qm = np.zeros(nq, dtype=np.uint64)
    i = 0
    while i < nq:
        m = int(rq.integers(1, 4))
        bits = rq.choice(64, size=m, replace=False, p=pw)
        prod = float(np.prod(p[bits]))
        if not (sel_lo <= prod <= sel_hi):
            continue
        v = 0
        for b in bits:
            v |= 1 << int(b)
        qm[i] = v
        i += 1
    return Workload("subset", x, q, filters_subset(qm), BoolFilterBuilder().aux(),
                    attr_mask=masks, dist_a=F_SUBSET,
                    params=dict(n=n, d=d, nq=nq, seed=seed, n_centres=n_centres))


def make_mixed(n=1_000_000, d=128, nq=10_000, seed=0, n_centres=100, nbits=32,
               p_bit=0.3, query_seed=None) -> Workload:
    """Float-range and boolean filters over one point set; the graph is built
    on the float attribute (``dist_a`` = range) -- the boolean column is
    carried for filtering.  query_seed: draw the queries from another seed
    over the same base set; None = seed."""
    centres = mixture_centres(_rng(seed, 30), n_centres, d)
    x = gaussian_mixture(_rng(seed, 31), n, d, centres)
    af = _rng(seed, 32).random(n, dtype=np.float32)
    rb = _rng(seed, 33)
    masks = np.zeros(n, dtype=np.uint64)
    for j in range(nbits):
        masks |= (rb.random(n) < p_bit).astype(np.uint64) << np.uint64(j)
    qs = seed if query_seed is None else query_seed
    q = gaussian_mixture(_rng(qs, 34), nq, d, centres)
    rf = _rng(qs, 35)
    is_bool = rf.random(nq) < 0.5
    w = (10.0 ** rf.uniform(-4.0, 0.0, size=nq)).astype(np.float32)
    lo = (rf.random(nq) * (1.0 - w)).astype(np.float32)
    hi = (lo + w).astype(np.float32)
    bb = BoolFilterBuilder()
    recs = filters_range_f32(lo, hi)
    for i in np.nonzero(is_bool)[0]:
        vs = rf.choice(nbits, size=3, replace=False)
        form = int(rf.integers(0, 4))
        # the form's variables (a, b, c) are vs[0..2]; the table is indexed
        # by the involved bits in increasing bit position
        order = np.argsort(vs)
        tab = _form_table(form)
        table = np.zeros(8, dtype=np.uint8)
        for s in range(8):
            # s indexes sorted positions; rebuild (a, b, c) assignment
            vals = [(s >> k) & 1 for k in range(3)]
            abc = [0, 0, 0]
            for k in range(3):
                abc[order[k]] = vals[k]
            table[s] = tab[abc[0] | (abc[1] << 1) | (abc[2] << 2)]
        vm = 0
        for v in vs:
            vm |= 1 << int(v)
        off, _ = bb.add(vm, table)
        recs[i]["kind"] = F_BOOL
        recs[i]["aux_off"] = off
        recs[i]["payload"] = np.uint64(vm)
    return Workload("mixed", x, q, recs, bb.aux(), attr_f32=af, attr_mask=masks,
                    dist_a=F_RANGE_F32,
                    params=dict(n=n, d=d, nq=nq, seed=seed, n_centres=n_centres))


def make_range_f32(n=10_000_000, d=100, nq=10_000, seed=0, n_centres=200,
                   log_sel_lo=-4.0) -> Workload:
    """Float attribute U[0,1), range widths log-uniform in [1e-4, 1]."""
    centres = mixture_centres(_rng(seed, 40), n_centres, d)
    x = gaussian_mixture(_rng(seed, 41), n, d, centres)
    af = _rng(seed, 42).random(n, dtype=np.float32)
    q = gaussian_mixture(_rng(seed, 43), nq, d, centres)
    rf = _rng(seed, 44)
    w = (10.0 ** rf.uniform(log_sel_lo, 0.0, size=nq)).astype(np.float32)
    lo = (rf.random(nq) * (1.0 - w)).astype(np.float32)
    hi = (lo + w).astype(np.float32)
    return Workload("range_f32", x, q, filters_range_f32(lo, hi), BoolFilterBuilder().aux(),
                    attr_f32=af, dist_a=F_RANGE_F32,
                    params=dict(n=n, d=d, nq=nq, seed=seed, n_centres=n_centres))


def random_bool_filters(rng, nq, nbits, m, p_true=0.5):
    """Random truth tables over m random variables (used by edge-case tests)."""
    bb = BoolFilterBuilder()
    entries = []
    for _ in range(nq):
        vs = rng.choice(nbits, size=m, replace=False)
        vm = 0
        for v in vs:
            vm |= 1 << int(v)
        table = (rng.random(1 << m) < p_true).astype(np.uint8)
        entries.append(bb.add(vm, table))
    return filters_bool(entries), bb.aux()


def mlp_init_params(nl, seed=0):
    """Seeded initial parameters of the policy network (12 -> 64 -> 64 ->
    nl + 1), flat fp32 in the layout W1, b1, W2, b2, W3, b3: He-scaled normal
    weights, zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = [rng.standard_normal((64, 12)) * np.sqrt(2.0 / 12), np.zeros(64),
             rng.standard_normal((64, 64)) * np.sqrt(2.0 / 64), np.zeros(64),
             rng.standard_normal((nl + 1, 64)) * np.sqrt(1.0 / 64), np.zeros(nl + 1)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)
