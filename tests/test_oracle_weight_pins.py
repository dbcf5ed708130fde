"""Pins of the oracle's Weight-JAG build (the weighted variant of Sec. 3 and
its weight selection in the implementation-details appendix).  CPU only.

- h = sigma / sigma_A against numpy's standard deviation of the same sample.
- With the single weight 0, D_A^0 = dist and the bucket rule is the one of
  a single threshold: the graph equals Threshold-JAG's with T = {100%} when
  that threshold (the sample's largest dist_A) covers every dist_A, so that
  the capped attribute distance is 0 everywhere -- labels.
- The weighted prune ranks by w dist_A + dist: with w = 0 its first pick is
  the nearest candidate, with a weight that dwarfs every distance it is the
  nearest candidate of the same label.
"""
import numpy as np
import pytest

from oracle import jag_oracle as O
from paper_2602_10258_gb300 import datagen as D


@pytest.fixture(scope="module")
def small():
    w = D.make_label_zipf(n=3000, d=24, nq=10, seed=41, n_labels=12, n_centres=6)
    return w


def _sample(n, p, S, seed):
    ids = []
    for i in range(S):
        r = int(O.sm64(seed, (p << 20) | i)) % (n - 1)
        ids.append(r if r < p else r + 1)
    return np.array(ids)


@pytest.mark.parametrize("kind", ["label", "range"])
def test_weight_scale_is_the_ratio_of_standard_deviations(small, kind):
    if kind == "label":
        w = small
        ix = O.Index.from_workload(w, R=16)
    else:
        w = D.make_range_i32(n=2000, d=16, nq=5, seed=42)
        ix = O.Index.from_workload(w, R=16)
    mult = (0.0, 1.0, 2.5, 100.0)
    W, h = O.weights(ix, mult, S=300, seed=7)
    for p in (0, 17, 555, ix.n - 1):
        ids = _sample(ix.n, p, 300, 7)
        a = np.array([O.dist_A_value(ix, p, v) for v in ids], np.float64)
        d = O.dist_canon_rows(np.repeat(ix.x[p:p + 1], len(ids), 0), ix.x[ids]).astype(np.float64)
        ref = d.std() / a.std() if a.std() > 0 else 0.0
        assert h[p] == pytest.approx(ref, rel=1e-12)
        assert np.array_equal(W[p], np.float32(np.array(mult) * h[p]))


def test_single_zero_weight_is_the_unfiltered_threshold_build(small):
    w = small
    a = O.Index.from_workload(w, R=16)
    thr = O.build(a, pct=(100,), lb=32)
    assert (thr == 1).all()       # every point's sample holds another label
    b = O.Index.from_workload(w, R=16)
    O.build_weighted(b, mult=(0.0,), lb=32)
    assert a.entry == b.entry
    assert np.array_equal(a.graph, b.graph)


def test_weighted_graph_invariants(small):
    w = small
    ix = O.Index.from_workload(w, R=16)
    O.build_weighted(ix, mult=(0.0, 1.0, 10.0), lb=32)
    g = ix.graph
    for v in range(ix.n):
        row = g[v][g[v] >= 0]
        assert len(row) <= 16 and len(set(row.tolist())) == len(row)
        assert v not in row and (row < ix.n).all()
    assert (g >= 0).sum(1).min() >= 1


def test_weighted_prune_ranks_by_weighted_distance(small):
    w = small
    ix = O.Index.from_workload(w, R=16)
    p = 5
    rng = np.random.default_rng(3)
    cand = rng.choice(np.arange(1, ix.n), 200, replace=False).astype(np.int32)
    dpc = O.dist_canon_rows(np.repeat(ix.x[p:p + 1], len(cand), 0), ix.x[cand])
    first = O.joint_prune_weighted(ix, p, cand, dpc, [0.0])[0]
    assert first == cand[np.lexsort((cand, dpc))[0]]
    big = np.float32(1e3 * dpc.max())
    first = O.joint_prune_weighted(ix, p, cand, dpc, [big])[0]
    same = w.attr_i32[cand] == w.attr_i32[p]
    assert same.any()
    sc = cand[same]
    assert first == sc[np.lexsort((sc, dpc[same]))[0]]
