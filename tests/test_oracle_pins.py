"""Pins of the CPU oracle against facts outside its own code: exhaustive
enumeration over small domains, closed forms, textbook special cases, the
paper's validity axioms, hand-worked examples (tests/golden) and published
generator test vectors.  CPU only."""
import itertools
import os
from collections import deque
from fractions import Fraction

import numpy as np
import pytest

from oracle import jag_oracle as O
from paper_2602_10258_gb300 import datagen as D

from _golden import read_build_golden

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _ix1(attr_i32=None, attr_f32=None, attr_mask=None, n=None, dist_a=O.K_LABEL, d=4):
    n = n or len(next(a for a in (attr_i32, attr_f32, attr_mask) if a is not None))
    x = np.zeros((n, d), np.float32)
    return O.Index(x, attr_i32, attr_f32, attr_mask, dist_a=dist_a, R=4)


# ---------------------------------------------------------------------------
# filter distances: exhaustive over small domains (Sec. 2, Sec. 3.1)
# ---------------------------------------------------------------------------

def test_label_filter_exhaustive():
    L = 8
    ix = _ix1(attr_i32=np.arange(L, dtype=np.int32))
    pts = np.arange(L)
    for f in range(L):
        rec = D.filters_label([f])
        df = O.dist_F(ix, rec, np.zeros(8, np.uint8), pts)
        g = O.g(ix, rec, np.zeros(8, np.uint8), pts)
        assert list(g) == [a == f for a in range(L)]
        assert list(df) == [int(a != f) for a in range(L)]
        assert all((df == 0) == g)  # validity axiom


def test_range_i32_filter_exhaustive():
    dom = np.arange(16, dtype=np.int32)
    ix = _ix1(attr_i32=dom)
    aux = np.zeros(8, np.uint8)
    for lo in range(16):
        for hi in range(16):
            rec = D.filters_range_i32([lo], [hi])
            df = O.dist_F(ix, rec, aux, np.arange(16))
            g = O.g(ix, rec, aux, np.arange(16))
            interval = list(range(lo, hi + 1))
            for a in range(16):
                assert g[a] == (a in interval)
                if interval:
                    # distance from a to the (integer) interval, by enumeration
                    assert df[a] == min(abs(a - b) for b in interval)
                else:
                    assert df[a] > 0
            assert all((df == 0) == g)


def test_range_f32_filter_rounding():
    rng = np.random.default_rng(5)
    a = rng.random(4000).astype(np.float32)
    a[:10] = [0.0, 1.0, 0.25, 0.5, 0.75, 0.2, 0.3, 1e-30, 0.2000001, 0.3]
    ix = _ix1(attr_f32=a, dist_a=O.K_RANGE_F32)
    aux = np.zeros(8, np.uint8)
    for lo, hi in [(0.2, 0.3), (0.0, 0.0), (0.5, 0.25), (0.1, 0.9), (-1.0, 2.0)]:
        lo32, hi32 = np.float32(lo), np.float32(hi)
        rec = D.filters_range_f32([lo32], [hi32])
        df = O.dist_F(ix, rec, aux, np.arange(len(a))).view(np.float32)
        g = O.g(ix, rec, aux, np.arange(len(a)))
        for i in range(len(a)):
            ai = a[i]
            inside = lo32 <= ai <= hi32
            assert g[i] == inside
            if ai < lo32:
                exact = Fraction(float(lo32)) - Fraction(float(ai))
            elif ai > hi32:
                exact = Fraction(float(ai)) - Fraction(float(hi32))
            else:
                exact = Fraction(0)
            # one correctly rounded fp32 subtraction of the exact difference
            assert df[i] == np.float32(float(exact))
            assert (df[i] == 0) == inside


def test_subset_filter_exhaustive():
    L = 6
    vals = np.arange(1 << L, dtype=np.uint64)
    ix = _ix1(attr_mask=vals, dist_a=O.K_SUBSET)
    aux = np.zeros(8, np.uint8)
    pts = np.arange(1 << L)
    for f in range(1 << L):
        rec = D.filters_subset([f])
        df = O.dist_F(ix, rec, aux, pts)
        g = O.g(ix, rec, aux, pts)
        for a in range(1 << L):
            assert g[a] == ((f & a) == f)
            # fewest bit changes to a that make it contain f, by enumeration
            best = min(bin(a ^ b).count("1") for b in range(1 << L) if (f & b) == f)
            assert df[a] == best
        assert all((df == 0) == g)


@pytest.mark.parametrize("L,m,seed", [(6, 3, 0), (8, 4, 1), (10, 5, 2), (9, 9, 3), (7, 1, 4)])
def test_bool_filter_vs_enumeration(L, m, seed):
    """dist_F = min Hamming(a, a') over all a' in {0,1}^L with f(a') = 1,
    enumerated over every attribute value (not only the involved bits)."""
    rng = np.random.default_rng(seed)
    vals = np.arange(1 << L, dtype=np.uint64)
    ix = _ix1(attr_mask=vals, dist_a=O.K_BOOL)
    for trial in range(6):
        p_true = [0.5, 0.1, 0.02, 0.0, 1.0, 0.3][trial]
        recs, aux = D.random_bool_filters(rng, 1, L, m, p_true)
        rec = recs[0]
        vm = int(rec["payload"])
        pos = [j for j in range(L) if (vm >> j) & 1]
        table = np.unpackbits(aux[rec["aux_off"]:], bitorder="little")[: 1 << m]

        def f_of(a):
            s = sum(((a >> p) & 1) << j for j, p in enumerate(pos))
            return table[s]

        sat = [b for b in range(1 << L) if f_of(b)]
        df = O.dist_F(ix, recs, aux, np.arange(1 << L))
        g = O.g(ix, recs, aux, np.arange(1 << L))
        for a in range(1 << L):
            assert g[a] == bool(f_of(a))
            if sat:
                assert df[a] == min(bin(a ^ b).count("1") for b in sat)
            else:
                assert df[a] == 255
        assert all((df == 0) == g)


def test_bool_lut_unsatisfiable_and_tautology():
    lut, sat = O.bool_lut(0b1011, np.zeros(2, np.uint8))
    assert not sat and (lut == 255).all()
    lut, sat = O.bool_lut(0b1011, np.full(2, 255, np.uint8))
    assert sat and (lut == 0).all()


def test_none_filter_is_unfiltered():
    ix = _ix1(attr_i32=np.arange(10, dtype=np.int32))
    df = O.dist_F(ix, D.filters_none(1), np.zeros(8, np.uint8), np.arange(10))
    assert (df == 0).all()


# ---------------------------------------------------------------------------
# attribute distances and the capped form (Sec. 3.1, Sec. 3.2)
# ---------------------------------------------------------------------------

def test_dist_A_validity_and_forms():
    a = np.array([0, 3, 3, -7, 2**31 - 1, -2**31], np.int32)
    ix = _ix1(attr_i32=a, dist_a=O.K_RANGE_I32)
    for i, j in itertools.product(range(len(a)), repeat=2):
        da = O.dist_A(ix, i, j)
        assert da == abs(int(a[i]) - int(a[j]))
        assert (da == 0) == (a[i] == a[j])
    ixl = _ix1(attr_i32=a, dist_a=O.K_LABEL)
    for i, j in itertools.product(range(len(a)), repeat=2):
        assert O.dist_A(ixl, i, j) == int(a[i] != a[j])
    m = np.array([0, 1, 0xFF, 0xF0F0F0F0F0F0F0F0, 2**64 - 1], np.uint64)
    ixm = _ix1(attr_mask=m, dist_a=O.K_SUBSET)
    for i, j in itertools.product(range(len(m)), repeat=2):
        bits = np.unpackbits(np.array([m[i] ^ m[j]], np.uint64).view(np.uint8))
        assert O.dist_A(ixm, i, j) == int(bits.sum())
    f = np.array([0.1, 0.7, 0.1, 1e-30], np.float32)
    ixf = _ix1(attr_f32=f, dist_a=O.K_RANGE_F32)
    for i, j in itertools.product(range(len(f)), repeat=2):
        v = np.uint32(O.dist_A(ixf, i, j)).view(np.float32)
        assert v == np.float32(abs(Fraction(float(f[i])) - Fraction(float(f[j]))))
        assert O.dist_A(ixf, i, j) == O.dist_A(ixf, j, i)


def test_capped_distance_properties():
    for da in range(0, 40):
        for t in range(0, 40):
            c = O.capped(O.K_RANGE_I32, da, t)
            assert (c == 0) == (da <= t)             # within t counts as equal
            if da > t:
                assert c + t == da
        assert O.capped(O.K_RANGE_I32, da, 0) == da   # t = 0: uncapped
    f = np.float32
    for da, t in [(0.5, 0.25), (0.25, 0.5), (1e-7, 0.0), (0.3, 0.3)]:
        c = np.uint32(O.capped(O.K_RANGE_F32, int(f(da).view(np.uint32)), int(f(t).view(np.uint32))))
        cv = c.view(np.float32)
        assert (cv == 0) == (f(da) <= f(t))
        if f(da) > f(t):
            assert cv == np.float32(float(Fraction(float(f(da))) - Fraction(float(f(t)))))


# ---------------------------------------------------------------------------
# vector distance
# ---------------------------------------------------------------------------

def test_canonical_distance_single_element_is_rounded_square():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        q, x = rng.standard_normal(2).astype(np.float32) * np.float32(10 ** rng.uniform(-3, 3))
        t = np.float32(q - x)
        exact = Fraction(float(t)) ** 2
        assert O.dist_canon(np.array([q]), np.array([x])) == np.float32(float(exact))


def test_canonical_distance_exact_on_integers():
    """Small integer inputs keep every partial sum exact: the result is the
    exact sum whatever the order, so a dropped term or index fails."""
    rng = np.random.default_rng(2)
    for d in [1, 3, 4, 5, 31, 32, 100, 128, 129, 200, 1000]:
        for _ in range(20):
            q = rng.integers(-50, 50, d).astype(np.float32)
            x = rng.integers(-50, 50, d).astype(np.float32)
            exact = int(((q.astype(np.int64) - x.astype(np.int64)) ** 2).sum())
            assert O.dist_canon(q, x) == exact


def test_canonical_distance_error_bound():
    """(P5) |d32 - d| <= gamma_n d with gamma_n = n u / (1 - n u), u = 2^-24,
    n = d + 2 (a bound valid for any summation order of d rounded squares),
    against the exact value in rational arithmetic."""
    rng = np.random.default_rng(3)
    u = 2.0 ** -24
    for d in [2, 32, 100, 128, 777]:
        n = d + 2
        gamma = n * u / (1 - n * u)
        for _ in range(5):
            q = rng.standard_normal(d).astype(np.float32)
            x = rng.standard_normal(d).astype(np.float32)
            exact = sum((Fraction(float(a)) - Fraction(float(b))) ** 2 for a, b in zip(q, x))
            d32 = Fraction(float(O.dist_canon(q, x)))
            assert abs(d32 - exact) <= Fraction(gamma) * exact
            d64 = O.dist_f64(q, x)
            assert abs(d64 - float(exact)) <= 4 * d * 2.0 ** -53 * float(exact)
            assert O.dist_canon(q, x) == O.dist_canon(x, q)


# ---------------------------------------------------------------------------
# exact filtered k-NN (Sec. 2; Pre-Filtering)
# ---------------------------------------------------------------------------

def test_brute_force_vs_numpy():
    w = D.make_range_i32(n=3000, d=16, nq=40, seed=7, width=50)
    ix = O.Index.from_workload(w)
    k = 10
    ids, d32, d64, npass = O.brute_force(ix, w.q, w.filters, w.aux, k)
    ff = D.filter_fields(w.filters)
    for i in range(len(w.q)):
        ok = (w.attr_i32 >= ff["i_lo"][i]) & (w.attr_i32 <= ff["i_hi"][i])
        assert npass[i] == ok.sum()
        cand = np.nonzero(ok)[0]
        dd = ((w.x[cand].astype(np.float64) - w.q[i].astype(np.float64)) ** 2).sum(1)
        order = np.lexsort((cand, dd))
        ref = cand[order[:k]]
        if len(cand) > k and dd[order[k]] - dd[order[k - 1]] < 1e-5 * dd[order[k]]:
            continue
        assert list(ids[i][: min(k, len(cand))]) == list(ref)
        np.testing.assert_allclose(d64[i][: len(ref)], dd[order[:k]][: len(ref)], rtol=1e-12)
        np.testing.assert_allclose(d32[i][: len(ref)], dd[order[:k]][: len(ref)], rtol=1e-5)


def test_brute_force_short_results_padded():
    w = D.make_range_i32(n=500, d=8, nq=5, seed=3)
    ix = O.Index.from_workload(w)
    f = D.filters_range_i32([5, 2000, 10], [4, 3000, 10])   # empty, none, few
    ids, d32, _, npass = O.brute_force(ix, w.q[:3], f, w.aux, 10)
    assert (ids[0] == -1).all() and np.isinf(d32[0]).all() and npass[0] == 0
    assert (ids[1] == -1).all()
    m = int(npass[2])
    assert m < 10 and (ids[2][:m] >= 0).all() and (ids[2][m:] == -1).all()


# ---------------------------------------------------------------------------
# hand-worked build and query (tests/golden/build_1d_5pts.txt)
# ---------------------------------------------------------------------------

def test_build_hand_worked_example():
    rows, entry, query, answer = read_build_golden()
    x = np.array([[0], [2], [3], [7], [9]], np.float32)
    lab = np.arange(5, dtype=np.int32)
    ix = O.Index(x, attr_i32=lab, dist_a=O.K_LABEL, R=2)
    thr = O.build(ix, pct=(100,), lb=4, alpha=1.2, seed=0, nthreads=1)
    assert (thr == 1).all()
    assert ix.entry == entry
    for r, v in rows.items():
        assert list(ix.graph[r]) == v, (r, ix.graph[r], v)
    xq, lo, hi, ls, k = query
    f = D.filters_range_i32([int(lo)], [int(hi)])
    ids, dist, _ = O.query(ix, np.array([[xq]], np.float32), f, np.zeros(8, np.uint8), int(k), int(ls))
    assert list(ids[0]) == [int(answer[0]), int(answer[2])]
    assert list(dist[0]) == [answer[1], answer[3]]
    ids2, _, _ = O.query(ix, np.array([[xq]], np.float32), f, np.zeros(8, np.uint8), int(k), int(ls),
                         literal=True)
    assert list(ids2[0]) == list(ids[0])


# ---------------------------------------------------------------------------
# generator and thresholds
# ---------------------------------------------------------------------------

def test_splitmix64_published_vectors():
    for line in open(os.path.join(GOLD, "splitmix64_seed0.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        c, v = line.split()
        assert O.sm64(0, int(c)) == int(v, 16)


def test_threshold_quantiles_match_population():
    """Thresholds are quantiles of a 500-point sample of dist_A(a_p, .): they
    must be attained values, ordered by percentile, and lie within a
    binomial band of the population quantile."""
    n = 20000
    rng = np.random.default_rng(11)
    a = rng.integers(0, 1000, n).astype(np.int32)
    ix = O.Index(np.zeros((n, 2), np.float32), attr_i32=a, dist_a=O.K_RANGE_I32)
    pct = (100, 10, 1, 0)
    thr = O.thresholds(ix, pct, S=500, seed=3)
    for p in rng.choice(n, 40, replace=False):
        pop = np.sort(np.abs(a.astype(np.int64) - a[p]))[1:]   # drop p's own zero
        t = thr[p]
        assert t[0] >= t[1] >= t[2] >= t[3]
        assert t[0] <= pop[-1] and t[3] >= 0
        for qv, tv in zip(pct, t):
            assert tv in pop
            if 0 < qv < 100:
                frac = np.searchsorted(pop, tv, side="right") / len(pop)
                lo_frac = np.searchsorted(pop, tv, side="left") / len(pop)
                sd = np.sqrt(qv / 100 * (1 - qv / 100) / 500)
                assert lo_frac - 4 * sd <= qv / 100 <= frac + 4 * sd


def test_thresholds_labels():
    n = 3000
    lab = np.zeros(n, np.int32)
    lab[::10] = np.arange(len(lab[::10])) + 1         # 300 singletons among zeros
    ix = O.Index(np.zeros((n, 2), np.float32), attr_i32=lab, dist_a=O.K_LABEL)
    thr = O.thresholds(ix, (100, 1, 0), S=500, seed=0)
    assert (thr[lab == 0][:, 2] == 0).all()      # min: some sample shares label 0
    assert (thr[lab != 0][:, 2] == 1).all()      # singletons: every sample differs
    assert (thr[:, 0] == 1).all()


# ---------------------------------------------------------------------------
# GreedySearch / Query
# ---------------------------------------------------------------------------

def _reachable(graph, s):
    seen = {s}
    dq = deque([s])
    while dq:
        v = dq.popleft()
        for u in graph[v]:
            if u >= 0 and u not in seen:
                seen.add(u)
                dq.append(u)
    return seen


@pytest.fixture(scope="module")
def small_built():
    w = D.make_range_i32(n=1500, d=16, nq=60, seed=4, width=100)
    ix = O.Index.from_workload(w, R=16)
    O.build(ix, pct=(100, 1, 0), lb=32, alpha=1.2, seed=0)
    return w, ix


def test_graph_invariants(small_built):
    w, ix = small_built
    g = ix.graph
    n, R = g.shape
    for v in range(n):
        row = [u for u in g[v] if u >= 0]
        assert all(0 <= u < n for u in row)
        assert v not in row
        assert len(set(row)) == len(row)
        # padding only at the end
        k = len(row)
        assert (g[v][k:] == -1).all()
    assert len(_reachable(g, ix.entry)) == n


def test_search_full_beam_equals_brute_force(small_built):
    """(P1) With l_s >= N and every vertex reachable from s, the beam never
    drops anything, so GreedySearch ranks every point: the answer equals the
    exact filtered k-NN.  (P2) the unfiltered case is the special case
    dist_F = 0."""
    w, ix = small_built
    k = 10
    q = w.q[:15]
    for filt in (w.filters[:15], D.filters_none(15)):
        ids, dist, _ = O.query(ix, q, filt, w.aux, k, ls=ix.n)
        bi, bd, _, _ = O.brute_force(ix, q, filt, w.aux, k)
        assert (ids == bi).all()
        assert (dist == bd).all()


@pytest.mark.parametrize("ls", [10, 16, 40, 100])
def test_literal_and_direct_search_agree(small_built, ls):
    w, ix = small_built
    a, da, _ = O.query(ix, w.q, w.filters, w.aux, 10, ls, literal=False)
    b, db, _ = O.query(ix, w.q, w.filters, w.aux, 10, ls, literal=True)
    assert (a == b).all()
    assert (da == db).all()


def test_literal_and_direct_search_agree_other_filters():
    rng = np.random.default_rng(9)
    n, d = 1200, 8
    x = rng.standard_normal((n, d)).astype(np.float32)
    masks = rng.integers(0, 2 ** 12, n).astype(np.uint64)
    ix = O.Index(x, attr_mask=masks, dist_a=O.K_SUBSET, R=12)
    O.build(ix, pct=(100, 10, 0), lb=24, seed=1)
    q = rng.standard_normal((40, d)).astype(np.float32)
    fs = D.filters_subset(rng.integers(0, 2 ** 12, 40) & rng.integers(0, 2 ** 12, 40)
                          & rng.integers(0, 2 ** 12, 40))
    fb, aux = D.random_bool_filters(rng, 40, 12, 4, 0.2)
    for f, ax in ((fs, np.zeros(8, np.uint8)), (fb, aux)):
        for ls in (10, 30):
            a, _, _ = O.query(ix, q, f, ax, 10, ls)
            b, _, _ = O.query(ix, q, f, ax, 10, ls, literal=True)
            assert (a == b).all()


def test_search_result_invariants(small_built):
    """(P3) every answer passes its filter, answers are sorted by distance
    with id tie-break, carry their fp32 distance, and hold no duplicate."""
    w, ix = small_built
    ids, dist, _ = O.query(ix, w.q, w.filters, w.aux, 10, 32)
    ff = D.filter_fields(w.filters)
    for i in range(len(w.q)):
        m = ids[i] >= 0
        got = ids[i][m]
        assert len(set(got)) == len(got)
        a = w.attr_i32[got]
        assert ((a >= ff["i_lo"][i]) & (a <= ff["i_hi"][i])).all()
        dd = dist[i][m]
        assert (np.diff(dd) >= 0).all()
        ref = ((w.x[got].astype(np.float64) - w.q[i]) ** 2).sum(1)
        np.testing.assert_allclose(dd, ref, rtol=1e-5)
        assert np.isinf(dist[i][~m]).all()


def test_search_termination_certificate(small_built):
    """At termination every member p of L has been expanded, so each
    out-neighbour u of p is in L, or L is full and u ranks after L's last
    entry (keys recomputed here in fp64 order-independent form)."""
    w, ix = small_built
    ls = 24
    ids, k1, dist, ln = O.query_lists(ix, w.q, w.filters, w.aux, ls)
    ff = D.filter_fields(w.filters)
    for i in range(len(w.q)):
        L = list(ids[i][: ln[i]])
        lo, hi = int(ff["i_lo"][i]), int(ff["i_hi"][i])

        def key(u):
            a = int(w.attr_i32[u])
            df = lo - a if a < lo else (a - hi if a > hi else 0)
            return (df, float(((w.x[u].astype(np.float64) - w.q[i]) ** 2).sum()), u)

        keys = [key(u) for u in L]
        assert keys == sorted(keys)
        last = keys[-1]
        inL = set(L)
        for p in L:
            for u in ix.graph[p]:
                if u < 0 or u in inL:
                    continue
                assert ln[i] == ls
                ku = key(u)
                assert (ku[0], ku[1]) >= (last[0], last[1] * (1 - 1e-6))


def test_search_counters_and_early_stop(small_built):
    w, ix = small_built
    _, _, c = O.query(ix, w.q, w.filters, w.aux, 10, 32)
    hops, seen, dc = c[:, 0], c[:, 1], c[:, 2]
    assert (hops >= 1).all()
    assert (dc <= seen + 1).all()               # early rejection skips distances
    assert (seen <= hops * ix.R).all()


# ---------------------------------------------------------------------------
# JointRobustPrune (Algorithm 4)
# ---------------------------------------------------------------------------

def _robust_prune_textbook(x, p, cand, alpha2, limit):
    """DiskANN's RobustPrune (sort by distance to p, keep v unless some kept
    u has alpha * d(u, v) <= d(p, v)), stopping at `limit` members."""
    dp = [float(np.float32(((x[c].astype(np.float64) - x[p]) ** 2).sum())) for c in cand]
    order = sorted(range(len(cand)), key=lambda i: (dp[i], cand[i]))
    kept = []
    for i in order:
        v = cand[i]
        ok = True
        for u in kept:
            duv = ((x[u].astype(np.float64) - x[v]) ** 2).sum()
            if not (alpha2 * duv > dp[i]):
                ok = False
                break
        if ok:
            kept.append(v)
        if len(kept) >= limit:
            break
    return kept


def test_joint_prune_reduces_to_robust_prune():
    """(P4) with one threshold at least max dist_A every capped distance is
    0, and JointRobustPrune is RobustPrune with the 0.9 R cap."""
    rng = np.random.default_rng(21)
    n, d, R = 400, 6, 16
    x = (rng.integers(-20, 20, (n, d))).astype(np.float32)   # exact distances
    lab = rng.integers(0, 5, n).astype(np.int32)
    ix = O.Index(x, attr_i32=lab, dist_a=O.K_LABEL, R=R)
    a2 = O.alpha2_of(1.2)
    for trial in range(30):
        p = int(rng.integers(0, n))
        cand = [int(c) for c in rng.choice(n, 80, replace=False) if c != p]
        dpc = np.array([O.dist_canon(x[p], x[c]) for c in cand], np.float32)
        got = O.joint_prune(ix, p, cand, dpc, [1])
        limit = int(np.ceil(0.9 * R))          # stop at |V'| >= 14.4 -> 15
        assert list(got) == _robust_prune_textbook(x, p, cand, a2, limit)


def test_joint_prune_buckets():
    rng = np.random.default_rng(22)
    n, d, R = 300, 5, 12
    x = rng.standard_normal((n, d)).astype(np.float32)
    lab = rng.integers(0, 3, n).astype(np.int32)
    ix = O.Index(x, attr_i32=lab, dist_a=O.K_LABEL, R=R)
    for trial in range(30):
        p = int(rng.integers(0, n))
        cand = [int(c) for c in rng.choice(n, 60, replace=False) if c != p]
        dpc = np.array([O.dist_canon(x[p], x[c]) for c in cand], np.float32)
        T = [1, 0]
        got = list(O.joint_prune(ix, p, cand, dpc, T))
        assert len(got) == len(set(got)) <= R and p not in got
        # the first bucket is plain RobustPrune with cap 0.9 R / |T| = 5.4 -> 6
        first = _robust_prune_textbook(x, p, cand, O.alpha2_of(1.2), 6)
        assert got[: len(first)] == first
        # the second threshold (t = 0) ranks same-label candidates first: every
        # new member it adds shares p's label unless too few same-label ones
        same = [c for c in cand if lab[c] == lab[p]]
        extra = got[len(first):]
        if len(same) >= 12:
            assert all(lab[v] == lab[p] for v in extra)
        # identical thresholds: the second bucket only carries the first
        got2 = list(O.joint_prune(ix, p, cand, dpc, [1, 1]))
        assert got2 == _robust_prune_textbook(x, p, cand, O.alpha2_of(1.2), 6)


def test_build_thread_independent():
    w = D.make_range_i32(n=1200, d=8, nq=1, seed=5)
    g = []
    for nt in (1, 3, 8):
        ix = O.Index.from_workload(w, R=12)
        O.build(ix, lb=24, nthreads=nt)
        g.append(ix.graph.copy())
    assert (g[0] == g[1]).all() and (g[0] == g[2]).all()


def test_build_recall_sanity():
    """The paper's qualitative claim: enough beam gives near-perfect recall."""
    w = D.make_range_i32(n=4000, d=16, nq=100, seed=6)
    ix = O.Index.from_workload(w, R=24)
    O.build(ix, lb=48)
    ids, _, _ = O.query(ix, w.q, w.filters, w.aux, 10, 64)
    bi, _, _, _ = O.brute_force(ix, w.q, w.filters, w.aux, 10)
    rec = np.mean([len(set(a) & set(b)) / 10 for a, b in zip(ids, bi)])
    assert rec >= 0.95


# ---------------------------------------------------------------------------
# routing to the exact scan
# ---------------------------------------------------------------------------

def test_route_rule_and_scan_equals_brute_force():
    """(P6) routed queries answer exactly (brute force)."""
    w = D.make_range_i32(n=5000, d=8, nq=30, seed=8, width=100)
    ix = O.Index.from_workload(w, R=12)
    O.build(ix, lb=24)
    lo = np.arange(30, dtype=np.int32) * 30
    width = np.array([1, 2, 3, 5, 8, 13, 21, 34, 55, 89] * 3, np.int32)
    f = D.filters_range_i32(lo, lo + width - 1)
    s0 = 100
    ids, _, cnt = O.query(ix, w.q, f, w.aux, 10, 16, s0=s0)
    bi, _, _, npass = O.brute_force(ix, w.q, f, w.aux, 10)
    for i in range(30):
        routed, exact = O.route(ix, f[i], w.aux, s0)
        assert exact == npass[i]
        assert routed == (npass[i] < s0)
        assert cnt[i, 3] == int(routed)
        if routed:
            assert (ids[i] == bi[i]).all()


def test_route_sampled_estimator():
    n = 8192
    m = np.zeros(n, np.uint64)
    m[::2] = 1                      # bit 0 on even ids: sample ids j*2 all hit
    m[1::64] |= 2                   # bit 1 on ids = 1 mod 64: never sampled
    ix = O.Index(np.zeros((n, 2), np.float32), attr_mask=m, dist_a=O.K_SUBSET)
    aux = np.zeros(8, np.uint8)
    r, c = O.route(ix, D.filters_subset([1])[0], aux, s0=2048)
    assert c == n // 2 and not r
    r, c = O.route(ix, D.filters_subset([2])[0], aux, s0=2048)
    assert c == n // 64 and r          # estimator sees 0 hits -> scan
    r, c = O.route(ix, D.filters_subset([2])[0], aux, s0=2048, scan_cap=100)
    assert not r                        # exact count above the scan capacity
