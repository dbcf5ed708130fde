"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs and the same graph.  Search answers must be bit-identical
(ids and fp32 distances) on at least 99.9% of queries -- in practice all --
and the GPU build must reproduce the oracle's graph exactly."""
import numpy as np
import pytest

from oracle import jag_oracle as O
from paper_2602_10258_gb300 import datagen as D

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
jag = pytest.importorskip("paper_2602_10258_gb300.jag")

DIST_RTOL = 1e-5


def oracle_built(w, R=32, lb=64, pct=(100, 1, 0)):
    ix = O.Index.from_workload(w, R=R)
    thr = O.build(ix, pct=pct, lb=lb)
    return ix, thr


def gpu_index_from(w, ix):
    return jag.Index.from_workload(w, R=ix.R, graph=ix.graph, entry=ix.entry)


def gpu_search(gi, q, filters, aux, k, beam, **kw):
    qt = torch.from_numpy(np.ascontiguousarray(q, np.float32)).cuda()
    ids, dist, cnt = gi.search(qt, filters, aux, k, beam, counters=True, **kw)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dist.cpu().numpy(), cnt.cpu().numpy()


def assert_parity(ids, dist, rids, rdist, what=""):
    same = (ids == rids).all(axis=1)
    frac = same.mean()
    bad = np.nonzero(~same)[0][:5]
    assert frac >= 0.999, "%s: ids differ on %d/%d queries, e.g. %s\n gpu %s\n ora %s" % (
        what, (~same).sum(), len(same), bad, ids[bad[:1]], rids[bad[:1]])
    m = same[:, None] & (rids >= 0)
    np.testing.assert_allclose(dist[m], rdist[m], rtol=DIST_RTOL)
    if m.any():
        assert (dist[m] == rdist[m]).mean() >= 0.999
    assert np.isinf(dist[same[:, None] & (rids < 0)]).all()


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def range_small():
    """The small plain-fp32 workload at its full size: N=10,000, d=32, int
    attribute in [0,1000), 200 range queries of width 100, R=32, beam 64."""
    w = D.make_range_i32(n=10_000, d=32, nq=200, seed=0)
    ix, thr = oracle_built(w, R=32, lb=64)
    return w, ix, thr, gpu_index_from(w, ix)


@pytest.fixture(scope="module")
def label_case():
    w = D.make_label_zipf(n=20_000, d=64, nq=300, seed=1, n_labels=60, n_centres=20)
    ix, thr = oracle_built(w, R=24, lb=48)
    return w, ix, thr, gpu_index_from(w, ix)


@pytest.fixture(scope="module")
def subset_case():
    w = D.make_subset(n=20_000, d=24, nq=300, seed=2, n_centres=20, sel_lo=1e-3)
    ix, thr = oracle_built(w, R=24, lb=48)
    return w, ix, thr, gpu_index_from(w, ix)


@pytest.fixture(scope="module")
def mixed_case():
    w = D.make_mixed(n=20_000, d=100, nq=300, seed=3, n_centres=20)
    ix, thr = oracle_built(w, R=32, lb=64)
    return w, ix, thr, gpu_index_from(w, ix)


# ---------------------------------------------------------------------------
# graph search parity
# ---------------------------------------------------------------------------

def test_range_small_graph_search(range_small):
    w, ix, _, gi = range_small
    rid, rd, rc = O.query(ix, w.q, w.filters, w.aux, 10, 64, s0=0)
    ids, dist, cnt = gpu_search(gi, w.q, w.filters, w.aux, 10, 64, s0=0)
    assert_parity(ids, dist, rid, rd, "range N=10k beam 64")
    # same trajectory: the number of expansions matches the oracle
    assert (cnt[:, 0] == rc[:, 0]).mean() >= 0.999
    assert (cnt[:, 3] == 0).all()


@pytest.mark.parametrize("k,beam", [(1, 1), (1, 8), (10, 10), (10, 16), (10, 33), (32, 100), (10, 128),
                                    (64, 200), (256, 256), (10, 300), (10, 512), (256, 512)])
def test_range_small_beams(range_small, k, beam):
    w, ix, _, gi = range_small
    q, f = w.q[:80], w.filters[:80]
    rid, rd, _ = O.query(ix, q, f, w.aux, k, beam, s0=0)
    ids, dist, _ = gpu_search(gi, q, f, w.aux, k, beam, s0=0)
    assert_parity(ids, dist, rid, rd, "k=%d beam=%d" % (k, beam))


@pytest.mark.parametrize("hbits", [5, 7, 11, 13])
def test_visited_set_size_does_not_change_answers(range_small, hbits):
    """A small visited set forgets ids; answers must not change."""
    w, ix, _, gi = range_small
    q, f = w.q[:60], w.filters[:60]
    rid, rd, _ = O.query(ix, q, f, w.aux, 10, 64, s0=0)
    ids, dist, _ = gpu_search(gi, q, f, w.aux, 10, 64, s0=0, hash_bits=hbits)
    assert_parity(ids, dist, rid, rd, "hash_bits=%d" % hbits)


def test_label_graph_and_routing(label_case):
    w, ix, _, gi = label_case
    for s0 in (0, 400):
        rid, rd, rc = O.query(ix, w.q, w.filters, w.aux, 10, 48, s0=s0, scan_cap=8192)
        ids, dist, cnt = gpu_search(gi, w.q, w.filters, w.aux, 10, 48, s0=s0)
        assert_parity(ids, dist, rid, rd, "label s0=%d" % s0)
        assert (cnt[:, 3] == rc[:, 3]).all(), "routing differs"
    assert rc[:, 3].sum() > 0 and rc[:, 3].sum() < len(rc)


def test_subset_graph_and_routing(subset_case):
    w, ix, _, gi = subset_case
    for s0 in (0, 300):
        rid, rd, rc = O.query(ix, w.q, w.filters, w.aux, 10, 48, s0=s0, scan_cap=8192)
        ids, dist, cnt = gpu_search(gi, w.q, w.filters, w.aux, 10, 48, s0=s0)
        assert_parity(ids, dist, rid, rd, "subset s0=%d" % s0)
        assert (cnt[:, 3] == rc[:, 3]).all(), "routing differs"


def test_subset_scan_capacity_sends_back_to_graph(subset_case):
    w, ix, _, gi = subset_case
    rid, rd, rc = O.query(ix, w.q, w.filters, w.aux, 10, 48, s0=4000, scan_cap=50)
    ids, dist, cnt = gpu_search(gi, w.q, w.filters, w.aux, 10, 48, s0=4000, scan_cap=50)
    assert_parity(ids, dist, rid, rd, "subset cap=50")
    assert (cnt[:, 3] == rc[:, 3]).all()


def test_mixed_float_range_and_bool(mixed_case):
    w, ix, _, gi = mixed_case
    assert (w.filters["kind"] == D.F_BOOL).any() and (w.filters["kind"] == D.F_RANGE_F32).any()
    for beam, s0 in ((32, 0), (64, 0), (64, 500)):
        rid, rd, rc = O.query(ix, w.q, w.filters, w.aux, 10, beam, s0=s0, scan_cap=8192)
        ids, dist, cnt = gpu_search(gi, w.q, w.filters, w.aux, 10, beam, s0=s0)
        assert_parity(ids, dist, rid, rd, "mixed beam=%d s0=%d" % (beam, s0))
        assert (cnt[:, 3] == rc[:, 3]).all()


@pytest.mark.parametrize("d", [3, 7, 16, 33, 130, 256, 700])
def test_row_layouts(d):
    """Row mappings: 8/16/32 lanes per row, several chunks per lane, padded d."""
    w = D.make_range_i32(n=2500, d=d, nq=40, seed=10 + d, width=200)
    ix, _ = oracle_built(w, R=16, lb=32)
    gi = gpu_index_from(w, ix)
    rid, rd, _ = O.query(ix, w.q, w.filters, w.aux, 10, 32, s0=0)
    ids, dist, _ = gpu_search(gi, w.q, w.filters, w.aux, 10, 32, s0=0)
    assert_parity(ids, dist, rid, rd, "d=%d" % d)


def test_bool_many_variables():
    rng = np.random.default_rng(5)
    n, d = 6000, 16
    x = rng.standard_normal((n, d)).astype(np.float32)
    masks = rng.integers(0, 2 ** 62, n).astype(np.uint64)
    ix = O.Index(x, attr_mask=masks, dist_a=O.K_SUBSET, R=16)
    O.build(ix, lb=32)
    gi = jag.Index(x, attr_mask=masks, dist_a=jag.JAG_F_SUBSET, R=16, graph=ix.graph, entry=ix.entry)
    q = rng.standard_normal((60, d)).astype(np.float32)
    for m, p in ((16, 0.001), (12, 0.01), (1, 0.5), (5, 0.0)):
        f, aux = D.random_bool_filters(rng, 60, 62, m, p)
        rid, rd, _ = O.query(ix, q, f, aux, 10, 32, s0=0)
        ids, dist, _ = gpu_search(gi, q, f, aux, 10, 32, s0=0)
        assert_parity(ids, dist, rid, rd, "bool m=%d" % m)


# ---------------------------------------------------------------------------
# exact scan / brute force
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["range_small", "label_case", "subset_case", "mixed_case"])
def test_brute_force_scan(case, request):
    w, ix, _, gi = request.getfixturevalue(case)
    q, f = w.q[:100], w.filters[:100]
    bi, bd, _, _ = O.brute_force(ix, q, f, w.aux, 10)
    ids, dist, cnt = gpu_search(gi, q, f, w.aux, 10, 10, flags=jag.JAG_SEARCH_SCAN_ALL)
    assert (ids == bi).all()
    assert (dist == bd).all()


def test_scan_route_equals_brute_force(range_small):
    w, ix, _, gi = range_small
    lo = (np.arange(200) * 4).astype(np.int32)
    width = np.array([1, 3, 9, 27, 81, 243, 500, 0], np.int32)[np.arange(200) % 8]
    f = D.filters_range_i32(lo, lo + width - 1)
    bi, bd, _, npass = O.brute_force(ix, w.q, f, w.aux, 10)
    ids, dist, cnt = gpu_search(gi, w.q, f, w.aux, 10, 64, s0=1000)
    routed = cnt[:, 3] == 1
    assert (routed == (npass < 1000)).all()
    assert (ids[routed] == bi[routed]).all() and (dist[routed] == bd[routed]).all()


# ---------------------------------------------------------------------------
# the GPU build reproduces the oracle build
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["range_small", "label_case", "subset_case", "mixed_case"])
def test_gpu_build_equals_oracle_build(case, request):
    w, ix, thr, _ = request.getfixturevalue(case)
    lb = {"range_small": 64, "label_case": 48, "subset_case": 48, "mixed_case": 64}[case]
    gb = jag.Index.from_workload(w, R=ix.R, l_b=lb, thresholds=(100, 1, 0))
    info = gb.info()
    assert info["entry"] == ix.entry
    assert (gb.thresholds() == thr).all()
    g = gb.graph()
    rows_same = (g == ix.graph).all(axis=1)
    assert rows_same.all(), "%d rows differ, first %s" % ((~rows_same).sum(), np.nonzero(~rows_same)[0][:5])
    gb.close()


def test_gpu_build_hand_worked_example():
    from _golden import read_build_golden
    rows, entry, _, _ = read_build_golden()
    x = np.array([[0], [2], [3], [7], [9]], np.float32)
    gb = jag.Index(x, attr_i32=np.arange(5, dtype=np.int32), dist_a=jag.JAG_F_LABEL, R=2, l_b=4,
                   thresholds=(100,))
    assert gb.info()["entry"] == entry
    g = gb.graph()
    for r, v in rows.items():
        assert list(g[r]) == v


def test_gpu_build_thread_and_repeat_determinism():
    w = D.make_range_i32(n=6000, d=16, nq=1, seed=12)
    g1 = jag.Index.from_workload(w, R=16, l_b=32).graph()
    g2 = jag.Index.from_workload(w, R=16, l_b=32).graph()
    assert (g1 == g2).all()


# ---------------------------------------------------------------------------
# edge cases and API behaviour
# ---------------------------------------------------------------------------

def test_empty_and_degenerate_queries(range_small):
    w, ix, _, gi = range_small
    f = D.filters_range_i32([5, 2000, 10, 0], [4, 3000, 10, 999])    # empty, none, one value, all
    q = w.q[:4]
    for s0 in (0, 2048):
        rid, rd, _ = O.query(ix, q, f, w.aux, 10, 64, s0=s0, scan_cap=8192)
        ids, dist, _ = gpu_search(gi, q, f, w.aux, 10, 64, s0=s0)
        assert (ids == rid).all() and (dist == rd).all()
        assert (ids[0] == -1).all() and np.isinf(dist[0]).all()
        assert (ids[1] == -1).all()
    # no queries at all
    ids, dist, _ = gpu_search(gi, w.q[:0], f[:0], w.aux, 10, 64)
    assert ids.shape == (0, 10)


def test_unfiltered_and_unsatisfiable(mixed_case):
    w, ix, _, gi = mixed_case
    q = w.q[:20]
    f = D.filters_none(20)
    rid, rd, _ = O.query(ix, q, f, w.aux, 10, 64, s0=0)
    ids, dist, _ = gpu_search(gi, q, f, w.aux, 10, 64, s0=0)
    assert (ids == rid).all() and (dist == rd).all()
    bb = D.BoolFilterBuilder()
    off, vm = bb.add(0b111, np.zeros(8, np.uint8))
    fb = D.filters_bool([(off, vm)] * 20)
    aux = bb.aux()
    ids, dist, _ = gpu_search(gi, q, fb, aux, 10, 64)
    assert (ids == -1).all()


def test_invalid_filter_reported_by_host_call(range_small):
    w, ix, _, gi = range_small
    f = w.filters[:8].copy()
    f["kind"][3] = 99
    ids, dist, _ = gpu_search(gi, w.q[:8], f, w.aux, 10, 64, s0=0)
    assert (ids[3] == -1).all()
    with pytest.raises(jag.JagError) as e:
        gi.search_host(w.q[:8], f, w.aux, 10, 64, s0=0)
    assert e.value.status == jag.JAG_EINVAL


def test_argument_errors(range_small):
    w, ix, _, gi = range_small
    q = torch.from_numpy(w.q[:4]).cuda()
    for k, beam in ((11, 10), (0, 10), (1, 513), (257, 300)):
        with pytest.raises(jag.JagError) as e:
            gi.search(q, w.filters[:4], w.aux, k, beam)
        assert e.value.status == jag.JAG_EINVAL
    with pytest.raises(jag.JagError):
        jag.Index(w.x, attr_i32=w.attr_i32, R=0)
    bad = w.x.copy()
    bad[3, 1] = np.nan
    with pytest.raises(jag.JagError):
        jag.Index(bad, attr_i32=w.attr_i32, R=8, graph=np.full((len(bad), 8), -1, np.int32))


def test_host_call_matches_device_call(range_small):
    w, ix, _, gi = range_small
    ids, dist, cnt = gpu_search(gi, w.q, w.filters, w.aux, 10, 64)
    hi, hd, hc = gi.search_host(w.q, w.filters, w.aux, 10, 64, counters=True)
    assert (hi == ids).all() and (hd == dist).all() and (hc == cnt).all()


def test_concurrent_streams_same_answers(range_small):
    w, ix, _, gi = range_small
    q = torch.from_numpy(w.q).cuda()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    out = []
    for s in (s1, s2):
        with torch.cuda.stream(s):
            out.append(gi.search(q, w.filters, w.aux, 10, 64, stream=s))
    torch.cuda.synchronize()
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


def test_flat_query_call(label_case):
    """jag_query (the flat Query(G, q, l_s, k) call with the library defaults)
    answers as jag_search with s0 = 2048 and as the oracle."""
    w, ix, _, gi = label_case
    q = torch.from_numpy(w.q).cuda()
    ft = jag.filters_to_device(w.filters, q.device)
    at = jag.aux_to_device(w.aux, q.device)
    ids = torch.empty((len(w.q), 10), dtype=torch.int32, device=q.device)
    dist = torch.empty((len(w.q), 10), dtype=torch.float32, device=q.device)
    jag.jag_query(gi.h, q, ft, at, 10, 48, ids, dist)
    torch.cuda.synchronize()
    rid, rd, rc = O.query(ix, w.q, w.filters, w.aux, 10, 48, s0=2048, scan_cap=8192)
    assert_parity(ids.cpu().numpy(), dist.cpu().numpy(), rid, rd, "jag_query")


@pytest.mark.parametrize("case", ["label_case", "subset_case", "mixed_case"])
def test_tensor_core_scan_preselects(case, request):
    """Scan-routed queries go through the tensor-core contraction: only the
    rows within the approximation threshold get an exact distance (counter
    1), far fewer than the passing set (counter 2), and the answers are the
    oracle's exact filtered k-NN."""
    w, ix, _, gi = request.getfixturevalue(case)
    ids, dist, cnt, = jag.jag_search_host(gi.h, w.q, w.filters, w.aux, 10, 48, counters=True, s0=4000,
                                          scan_cap=8192)
    routed = np.nonzero(cnt[:, 3] == 1)[0]
    assert len(routed) > 0
    bi, bd, _, _ = O.brute_force(ix, w.q[routed], w.filters[routed], w.aux, 10)
    assert (ids[routed] == bi).all() and np.array_equal(dist[routed].view(np.uint32), bd.view(np.uint32))
    big = routed[cnt[routed, 2] > 200]
    if len(big):
        assert (cnt[big, 1] < cnt[big, 2]).mean() > 0.9
        assert cnt[big, 1].mean() < 0.5 * cnt[big, 2].mean()


def test_large_beam_rejected_where_unsupported(range_small):
    """Beams above 256 are for the plain search: a policy or the serve loop
    rejects them, and a beam above 512 is rejected everywhere."""
    w, ix, _, gi = range_small
    q = torch.from_numpy(w.q[:4]).cuda()
    with pytest.raises(jag.JagError):
        gi.search(q, w.filters[:4], w.aux, 10, 513, s0=0)
    pol = jag.Policy(jag.JAG_POLICY_FORCED, h0=4, forced=torch.zeros((4, 2), dtype=torch.int32, device="cuda"))
    with pytest.raises(jag.JagError):
        gi.search(q, w.filters[:4], w.aux, 10, 300, s0=0, policy=pol)
    with pytest.raises(jag.JagError):
        jag.Server(gi, 10, 300)


@pytest.mark.parametrize("d", [3, 7, 33, 130, 256, 700])
def test_scan_route_row_layouts(d):
    """The exact scan at dimensions that are not a multiple of the tensor
    core's K step (8 elements), that span several K passes of 128, or both:
    every query goes to the scan (about 900 passing rows each, so the
    threshold selection runs) and must equal the oracle's brute force."""
    n = 3000
    w = D.make_range_i32(n=n, d=d, nq=40, seed=40 + d, width=300)
    ox = O.Index.from_workload(w, R=16)
    gi = jag.Index.from_workload(w, R=16, graph=np.full((n, 16), -1, np.int32), entry=0)
    ids, dist, cnt = gpu_search(gi, w.q, w.filters, w.aux, 10, 32, s0=100_000, scan_cap=100_000)
    assert (cnt[:, 3] == 1).all()
    assert (cnt[:, 1] < cnt[:, 2]).mean() > 0.9          # the threshold narrowed the candidates
    bi, bd, _, _ = O.brute_force(ox, w.q, w.filters, w.aux, 10)
    assert (ids == bi).all()
    assert np.array_equal(dist.view(np.uint32), bd.view(np.uint32))
    gi.close()


def test_scan_route_large_k(range_small):
    """k above 128: every passing row is a candidate of the exact scan."""
    w, ix, _, gi = range_small
    q, f = w.q[:30], w.filters[:30]
    ids, dist, cnt = gpu_search(gi, q, f, w.aux, 200, 256, s0=100_000, scan_cap=100_000)
    assert (cnt[:, 3] == 1).all() and (cnt[:, 1] == cnt[:, 2]).all()
    bi, bd, _, _ = O.brute_force(ix, q, f, w.aux, 200)
    assert (ids == bi).all()
    assert np.array_equal(dist.view(np.uint32), bd.view(np.uint32))
