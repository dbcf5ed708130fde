"""The serve loop (device-resident continuous batching) on the GPU.

- Every answer equals jag_search's for the same queries and options (exact
  scan of slices and gathered lists, graph search, BF16 re-rank, learned
  policy), bit for bit.
- A request's answers are the same alone and in a mix of concurrent
  requests of other filter types and selectivities.
- Admission waits are bounded (JAG_ETIMEOUT), an idle loop exits and is
  started again, and bad boolean filters are reported, not faulted on.
"""
import numpy as np
import pytest

from paper_2602_10258_gb300 import datagen as D

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
jag = pytest.importorskip("paper_2602_10258_gb300.jag")

K, BEAM = 10, 64


@pytest.fixture(scope="module", params=["label", "subset", "mixed"])
def case(request):
    if request.param == "label":
        w = D.make_label_zipf(n=20_000, d=64, nq=600, seed=31, n_labels=60, n_centres=20)
    elif request.param == "subset":
        w = D.make_subset(n=20_000, d=48, nq=600, seed=32, n_centres=20, sel_lo=1e-3)
    else:
        w = D.make_mixed(n=20_000, d=100, nq=600, seed=33, n_centres=20)
    ix = jag.Index.from_workload(w, R=24, l_b=48)
    yield w, ix
    ix.close()


def _batch_answers(ix, w, s0, policy=None, beam=BEAM):
    q = torch.from_numpy(np.ascontiguousarray(w.q)).cuda()
    ids, dist, cnt = ix.search(q, w.filters, w.aux, K, beam, counters=True, s0=s0, policy=policy)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dist.cpu().numpy(), cnt.cpu().numpy()


def _serve_all(srv, w, sizes):
    out_i = np.empty((len(w.q), K), np.int32)
    out_d = np.empty((len(w.q), K), np.float32)
    tickets, pos = [], 0
    for s in sizes:
        tickets.append((pos, s, srv.submit(w.q[pos:pos + s], w.filters[pos:pos + s], w.aux)))
        pos += s
    for p, s, t in tickets:
        i, d, tm = srv.wait(t)
        out_i[p:p + s], out_d[p:p + s] = i, d
        assert tm["device_s"] >= 0 and tm["done_s"] >= tm["submit_s"]
    return out_i, out_d


def _sizes(n, seed):
    rng = np.random.default_rng(seed)
    sizes = []
    while sum(sizes) < n:
        sizes.append(int(min(rng.integers(1, 97), n - sum(sizes))))
    return sizes


@pytest.mark.parametrize("s0", [0, 600])
def test_serve_equals_batch_search(case, s0):
    w, ix = case
    bi, bd, bc = _batch_answers(ix, w, s0)
    if s0:
        assert bc[:, 3].sum() > 0            # some queries take the exact scan
    srv = jag.Server(ix, K, BEAM, s0=s0)
    si, sd = _serve_all(srv, w, _sizes(len(w.q), 1))
    srv.stop()
    assert np.array_equal(si, bi)
    assert np.array_equal(sd.view(np.uint32), bd.view(np.uint32))


def test_same_alone_and_in_the_mix(case):
    w, ix = case
    srv = jag.Server(ix, K, BEAM, s0=600, max_queries=4096)
    sel = slice(100, 164)
    t = srv.submit(w.q[sel], w.filters[sel], w.aux)
    alone_i, alone_d, _ = srv.wait(t)
    # the same request in the middle of a stream of others, all in flight
    rng = np.random.default_rng(7)
    tickets = []
    for j in range(40):
        if j == 20:
            mine = srv.submit(w.q[sel], w.filters[sel], w.aux)
        a = int(rng.integers(0, len(w.q) - 96))
        b = a + int(rng.integers(1, 96))
        tickets.append(srv.submit(w.q[a:b], w.filters[a:b], w.aux))
    mix_i, mix_d, _ = srv.wait(mine)
    for t in tickets:
        srv.wait(t)
    srv.stop()
    assert np.array_equal(alone_i, mix_i)
    assert np.array_equal(alone_d.view(np.uint32), mix_d.view(np.uint32))


def test_replay_answers_and_latencies(case):
    w, ix = case
    bi, bd, _ = _batch_answers(ix, w, 600)
    sizes = np.array(_sizes(len(w.q), 3), np.int32)
    first = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    arrival = np.cumsum(np.random.default_rng(4).exponential(2e-4, len(sizes)))
    srv = jag.Server(ix, K, BEAM, s0=600)
    ids, dist, lat, dev = srv.replay(arrival, sizes, first, w.q, w.filters, w.aux)
    srv.stop()
    assert np.array_equal(ids, bi) and np.array_equal(dist.view(np.uint32), bd.view(np.uint32))
    assert (lat > 0).all() and (dev >= 0).all() and (dev <= lat + 1e-3).all()


def test_small_query_map_with_out_of_order_completion(case):
    # a 128-entry query map, a burst of requests mixing exact scans (quick)
    # and graph searches (slow): requests complete out of order, admission
    # waits for the map's window, and most warps hold tickets ahead of the
    # published count; every answer must still be the batch path's
    w, ix = case
    bi, bd, _ = _batch_answers(ix, w, 600)
    rng = np.random.default_rng(11)
    n_req = 300
    sizes = rng.integers(1, 49, n_req).astype(np.int32)
    first = np.array([rng.integers(0, len(w.q) - s + 1) for s in sizes], np.int64)
    arrival = np.cumsum(rng.exponential(2e-6, n_req))
    srv = jag.Server(ix, K, BEAM, s0=600, max_queries=128)
    ids, dist, lat, dev = srv.replay(arrival, sizes, first, w.q, w.filters, w.aux, timeout_s=60.0)
    info = srv.info()
    srv.stop()
    assert info["queries_done"] == int(sizes.sum())
    for f, sz in zip(first, sizes):
        assert np.array_equal(ids[f:f + sz], bi[f:f + sz])
        assert np.array_equal(dist[f:f + sz].view(np.uint32), bd[f:f + sz].view(np.uint32))


def test_admission_timeout_and_unknown_ticket(case):
    w, ix = case
    srv = jag.Server(ix, K, BEAM, max_queries=64)
    t = srv.submit(w.q[:64], w.filters[:64], w.aux)
    with pytest.raises(jag.JagError) as e:
        srv.submit(w.q[:1], w.filters[:1], w.aux, timeout_s=0.05)    # room frees only on wait
    assert e.value.status == jag.JAG_ETIMEOUT
    with pytest.raises(jag.JagError) as e:
        srv.submit(w.q[:65], w.filters[:65], w.aux)                  # can never fit
    assert e.value.status == jag.JAG_EINVAL
    srv.wait(t)
    t2 = srv.submit(w.q[:1], w.filters[:1], w.aux, timeout_s=0.05)
    srv.wait(t2)
    with pytest.raises(jag.JagError) as e:
        jag._check(jag.load().jag_serve_wait(srv.h, 987654, None, None, None, 0.0))
    assert e.value.status == jag.JAG_EINVAL
    srv.stop()


def test_idle_exit_and_restart(case):
    import time
    w, ix = case
    bi, bd, _ = _batch_answers(ix, w, 0)
    srv = jag.Server(ix, K, BEAM, s0=0, idle_exit_s=0.02)
    i1, _, _ = srv.wait(srv.submit(w.q[:32], w.filters[:32], w.aux))
    time.sleep(0.2)                       # the loop exits after 20 ms without work
    i2, d2, _ = srv.wait(srv.submit(w.q[32:64], w.filters[32:64], w.aux))
    info = srv.info()
    srv.stop()
    assert info["launches"] >= 2 and info["queries_done"] == 64
    assert np.array_equal(i1, bi[:32]) and np.array_equal(i2, bi[32:64])


def test_bad_boolean_filter_is_reported():
    w = D.make_mixed(n=5_000, d=32, nq=40, seed=34, n_centres=5)
    ix = jag.Index.from_workload(w, R=16, l_b=32)
    f = w.filters.copy()
    b = np.nonzero(f["kind"] == D.F_BOOL)[0][0]
    f["aux_off"][b] = len(w.aux) + 64            # table outside the buffer
    srv = jag.Server(ix, K, 32, s0=0)
    ids, dist, tm = srv.wait(srv.submit(w.q, f, w.aux))
    srv.stop()
    ix.close()
    assert tm["status"] & 4
    assert (ids[b] == -1).all() and np.isinf(dist[b]).all()
    ok = np.arange(len(f)) != b
    assert (ids[ok, 0] >= 0).any()


@pytest.mark.parametrize("storage", [1, 2])
def test_serve_low_precision_rows(storage):
    w = D.make_mixed(n=20_000, d=100, nq=300, seed=35, n_centres=20)
    ix = jag.Index.from_workload(w, R=24, l_b=48, storage=storage)
    bi, bd, _ = _batch_answers(ix, w, 600)
    srv = jag.Server(ix, K, BEAM, s0=600)
    si, sd = _serve_all(srv, w, _sizes(len(w.q), 5))
    srv.stop()
    ix.close()
    assert np.array_equal(si, bi) and np.array_equal(sd.view(np.uint32), bd.view(np.uint32))


def test_serve_learned_policy(case):
    w, ix = case
    theta = D.mlp_init_params(len(jag.LADDER), seed=3)
    theta[-1] = 0.6
    pol = jag.Policy.learned(torch.from_numpy(theta).cuda(), h0=6, tau=0.2)
    torch.cuda.synchronize()
    bi, bd, _ = _batch_answers(ix, w, 600, policy=pol, beam=128)
    srv = jag.Server(ix, K, 128, s0=600, policy=pol)
    si, sd = _serve_all(srv, w, _sizes(len(w.q), 6))
    srv.stop()
    assert np.array_equal(si, bi) and np.array_equal(sd.view(np.uint32), bd.view(np.uint32))
