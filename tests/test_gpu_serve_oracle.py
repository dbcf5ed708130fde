"""The serve loop against the oracle itself (not against jag_search).

The loop inlines its own routing, exact scan (label / range slices of the
sorted columns, gathered subset / boolean passing sets), graph search, fp32
re-rank of BF16 / FP8 rows and policy search.  Here each of those is compared
bit for bit with the oracle's Query (Algorithm 2, with the pre-filter scan
below s0) on the same graph: requests of mixed sizes go through the loop, and
every answer must equal O.query / O.query_policy with the same k, beam, s0
and scan_cap."""
import numpy as np
import pytest

from oracle import jag_mlp as M
from oracle import jag_oracle as O
from paper_2602_10258_gb300 import datagen as D

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
jag = pytest.importorskip("paper_2602_10258_gb300.jag")

K, BEAM, S0, CAP = 10, 64, 600, 4096


@pytest.fixture(scope="module", params=["label", "subset", "mixed"])
def case(request):
    if request.param == "label":
        w = D.make_label_zipf(n=20_000, d=64, nq=500, seed=41, n_labels=60, n_centres=20)
        ix = O.Index.from_workload(w, R=24)
        O.build(ix, lb=48)
    elif request.param == "subset":
        w = D.make_subset(n=20_000, d=48, nq=500, seed=42, n_centres=20, sel_lo=1e-3)
        ix = O.Index.from_workload(w, R=24)
        O.build(ix, lb=48)
    else:
        w = D.make_mixed(n=20_000, d=100, nq=500, seed=43, n_centres=20)
        ix = O.Index.from_workload(w, R=24)
        O.build(ix, lb=48)
    return request.param, w, ix


def _sizes(n, seed):
    rng = np.random.default_rng(seed)
    sizes = []
    while sum(sizes) < n:
        sizes.append(int(min(rng.integers(1, 97), n - sum(sizes))))
    return sizes


def _serve_all(srv, w, sizes):
    out_i = np.empty((len(w.q), K), np.int32)
    out_d = np.empty((len(w.q), K), np.float32)
    tickets, pos = [], 0
    for s in sizes:
        tickets.append((pos, s, srv.submit(w.q[pos:pos + s], w.filters[pos:pos + s], w.aux)))
        pos += s
    for p, s, t in tickets:
        i, d, _ = srv.wait(t)
        out_i[p:p + s], out_d[p:p + s] = i, d
    return out_i, out_d


def _assert_same(si, sd, oi, od):
    bad = np.nonzero(~(si == oi).all(axis=1))[0]
    assert len(bad) == 0, "queries %s differ" % bad[:8]
    assert np.array_equal(sd.view(np.uint32), od.view(np.uint32))


@pytest.mark.parametrize("storage", [0, 1, 2], ids=["fp32", "bf16", "fp8"])
def test_serve_loop_equals_oracle_query(case, storage):
    name, w, ix = case
    ox = ix if storage == 0 else O.Index.from_workload(w, R=ix.R, graph=ix.graph, entry=ix.entry, storage=storage)
    oi, od, oc = O.query(ox, w.q, w.filters, w.aux, K, BEAM, s0=S0, scan_cap=CAP)
    routed = oc[:, 3] == 1
    assert routed.any() and (~routed).any()        # both the scan and the graph route are taken
    gi = jag.Index.from_workload(w, R=ix.R, graph=ix.graph, entry=ix.entry, storage=storage)
    srv = jag.Server(gi, K, BEAM, s0=S0, scan_cap=CAP)
    si, sd = _serve_all(srv, w, _sizes(len(w.q), 5 + storage))
    srv.stop()
    gi.close()
    _assert_same(si, sd, oi, od)


def test_serve_loop_learned_policy_equals_oracle(case):
    """BF16 rows with a learned beam / stop policy, scan route on."""
    name, w, ix = case
    nl = len(jag.LADDER)
    theta = M.init_params(nl, seed=13)
    theta[-1] = 0.5                                  # stop output near 32 hops at scale 64
    theta = theta.astype(np.float32)
    ox = O.Index.from_workload(w, R=ix.R, graph=ix.graph, entry=ix.entry, storage=1)
    opol = O.Policy(O.POL_LEARNED, h0=4, theta=theta, tau=0.0, stop_scale=64.0, nq=len(w.q), want_decisions=True)
    oi, od, oc = O.query_policy(ox, w.q, w.filters, w.aux, K, BEAM, opol, s0=S0, scan_cap=CAP)
    graph_q = oc[:, 3] == 0
    assert (opol.decisions[graph_q, 3] == 1).mean() > 0.9          # the network decides
    gi = jag.Index.from_workload(w, R=ix.R, graph=ix.graph, entry=ix.entry, storage=1)
    pol = jag.Policy.learned(torch.from_numpy(theta).cuda(), h0=4, tau=0.0, stop_scale=64.0)
    srv = jag.Server(gi, K, BEAM, s0=S0, scan_cap=CAP, policy=pol)
    si, sd = _serve_all(srv, w, _sizes(len(w.q), 9))
    srv.stop()
    gi.close()
    _assert_same(si, sd, oi, od)
