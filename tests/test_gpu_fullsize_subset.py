"""Parity at full size on the precision form's workload: N=1,000,000, d=100
from a 200-component Gaussian mixture, a 64-bit label mask per point (bit j
set with probability 0.5/(j+1)), 10,000 subset queries requiring 1-3 labels
(selectivity 1e-4..0.5), k=10, the benchmark's graph (Weight-JAG, R=64,
weights {0, 1, 5}, Hamming dist_A), rows stored as BF16 and as FP8-E4M3 with an fp32 re-rank of the
leading min(4k, beam) candidates, in the launch configuration the benchmark
times (one jag_search over the batch, s0 = scan_cap = 16,384).

The graph comes from the GPU build (equal to the oracle build bit for bit at
smaller sizes); on it, sampled queries are answered by the oracle one by one
and must match exactly, and the answer invariants are checked for every
query."""
import numpy as np
import pytest

from oracle import jag_oracle as O
from paper_2602_10258_gb300 import datagen as D

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
jag = pytest.importorskip("paper_2602_10258_gb300.jag")

N, NQ, K, S0, CAP = 1_000_000, 10_000, 10, 16384, 16384


@pytest.fixture(scope="module")
def full():
    w = D.make_subset(n=N, d=100, nq=NQ, seed=0)
    gi = jag.Index.from_workload(w, R=64, l_b=64, alpha=1.2, weights=(0, 1, 5))
    info = gi.info()
    graph = gi.graph()
    gi.close()
    return w, graph, info["entry"]


@pytest.mark.parametrize("fmt,beam", [(0, 128), (1, 128), (1, 256), (2, 256)], ids=["fp32-128", "bf16-128",
                                                                                 "bf16-256", "fp8-256"])
def test_subset_full_size_matches_oracle(full, fmt, beam):
    w, graph, entry = full
    gi = jag.Index.from_workload(w, R=64, graph=graph, entry=entry, storage=fmt)
    q = torch.from_numpy(w.q).cuda()
    ids, dist, cnt = gi.search(q, w.filters, w.aux, K, beam, counters=True, s0=S0, scan_cap=CAP)
    torch.cuda.synchronize()
    ids, dist, cnt = ids.cpu().numpy(), dist.cpu().numpy(), cnt.cpu().numpy()
    gi.close()
    assert (cnt[:, 3] == 1).any() and (cnt[:, 3] == 0).any()        # both routes taken
    ox = O.Index.from_workload(w, R=64, graph=graph, entry=entry, storage=fmt)
    sample = np.random.default_rng(31 + fmt).choice(NQ, 32, replace=False)
    rid, rd, rc = O.query(ox, w.q[sample], w.filters[sample], w.aux, K, beam, s0=S0, scan_cap=CAP)
    assert (cnt[sample, 3] == rc[:, 3]).all()
    bad = sample[~(ids[sample] == rid).all(axis=1)]
    assert len(bad) == 0, "differs on %s" % bad
    assert np.array_equal(dist[sample].view(np.uint32), rd.view(np.uint32))
    # every answer passes its filter, answers are a sorted prefix, distances are fp32-exact
    req = w.filters["payload"].astype(np.uint64)
    valid = ids >= 0
    got = w.attr_mask[np.maximum(ids, 0)]
    assert ((got & req[:, None]) == req[:, None])[valid].all()
    assert (np.diff(valid.astype(np.int8), axis=1) <= 0).all()
    dd = np.where(valid, dist, np.inf)
    assert (dd[:, 1:] >= dd[:, :-1]).all()
    for i in range(0, NQ, 211):
        v = ids[i][valid[i]]
        ref = O.dist_canon_rows(np.repeat(w.q[i:i + 1], len(v), 0), w.x[v])
        assert (ref == dist[i][valid[i]]).all()
