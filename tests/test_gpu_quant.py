"""GPU parity of the low-precision storage: the device quantizer against the
oracle's format-definition converters (byte for byte), and BF16 / FP8 search
with the fp32 re-rank against the oracle's search on the same graph and the
same stored rows (bit-identical answers)."""
import numpy as np
import pytest

from oracle import jag_oracle as O
from paper_2602_10258_gb300 import datagen as D

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
jag = pytest.importorskip("paper_2602_10258_gb300.jag")

FMTS = [(jag.JAG_VEC_BF16, O.FMT_BF16), (jag.JAG_VEC_FP8, O.FMT_FP8)]


@pytest.mark.parametrize("gfmt,ofmt", FMTS)
@pytest.mark.parametrize("d", [5, 100, 128, 200])
def test_quantizer_matches_oracle(gfmt, ofmt, d):
    rng = np.random.default_rng(d)
    n = 3000
    x = (rng.standard_normal((n, d)) * np.exp(rng.uniform(-8, 8, (n, 1)))).astype(np.float32)
    x[0] = 0.0
    x[1, :] = 448.0
    x[2, :3] = [1e-30, -3e-39, 7.0]        # tiny and subnormal fp32 values
    gi = jag.Index(x, attr_i32=np.zeros(n, np.int32), R=4, graph=np.full((n, 4), -1, np.int32), storage=gfmt)
    rows, sc = gi.stored_rows()
    orows, osc = O.quantize(x, ofmt)
    assert rows.shape == orows.shape
    assert (sc == osc).all()
    bad = np.nonzero((rows != orows).any(axis=1))[0]
    assert len(bad) == 0, "rows differ: %s" % bad[:5]


@pytest.fixture(scope="module")
def quant_cases():
    out = {}
    w = D.make_mixed(n=15_000, d=100, nq=300, seed=31, n_centres=20)
    ix = O.Index.from_workload(w, R=32)
    O.build(ix, lb=64)
    out["mixed"] = (w, ix)
    w2 = D.make_label_zipf(n=15_000, d=128, nq=300, seed=32, n_labels=50, n_centres=20)
    ix2 = O.Index.from_workload(w2, R=24)
    O.build(ix2, lb=48)
    out["label"] = (w2, ix2)
    return out


@pytest.mark.parametrize("gfmt,ofmt", FMTS)
@pytest.mark.parametrize("case", ["mixed", "label"])
@pytest.mark.parametrize("beam,s0", [(16, 0), (64, 0), (64, 400), (200, 0)])
def test_quantized_search_matches_oracle(quant_cases, case, gfmt, ofmt, beam, s0):
    w, ix = quant_cases[case]
    ox = O.Index.from_workload(w, R=ix.R, graph=ix.graph, entry=ix.entry, storage=ofmt)
    gi = jag.Index.from_workload(w, R=ix.R, graph=ix.graph, entry=ix.entry, storage=gfmt)
    rid, rd, rc = O.query(ox, w.q, w.filters, w.aux, 10, beam, s0=s0, scan_cap=8192)
    qt = torch.from_numpy(w.q).cuda()
    ids, dist, cnt = gi.search(qt, w.filters, w.aux, 10, beam, counters=True, s0=s0)
    torch.cuda.synchronize()
    ids, dist, cnt = ids.cpu().numpy(), dist.cpu().numpy(), cnt.cpu().numpy()
    same = (ids == rid).all(axis=1)
    assert same.mean() >= 0.999, np.nonzero(~same)[0][:5]
    assert (dist[same] == rd[same]).all()
    assert (cnt[:, 3] == rc[:, 3]).all()
    assert (cnt[cnt[:, 3] == 0, 0] == rc[rc[:, 3] == 0, 0]).all()   # same trajectories


@pytest.mark.parametrize("gfmt,ofmt", FMTS)
def test_quantized_answers_are_fp32_exact(quant_cases, gfmt, ofmt):
    w, ix = quant_cases["label"]
    gi = jag.Index.from_workload(w, R=ix.R, graph=ix.graph, entry=ix.entry, storage=gfmt)
    ids, dist, _ = gi.search_host(w.q, w.filters, w.aux, 10, 64, s0=0)
    for i in range(0, len(ids), 7):
        m = ids[i] >= 0
        ref = O.dist_canon_rows(np.repeat(w.q[i:i + 1], m.sum(), 0), w.x[ids[i][m]])
        assert (ref == dist[i][m]).all()
