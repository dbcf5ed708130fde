"""Weight-JAG on the GPU against the oracle: the per-point weights
(w = fp32(c h), h = sigma / sigma_A) and the whole weighted build are
bit-identical; with the single weight 0 the GPU build equals the GPU
Threshold-JAG build with T = {100%} where that threshold covers every
attribute distance (labels); a search on the weighted graph matches
the oracle's."""
import numpy as np
import pytest

from oracle import jag_oracle as O
from paper_2602_10258_gb300 import datagen as D

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
jag = pytest.importorskip("paper_2602_10258_gb300.jag")

MULT = (0.0, 1.0, 10.0)


@pytest.fixture(scope="module", params=["label", "range", "float"])
def case(request):
    if request.param == "label":
        w = D.make_label_zipf(n=6000, d=32, nq=200, seed=51, n_labels=30, n_centres=10)
    elif request.param == "range":
        w = D.make_range_i32(n=6000, d=32, nq=200, seed=52)
    else:
        w = D.make_mixed(n=6000, d=48, nq=200, seed=53, n_centres=10)
    ox = O.Index.from_workload(w, R=24)
    wts, h = O.build_weighted(ox, mult=MULT, lb=48)
    return w, ox, wts


def test_weights_and_graph_match_the_oracle(case):
    w, ox, wts = case
    gi = jag.Index.from_workload(w, R=24, l_b=48, weights=MULT)
    info = gi.info()
    assert info["weighted"] == 1 and info["n_thresholds"] == len(MULT)
    gw = gi.thresholds().view(np.float32)
    assert np.array_equal(gw.view(np.uint32), wts.view(np.uint32))
    assert info["entry"] == ox.entry
    g = gi.graph()
    same = (g == ox.graph).all(1)
    assert same.all(), "rows differ: %s" % np.nonzero(~same)[0][:10]
    # the query path on the weighted graph
    q = torch.from_numpy(w.q).cuda()
    ids, dist, _ = gi.search(q, w.filters, w.aux, 10, 48, s0=0)
    torch.cuda.synchronize()
    oi, od, _ = O.query(ox, w.q, w.filters, w.aux, 10, 48)
    assert np.array_equal(ids.cpu().numpy(), oi)
    assert np.array_equal(dist.cpu().numpy().view(np.uint32), od.view(np.uint32))
    gi.close()


def test_zero_weight_equals_threshold_100(case):
    """Holds when each point's 100% threshold (the largest dist_A in its
    sample) covers every dist_A from it, so that the capped distance is 0
    everywhere: labels, where that threshold is 1."""
    w, _, _ = case
    if w.name != "label_zipf":
        pytest.skip("the sample maximum of a range attribute does not cover every distance")
    a = jag.Index.from_workload(w, R=24, l_b=48, weights=(0.0,))
    b = jag.Index.from_workload(w, R=24, l_b=48, thresholds=(100,))
    assert (b.thresholds() == 1).all()
    assert np.array_equal(a.graph(), b.graph())
    a.close()
    b.close()
