"""A GPU build in which one vertex (a hub) receives more back-edges in a
single insertion batch than the prune's fixed candidate arrays hold: points
on the unit sphere (d = 256, so that they are nearly orthogonal: squared
distance about 2 between them, 1 to the origin) plus one point at the
origin, the nearest neighbour of every other point.  With 500,000 points the last batches insert 10,000
points each, and every one of them links to the origin.  The build must
succeed and give a valid graph (the prune of an oversized set runs with
arrays sized for it), and the search on it must work."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
jag = pytest.importorskip("paper_2602_10258_gb300.jag")


def test_hub_with_more_back_edges_than_the_fixed_arrays():
    n, d, R = 500_000, 256, 32
    rng = np.random.default_rng(5)
    x = rng.standard_normal((n, d)).astype(np.float32)
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    x[0] = 0.0
    attr = rng.integers(0, 100, n).astype(np.int32)
    ix = jag.Index(x, attr_i32=attr, dist_a=jag.JAG_F_RANGE_I32, R=R, l_b=32, thresholds=(100,))
    g = ix.graph()
    assert g.shape == (n, R)
    valid = g >= 0
    assert (g[valid] < n).all()
    assert not (g == np.arange(n)[:, None]).any()                 # no self-loops
    s = np.sort(np.where(valid, g, -1 - np.arange(R)[None, :]), axis=1)
    assert not (np.diff(s, axis=1) == 0).any()                    # no duplicates
    assert valid.sum(1).min() >= 1
    # nearly every point links to the origin, so each of the last batches
    # (10,000 points) sent it more back-edges than the fixed arrays hold
    assert (g == 0).any(axis=1).sum() >= 0.9 * n
    # the origin is everyone's nearest neighbour: an unfiltered query at a
    # base point finds it among its answers
    q = torch.from_numpy(x[1:201].copy()).cuda()
    from paper_2602_10258_gb300 import datagen as D
    f = D.filters_range_i32(np.zeros(200, np.int32), np.full(200, 99, np.int32))
    ids, dist, _ = ix.search(q, f, None, 10, 64, s0=0)
    torch.cuda.synchronize()
    ids = ids.cpu().numpy()
    assert (ids == 0).any(axis=1).mean() > 0.95
    ix.close()
