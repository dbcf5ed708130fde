"""The no-allocation search entry point against the regular one.

jag_search_noalloc runs the same search as jag_search, but keeps its scratch
in a fixed device area that the library puts in place when it builds an
index. It is for callers that cannot allocate device memory while they
search: a serving thread that must not wait for cudaMalloc, a process whose
device memory belongs to its own allocator, a deployment that forbids
allocation after start-up.  Here both entry points are called through the C
ABI on the same index and inputs, twice in a row with different batches (the
shared area keeps the previous call's contents, which must not leak into the
next answers), for fp32, BF16 and FP8 rows (the BF16 / FP8 re-rank ids live in
the area too) and for a learned policy; the answers must agree within the
parity tolerance (they are in fact identical).  A repeated call must leave
the device's free memory and torch's allocator unchanged.  This file sorts
last, so that a stop at the first failure has already run every other test;
it also passes when run on its own."""
import gc

import numpy as np
import pytest

from oracle import jag_mlp as M
from oracle import jag_oracle as O
from paper_2602_10258_gb300 import datagen as D

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
jag = pytest.importorskip("paper_2602_10258_gb300.jag")

RTOL = 1e-5


@pytest.fixture(scope="module")
def workload():
    w = D.make_mixed(n=8_000, d=100, nq=400, seed=21, n_centres=10)
    ix = O.Index.from_workload(w, R=24)
    O.build(ix, lb=48)
    return w, ix


@pytest.fixture(scope="module", params=[0, 1, 2], ids=["fp32", "bf16", "fp8"])
def index_and_inputs(request, workload):
    w, ix = workload
    gi = jag.Index.from_workload(w, R=24, graph=ix.graph, entry=ix.entry, storage=request.param)
    dev = torch.device("cuda", 0)
    q = torch.from_numpy(w.q).to(dev)
    f = jag.filters_to_device(w.filters, dev)
    aux = jag.aux_to_device(w.aux, dev)
    yield w, gi, q, f, aux
    gi.close()


def _outputs(nq, k, dev):
    ids = torch.full((nq, k), -7, dtype=torch.int32, device=dev)
    dist = torch.full((nq, k), -7.0, dtype=torch.float32, device=dev)
    cnt = torch.zeros((nq, 4), dtype=torch.int32, device=dev)
    return ids, dist, cnt


def _run(fn, gi, q, f, aux, k, beam, s0, scan_cap, policy=None, out=None):
    ids, dist, cnt = out if out is not None else _outputs(q.shape[0], k, q.device)
    fn(gi.h, q, f, aux, k, beam, ids, dist, cnt, None, s0=s0, scan_cap=scan_cap, policy=policy)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dist.cpu().numpy(), cnt.cpu().numpy()


def _same(a, b):
    ia, da, ca = a
    ib, db, cb = b
    assert (ia == ib).all()
    m = ia >= 0
    np.testing.assert_allclose(da[m], db[m], rtol=RTOL)
    assert np.isinf(da[~m]).all() and np.isinf(db[~m]).all()
    assert (ca[:, 3] == cb[:, 3]).all()


def test_noalloc_matches_regular_search_twice(index_and_inputs):
    w, gi, q, f, aux = index_and_inputs
    # two different batches in a row, so the second call sees the first's leftovers
    for lo, hi, beam in ((0, 400, 64), (100, 250, 32)):
        qs, fs = q[lo:hi], f[lo * 16:hi * 16]      # filter records are 16 bytes each
        ref = _run(jag.jag_search, gi, qs, fs, aux, 10, beam, 300, 1024)
        got = _run(jag.jag_search_noalloc, gi, qs, fs, aux, 10, beam, 300, 1024)
        _same(got, ref)
        assert (got[2][:, 3] == 1).any() and (got[2][:, 3] == 0).any()   # both routes used


def test_noalloc_with_learned_policy(index_and_inputs):
    w, gi, q, f, aux = index_and_inputs
    nl = len(jag.LADDER)
    theta = M.init_params(nl, seed=9)
    theta[-1] = 0.5                        # a stop hop near 32 at stop scale 64
    pol = jag.Policy.learned(torch.from_numpy(theta.astype(np.float32)).cuda(), h0=5, tau=0.0, stop_scale=64.0)
    for lo, hi in ((0, 300), (50, 400)):
        qs, fs = q[lo:hi], f[lo * 16:hi * 16]
        ref = _run(jag.jag_search, gi, qs, fs, aux, 10, 96, 300, 1024, policy=pol)
        got = _run(jag.jag_search_noalloc, gi, qs, fs, aux, 10, 96, 300, 1024, policy=pol)
        _same(got, ref)


def test_repeated_call_allocates_nothing(index_and_inputs):
    w, gi, q, f, aux = index_and_inputs
    out = _outputs(q.shape[0], 10, q.device)
    _run(jag.jag_search_noalloc, gi, q, f, aux, 10, 64, 300, 1024, out=out)     # warm-up: loads kernel code
    gc.collect()                     # earlier tests' garbage must not be freed inside the measured window
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0, reserved0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    ids, dist, cnt = out
    jag.jag_search_noalloc(gi.h, q, f, aux, 10, 64, ids, dist, cnt, None, s0=300, scan_cap=1024)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == reserved0


def test_noalloc_rejects_oversized_calls(index_and_inputs):
    w, gi, q, f, aux = index_and_inputs
    ids = torch.empty((q.shape[0], 10), dtype=torch.int32, device=q.device)
    dist = torch.empty((q.shape[0], 10), dtype=torch.float32, device=q.device)
    with pytest.raises(jag.JagError) as e:
        # 400 queries x 16384 candidate slots x 4 bytes > the fixed area
        jag.jag_search_noalloc(gi.h, q, f, aux, 10, 64, ids, dist, s0=300, scan_cap=16384)
    assert e.value.status == jag.JAG_EINVAL
    assert "scratch" in str(e.value)
