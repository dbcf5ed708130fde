"""GPU parity of the learned search policy and of the network's training
kernels against the CPU oracle.

- Search with a FORCED or LEARNED policy: answers, per-query decisions
  (beam, stop hop, last hop that changed the first k entries, learned flag)
  and the 12 features are bit-identical to the oracle's on the same graph.
- jag_mlp_loss_grad against the FP64 back-propagation of the oracle, within
  the fp32 rounding bound stated below; jag_mlp_export against the oracle's
  BF16 encoding (bit-exact); jag_mlp_train repeats bit for bit and lowers the
  loss.
"""
import numpy as np
import pytest

from oracle import jag_mlp as M
from oracle import jag_oracle as O
from paper_2602_10258_gb300 import datagen as D

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
jag = pytest.importorskip("paper_2602_10258_gb300.jag")

LADDER = (16, 24, 32, 48, 64, 96, 128, 192, 256)
NL = len(LADDER)


def _gpu_policy_search(gi, w, k, ls, pol):
    qt = torch.from_numpy(np.ascontiguousarray(w.q, np.float32)).cuda()
    ids, dist, cnt = gi.search(qt, w.filters, w.aux, k, ls, counters=True, s0=0, policy=pol)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dist.cpu().numpy(), cnt.cpu().numpy()


def _assert_same(gpu, ora, gpol, opol):
    gi, gd, gc = gpu
    oi, od, oc = ora
    assert (gi == oi).all(), np.nonzero(~(gi == oi).all(1))[0][:5]
    assert np.array_equal(gd.view(np.uint32), od.view(np.uint32))
    assert (gc[:, 0] == oc[:, 0]).all()                                   # hops
    assert (gpol.decisions.cpu().numpy() == opol.decisions).all()
    assert np.array_equal(gpol.features.cpu().numpy().view(np.uint32), opol.features.view(np.uint32))


@pytest.fixture(scope="module", params=["label", "mixed"])
def case(request):
    if request.param == "label":
        w = D.make_label_zipf(n=20_000, d=64, nq=400, seed=21, n_labels=60, n_centres=20)
        ix = O.Index.from_workload(w, R=24)
        O.build(ix, lb=48)
    else:
        w = D.make_mixed(n=20_000, d=100, nq=400, seed=22, n_centres=20)
        ix = O.Index.from_workload(w, R=32)
        O.build(ix, lb=64)
    return w, ix


def _gpu_index(w, ix, storage=0):
    return jag.Index.from_workload(w, R=ix.R, graph=ix.graph, entry=ix.entry, storage=storage)


@pytest.mark.parametrize("h0", [1, 6])
def test_forced_policy_parity(case, h0):
    w, ix = case
    nq = len(w.q)
    rng = np.random.default_rng(h0)
    forced = np.stack([rng.choice([0, 4, 10, 12, 40, 100, 128, 300], nq),
                       rng.choice([0, 0, 3, 20, 60, 400], nq)], axis=1).astype(np.int32)
    k, ls = 10, 128
    opol = O.Policy(O.POL_FORCED, h0=h0, forced=forced, nq=nq, want_features=True, want_decisions=True)
    ora = O.query_policy(ix, w.q, w.filters, w.aux, k, ls, opol)
    gi = _gpu_index(w, ix)
    gpol = jag.Policy(jag.JAG_POLICY_FORCED, h0=h0, forced=torch.from_numpy(forced).cuda(),
                      features=torch.zeros((nq, 12), dtype=torch.float32, device="cuda"),
                      decisions=torch.zeros((nq, 4), dtype=torch.int32, device="cuda"))
    _assert_same(_gpu_policy_search(gi, w, k, ls, gpol), ora, gpol, opol)
    # beams outside [k, l_s] are taken into it
    assert (opol.decisions[forced[:, 0] == 300, 0] == ls).all()
    assert (opol.decisions[forced[:, 0] == 4, 0] == k).all()
    gi.close()


@pytest.mark.parametrize("tau,seed,scale", [(0.0, 3, 64.0), (0.4, 4, 64.0), (float("inf"), 5, 64.0), (0.0, 6, 0.0)])
@pytest.mark.parametrize("storage", [0, 1])
def test_learned_policy_parity(case, tau, seed, scale, storage):
    w, ix = case
    nq = len(w.q)
    theta = M.init_params(NL, seed=seed)
    theta[-1] = 0.5            # stop output bias: a stop hop of ~32 at scale 64
    theta = theta.astype(np.float32)
    k, ls = 10, 160
    oix = ix if storage == 0 else O.Index.from_workload(w, R=ix.R, graph=ix.graph, entry=ix.entry, storage=storage)
    opol = O.Policy(O.POL_LEARNED, h0=5, theta=theta, ladder=LADDER, tau=tau, stop_scale=scale, nq=nq,
                    want_features=True, want_decisions=True)
    ora = O.query_policy(oix, w.q, w.filters, w.aux, k, ls, opol)
    gi = _gpu_index(w, ix, storage)
    params = torch.from_numpy(theta).cuda()
    gpol = jag.Policy.learned(params, ladder=LADDER, h0=5, tau=tau, stop_scale=scale,
                              features=torch.zeros((nq, 12), dtype=torch.float32, device="cuda"),
                              decisions=torch.zeros((nq, 4), dtype=torch.int32, device="cuda"))
    _assert_same(_gpu_policy_search(gi, w, k, ls, gpol), ora, gpol, opol)
    dec = opol.decisions
    if tau == float("inf"):
        assert (dec[:, 3] == 0).all()
    elif tau == 0.0:
        assert dec[:, 3].mean() > 0.9          # the network decides (almost) always
    if scale == 0.0:
        assert (dec[:, 1] == 0).all()
    gi.close()


@pytest.mark.parametrize("tau,seed,scale,h0", [(0.0, 3, 64.0, 5), (0.4, 4, 48.0, 1), (0.0, 6, 0.0, 7),
                                               (0.0, 7, 64.0, 300)])
@pytest.mark.parametrize("storage", [0, 1, 2])
@pytest.mark.parametrize("want_features", [False, True])
def test_learned_policy_without_trace(case, tau, seed, scale, h0, storage, want_features):
    """Without a trace (no decisions requested) the policy search takes the
    kernel that does not track the last change of the first k entries;
    answers, hop counts and features are the oracle's (h0 = 300 lies past
    every search's end)."""
    w, ix = case
    nq = len(w.q)
    theta = M.init_params(NL, seed=seed)
    theta[-1] = 0.5
    theta = theta.astype(np.float32)
    k, ls = 10, 160
    oix = ix if storage == 0 else O.Index.from_workload(w, R=ix.R, graph=ix.graph, entry=ix.entry, storage=storage)
    opol = O.Policy(O.POL_LEARNED, h0=h0, theta=theta, ladder=LADDER, tau=tau, stop_scale=scale, nq=nq,
                    want_features=True, want_decisions=True)
    oi, od, oc = O.query_policy(oix, w.q, w.filters, w.aux, k, ls, opol)
    gi = _gpu_index(w, ix, storage)
    feats = torch.full((nq, 12), 7.0, dtype=torch.float32, device="cuda") if want_features else None
    gpol = jag.Policy.learned(torch.from_numpy(theta).cuda(), ladder=LADDER, h0=h0, tau=tau, stop_scale=scale,
                              features=feats)
    gids, gd, gc = _gpu_policy_search(gi, w, k, ls, gpol)
    assert (gids == oi).all(), np.nonzero(~(gids == oi).all(1))[0][:5]
    assert np.array_equal(gd.view(np.uint32), od.view(np.uint32))
    assert (gc[:, 0] == oc[:, 0]).all()
    if want_features:
        assert np.array_equal(feats.cpu().numpy().view(np.uint32), opol.features.view(np.uint32))
    if h0 < 100 and scale > 0 and tau == 0.0:
        assert (opol.decisions[:, 1] > 0).any()      # some searches stop early
    gi.close()


def test_policy_plain_mode_is_the_plain_search(case):
    w, ix = case
    gi = _gpu_index(w, ix)
    qt = torch.from_numpy(np.ascontiguousarray(w.q, np.float32)).cuda()
    a = gi.search(qt, w.filters, w.aux, 10, 40, s0=0)
    b = gi.search(qt, w.filters, w.aux, 10, 40, s0=0, policy=jag.Policy(jag.JAG_POLICY_PLAIN))
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    gi.close()


# ---------------------------------------------------------------------------
# network training kernels
# ---------------------------------------------------------------------------

def _batch(m, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((m, 12)).astype(np.float32)
    y = rng.integers(0, NL, m).astype(np.int32)
    t = rng.uniform(0, 3, m).astype(np.float32)
    return X, y, t


@pytest.mark.parametrize("m", [1, 64, 1000])
def test_loss_grad_against_fp64_backprop(m):
    """Tolerance: every gradient entry is a sum over the m rows of products of
    quantities each computed by fp32 dot products of length <= 64 from
    operands of magnitude O(1); each carries a relative error below
    (64 + m / 64 + 64) * 2^-24 < 1e-5 of the sum of the magnitudes of its
    terms, which is below 10x the largest entry of the gradient for these
    inputs -- hence 1e-4 of the largest entry, with a 1e-7 floor."""
    X, y, t = _batch(m, m)
    theta = (M.init_params(NL, seed=1) + 0.05 * np.random.default_rng(2).standard_normal(M.n_params(NL)))
    theta32 = theta.astype(np.float32)
    ref_loss = M.loss(theta32.astype(np.float64), X, y, t, NL, 0.3)
    ref = M.grad(theta32.astype(np.float64), X, y, t, NL, 0.3)
    loss, g = jag.mlp_loss_grad(NL, torch.from_numpy(theta32).cuda(), torch.from_numpy(X).cuda(),
                                torch.from_numpy(y).cuda(), torch.from_numpy(t).cuda(), 0.3)
    g = g.cpu().numpy().astype(np.float64)
    assert abs(float(loss.item()) - ref_loss) <= 1e-5 * abs(ref_loss)
    assert np.abs(g - ref).max() <= 1e-4 * np.abs(ref).max() + 1e-7


def test_bad_class_makes_the_loss_nan():
    X, y, t = _batch(70, 7)
    y[65] = NL
    theta = M.init_params(NL, seed=1).astype(np.float32)
    loss, _ = jag.mlp_loss_grad(NL, torch.from_numpy(theta).cuda(), torch.from_numpy(X).cuda(),
                                torch.from_numpy(y).cuda(), torch.from_numpy(t).cuda(), 0.3)
    assert np.isnan(loss.item())


def test_export_is_the_bf16_encoding():
    theta = (M.init_params(NL, seed=8) * 3).astype(np.float32)
    w_ref, b_ref = O.split_params(theta, NL)
    pol = jag.Policy.learned(torch.from_numpy(theta).cuda(), ladder=LADDER)
    assert np.array_equal(pol.w_bf16.cpu().numpy().view(np.uint16), w_ref)
    assert np.array_equal(pol.b_f32.cpu().numpy(), b_ref)


def test_training_repeats_and_lowers_the_loss():
    X, y, t = _batch(3000, 9)
    y = (X[:, 0] > 0).astype(np.int32) * 3 + (X[:, 1] > 0).astype(np.int32)   # learnable classes
    t = (0.5 * X[:, 2] + 1).astype(np.float32)
    Xd, yd, td = (torch.from_numpy(a).cuda() for a in (X, y, t))
    theta = M.init_params(NL, seed=4).astype(np.float32)
    runs = []
    for _ in range(2):
        p = torch.from_numpy(theta.copy()).cuda()
        tr = jag.Trainer(NL, p)
        trace = tr.run(Xd, yd, td, epochs=20, batch=256, lr=3e-3, lam=0.5)
        runs.append((p.cpu().numpy(), trace, tr.step.value))
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    assert runs[0][2] == 20 * 12
    trace = runs[0][1]
    assert trace[-1] < 0.3 * trace[0]
    # the trained parameters' loss, by the FP64 oracle
    assert M.loss(runs[0][0].astype(np.float64), X, y, t, NL, 0.5) < 0.3 * M.loss(theta.astype(np.float64), X, y, t,
                                                                                   NL, 0.5)
