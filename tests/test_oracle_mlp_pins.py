"""Pins of the learned search policy's oracle: the FP64 back-propagation
against finite differences, the BF16 inference against the FP64 forward pass,
and the policy search's special cases that reduce to the plain search."""
import numpy as np
import pytest

from oracle import jag_mlp as M
from oracle import jag_oracle as O
from paper_2602_10258_gb300 import datagen as D

NL = 9


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = M.init_params(NL, seed=1) + 0.01 * rng.standard_normal(M.n_params(NL))
    X = rng.standard_normal((37, M.NFEAT))
    y = rng.integers(0, NL, 37)
    t = rng.standard_normal(37)
    g = M.grad(theta, X, y, t, NL, 0.3)
    idx = rng.choice(len(theta), 300, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (M.loss(theta + e, X, y, t, NL, 0.3) - M.loss(theta - e, X, y, t, NL, 0.3)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_loss_special_cases():
    # zero weights: uniform logits -> cross-entropy log(nl); stop output 0
    theta = np.zeros(M.n_params(NL))
    X = np.ones((5, M.NFEAT))
    y = np.arange(5)
    t = np.full(5, 2.0)
    assert np.isclose(M.loss(theta, X, y, t, NL, 1.0), np.log(NL) + 4.0)


def test_bf16_inference_matches_fp64_forward():
    rng = np.random.default_rng(2)
    theta = M.init_params(NL, seed=3).astype(np.float32)
    pol = O.Policy(O.POL_LEARNED, theta=theta)
    # the same BF16-rounded weights, fp64 arithmetic
    w_codes, b = O.split_params(theta, NL)
    w = (w_codes.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    h, f = 64, 12
    tq = np.concatenate([w[:h * f], b[:h], w[h * f:h * f + h * h], b[h:2 * h], w[h * f + h * h:], b[2 * h:]])
    X = rng.standard_normal((200, 12)).astype(np.float32)
    out = O.mlp_infer(pol, X)
    ref, _ = M.forward(tq, X, NL)
    scale = np.abs(ref).max() + 1.0
    assert np.abs(out - ref).max() <= 1e-4 * scale


@pytest.fixture(scope="module")
def small():
    w = D.make_label_zipf(n=4000, d=16, nq=60, seed=5, n_labels=20, n_centres=10)
    ix = O.Index.from_workload(w, R=16)
    O.build(ix, lb=32)
    return w, ix


def test_forced_fixed_beam_is_the_plain_search(small):
    w, ix = small
    ls = 48
    ids, dist, cnt = O.query(ix, w.q, w.filters, w.aux, 10, ls)
    forced = np.tile(np.array([[ls, 0]], np.int32), (len(w.q), 1))
    pol = O.Policy(O.POL_FORCED, h0=8, forced=forced, nq=len(w.q), want_decisions=True)
    pi, pd, pc = O.query_policy(ix, w.q, w.filters, w.aux, 10, ls, pol)
    assert (pi == ids).all() and (pd == dist).all() and (pc[:, 0] == cnt[:, 0]).all()


def test_learned_with_infinite_margin_is_the_plain_search(small):
    w, ix = small
    ids, dist, cnt = O.query(ix, w.q, w.filters, w.aux, 10, 40)
    pol = O.Policy(O.POL_LEARNED, theta=M.init_params(NL, 7).astype(np.float32), tau=np.inf, nq=len(w.q),
                   want_features=True, want_decisions=True)
    pi, pd, pc = O.query_policy(ix, w.q, w.filters, w.aux, 10, 40, pol)
    assert (pi == ids).all() and (pd == dist).all()
    assert (pol.decisions[:, 3] == 0).all() and (pol.decisions[:, 0] == 40).all()
    f = pol.features
    assert (f[:, 1] == 1).all() and (f[:, 2:6] == 0).all()          # label filters
    assert ((f[:, 6] >= 0) & (f[:, 6] <= 1) & (f[:, 9] >= 0) & (f[:, 9] <= 1)).all()


def test_stop_after_last_change_keeps_the_answer(small):
    """The search may stop once no hop can change the first k entries: with
    the stop hop at the last hop that inserted among them the answers equal
    the full search's; hops never exceed the stop."""
    w, ix = small
    ls = 64
    nq = len(w.q)
    plain = O.Policy(O.POL_FORCED, h0=4, forced=np.tile([[ls, 0]], (nq, 1)), nq=nq, want_decisions=True)
    ids, dist, cnt = O.query_policy(ix, w.q, w.filters, w.aux, 10, ls, plain)
    last = plain.decisions[:, 2]
    forced = np.stack([np.full(nq, ls), np.maximum(last, 4)], axis=1).astype(np.int32)
    pol = O.Policy(O.POL_FORCED, h0=4, forced=forced, nq=nq, want_decisions=True)
    pi, pd, pc = O.query_policy(ix, w.q, w.filters, w.aux, 10, ls, pol)
    assert (pi == ids).all() and (pd == dist).all()
    assert (pc[:, 0] <= np.maximum(last, 4)).all()
    assert (pc[:, 0] <= cnt[:, 0]).all()


def test_forced_beam_switch_invariants(small):
    w, ix = small
    nq = len(w.q)
    rng = np.random.default_rng(9)
    beams = rng.choice([10, 16, 24, 32, 48, 64, 80, 200], nq)
    forced = np.stack([beams, np.zeros(nq)], axis=1).astype(np.int32)
    pol = O.Policy(O.POL_FORCED, h0=6, forced=forced, nq=nq, want_decisions=True)
    ids, dist, cnt = O.query_policy(ix, w.q, w.filters, w.aux, 10, 64, pol)
    assert (pol.decisions[:, 0] == np.minimum(beams, 64)).all()        # the beam only shrinks
    lab = (w.filters["payload"] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    for i in range(nq):
        m = ids[i] >= 0
        assert (w.attr_i32[ids[i][m]] == lab[i]).all()
        assert (np.diff(dist[i][m]) >= 0).all()


@pytest.mark.parametrize("c,stop_out,scale", [(0, 0.9, 64.0), (4, -3.0, 64.0), (8, 0.2, 64.0), (3, 5.0, 0.0),
                                              (6, 2000.0, 64.0)])
def test_constant_network_is_a_forced_policy(small, c, stop_out, scale):
    """With W3 = 0 the outputs are b3 exactly (each fma adds an exact zero):
    the policy then equals a FORCED one with beam min(ladder[c], l_s) and stop
    rint(b3[nl] * scale), at least h0, at most 65535, none if scale <= 0."""
    w, ix = small
    nq = len(w.q)
    ladder = (16, 24, 32, 48, 64, 96, 128, 192, 256)
    theta = M.init_params(NL, seed=11).astype(np.float32)
    nw3 = (NL + 1) * 64
    off3 = 64 * 12 + 64 + 64 * 64 + 64
    theta[off3:off3 + nw3] = 0.0
    b3 = np.zeros(NL + 1, np.float32)
    b3[c] = 1.0
    b3[NL] = stop_out
    theta[off3 + nw3:] = b3
    h0 = 6
    pol = O.Policy(O.POL_LEARNED, h0=h0, theta=theta, ladder=ladder, tau=0.5, stop_scale=scale, nq=nq,
                   want_decisions=True)
    a = O.query_policy(ix, w.q, w.filters, w.aux, 10, 128, pol)
    stop = 0 if scale <= 0 else int(min(max(np.rint(np.float32(stop_out) * np.float32(scale)), h0), 65535))
    forced = np.tile(np.array([[ladder[c], stop]], np.int32), (nq, 1))
    fp = O.Policy(O.POL_FORCED, h0=h0, forced=forced, nq=nq, want_decisions=True)
    b = O.query_policy(ix, w.q, w.filters, w.aux, 10, 128, fp)
    assert all((x == y).all() for x, y in zip(a, b))
    assert (pol.decisions == fp.decisions).all()
    assert (pol.decisions[:, 1] == stop).all() and (pol.decisions[:, 0] == min(ladder[c], 128)).all()
    # margin 1.0 below tau: the fixed beam, no stop
    pol2 = O.Policy(O.POL_LEARNED, h0=h0, theta=theta, ladder=ladder, tau=1.5, stop_scale=scale, nq=nq,
                    want_decisions=True)
    O.query_policy(ix, w.q, w.filters, w.aux, 10, 128, pol2)
    assert (pol2.decisions[:, 0] == 128).all() and (pol2.decisions[:, 1] == 0).all() and (pol2.decisions[:, 3] == 0).all()
