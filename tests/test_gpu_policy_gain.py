"""What the trained policy network gains over the search without it.

The network is trained on the GPU (jag_mlp_train) on traces the plain search
generates: for each training query, the hop after which its first k answers
no longer changed.  At search time it sets a per-query stop hop after h0
hops.  The method without it spends the same hop budget uniformly: every
query stops at the same hop, the learned policy's mean.  At that equal
budget the learned stops must give a higher recall@10; and with no stop at
all (the plain search at the same beam) recall is an upper bound that the
learned stops approach within a few points while doing fewer hops.
"""
import numpy as np
import pytest

from paper_2602_10258_gb300 import datagen as D

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
jag = pytest.importorskip("paper_2602_10258_gb300.jag")
PL = pytest.importorskip("paper_2602_10258_gb300.policy")

K, BASE, H0 = 10, 256, 32


def _run(ix, q, ft, at, pol, n):
    cnt = None
    ids, _, cnt = ix.search(q, ft, at, K, BASE, counters=True, s0=0, policy=pol)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), cnt.cpu().numpy()


def test_learned_stop_beats_a_uniform_stop_at_equal_hops():
    n = 300_000
    w = D.make_label_zipf(n=n, d=64, nq=3000, seed=0, n_labels=200, n_centres=50)
    wt = D.make_label_zipf(n=n, d=64, nq=12000, seed=0, n_labels=200, n_centres=50, query_seed=101)
    ix = jag.Index.from_workload(w, R=32, l_b=64, thresholds=(100, 0))
    dev = torch.device("cuda")
    q, ft, at = (torch.from_numpy(w.q).to(dev), jag.filters_to_device(w.filters, dev),
                 jag.aux_to_device(w.aux, dev))
    qt, ftt, att = (torch.from_numpy(wt.q).to(dev), jag.filters_to_device(wt.filters, dev),
                    jag.aux_to_device(wt.aux, dev))
    gt, _ = PL.exact_answers(ix, q, ft, at, K)
    nl = len(jag.LADDER)
    # traces of the plain search at the base beam
    forced = torch.tensor([[BASE, 0]], dtype=torch.int32, device=dev).repeat(len(wt.q), 1)
    feats = torch.zeros((len(wt.q), 12), dtype=torch.float32, device=dev)
    dec = torch.zeros((len(wt.q), 4), dtype=torch.int32, device=dev)
    ix.search(qt, ftt, att, K, BASE, s0=0,
              policy=jag.Policy(jag.JAG_POLICY_FORCED, h0=H0, forced=forced, features=feats, decisions=dec))
    torch.cuda.synchronize()
    y = torch.full((len(wt.q),), nl - 1, dtype=torch.int32, device=dev)
    t = ((dec[:, 2].float() + 8.0) / 64.0).contiguous()
    params = torch.from_numpy(D.mlp_init_params(nl, 0)).to(dev)
    trace = jag.Trainer(nl, params).run(feats, y, t, epochs=60, batch=512, lr=2e-3, lam=1.0)
    assert trace[-1] < 0.5 * trace[0]
    plain_ids, plain_cnt = _run(ix, q, ft, at, None, len(w.q))
    r_plain = np.nanmean(PL.recall_rows(plain_ids, gt, K))
    learned = jag.Policy.learned(params, h0=H0, tau=0.0, stop_scale=96.0)
    l_ids, l_cnt = _run(ix, q, ft, at, learned, len(w.q))
    r_learned = np.nanmean(PL.recall_rows(l_ids, gt, K))
    hops_l = l_cnt[:, 0].mean()
    S = int(np.ceil(hops_l))
    uni = jag.Policy(jag.JAG_POLICY_FORCED, h0=H0,
                     forced=torch.tensor([[BASE, S]], dtype=torch.int32, device=dev).repeat(len(w.q), 1))
    u_ids, u_cnt = _run(ix, q, ft, at, uni, len(w.q))
    r_uniform = np.nanmean(PL.recall_rows(u_ids, gt, K))
    print("plain recall %.4f hops %.1f | learned recall %.4f hops %.1f | uniform stop %d recall %.4f hops %.1f"
          % (r_plain, plain_cnt[:, 0].mean(), r_learned, hops_l, S, r_uniform, u_cnt[:, 0].mean()))
    ix.close()
    assert u_cnt[:, 0].mean() >= hops_l - 1e-9
    assert r_learned > r_uniform
    assert hops_l < 0.9 * plain_cnt[:, 0].mean()
    assert r_learned > r_plain - 0.05


def test_learned_beam_saves_hops_on_mixed_filters():
    """The beam head on the mixed workload (float ranges on one graph,
    boolean filters on a graph built on the mask): trained on traces of
    20,000 training queries labelled with the smallest ladder beam that
    reaches recall 0.95 (raised one ladder step as a margin), the network's
    beams make the graph searches shorter than the plain search at the same
    base beam, and recall stays within 0.02 of the plain search's."""
    n, base = 200_000, 192
    ladder = (32, 48, 64, 96, 128, 160, 192, 224, 256)
    nl = len(ladder)
    w = D.make_mixed(n=n, d=64, nq=3000, seed=5, n_centres=40)
    wt = D.make_mixed(n=n, d=64, nq=20000, seed=5, n_centres=40, query_seed=105)
    dev = torch.device("cuda")
    graphs = {jag.JAG_F_RANGE_F32: (100, 10, 0), jag.JAG_F_BOOL: (100, 1, 0)}
    hops_plain, hops_learned, rec_plain, rec_learned = [], [], [], []
    traces, idx = [], {}
    for kind, thr in graphs.items():
        ix = jag.Index(w.x, attr_f32=w.attr_f32, attr_mask=w.attr_mask, dist_a=kind, R=64, l_b=64, thresholds=thr)
        idx[kind] = ix
        rows_t = np.nonzero(wt.filters["kind"] == kind)[0]
        qt = torch.from_numpy(np.ascontiguousarray(wt.q[rows_t])).to(dev)
        ft = jag.filters_to_device(wt.filters[rows_t], dev)
        at = jag.aux_to_device(wt.aux, dev)
        gt_t, _ = PL.exact_answers(ix, qt, ft, at, K)
        traces.append(PL.collect_traces(ix, qt, ft, at, K, base, gt_t, ladder=ladder, h0=16))
    tr = PL.concat_traces(traces)
    y, t = tr.labels(target=0.95, stop_margin=1.25, stop_extra=8)
    y = np.minimum(y + 1, nl - 1).astype(np.int32)
    keep = ~np.isnan(tr.recall).any(1)
    order = np.random.default_rng(0).permutation(np.nonzero(keep)[0])
    params = torch.from_numpy(D.mlp_init_params(nl, 1)).to(dev)
    jag.Trainer(nl, params).run(torch.from_numpy(np.ascontiguousarray(tr.X[order])).to(dev),
                                torch.from_numpy(y[order]).to(dev), torch.from_numpy(t[order]).to(dev),
                                epochs=40, batch=512, lr=2e-3, lam=0.25)
    pol = jag.Policy.learned(params, ladder=ladder, h0=16, tau=0.0, stop_scale=0.0)
    for kind, ix in idx.items():
        rows = np.nonzero(w.filters["kind"] == kind)[0]
        q = torch.from_numpy(np.ascontiguousarray(w.q[rows])).to(dev)
        f = jag.filters_to_device(w.filters[rows], dev)
        a = jag.aux_to_device(w.aux, dev)
        gt, _ = PL.exact_answers(ix, q, f, a, K)
        for p, hops, rec in ((None, hops_plain, rec_plain), (pol, hops_learned, rec_learned)):
            ids, _, cnt = ix.search(q, f, a, K, base, counters=True, s0=0, policy=p)
            torch.cuda.synchronize()
            hops.append(cnt.cpu().numpy()[:, 0])
            rec.append(PL.recall_rows(ids.cpu().numpy(), gt, K))
        ix.close()
    hp, hl = np.concatenate(hops_plain).mean(), np.concatenate(hops_learned).mean()
    rp, rl = np.nanmean(np.concatenate(rec_plain)), np.nanmean(np.concatenate(rec_learned))
    print("plain: %.1f hops, recall %.4f | learned beams: %.1f hops, recall %.4f" % (hp, rp, hl, rl))
    assert hl < 0.9 * hp
    assert rl > rp - 0.02
