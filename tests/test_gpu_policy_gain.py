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
