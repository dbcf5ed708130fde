"""Training data for, and training of, the learned beam / stop policy.

The policy (see ``jag_policy`` in include/jag.h) runs h0 hops of GreedySearch
(Algorithm 1) at the call's beam, then lets a small network choose the beam
for the rest of the search from a ladder, and a hop count after which the
search stops.  The paper's search has one fixed beam l_s; the policy is an
extension that spends hops where a query needs them.

Traces.  Each training query is searched once per ladder beam with a FORCED
policy: the first h0 hops are the same in every run, so the features at the
decision hop are too.  Each run's answers are scored against the exact
answers (recall@k), and the run reports the last hop that changed the first
k entries of L.  A query's label is the smallest beam whose recall reaches
the best recall over the ladder; its stop target is that run's last change,
times a margin, plus a few hops.

Everything here runs through the CUDA library: the searches, the exact
answers (the exact scan) and the training (jag_mlp_train).  Only the labels
are computed on the host, from the searches' outputs.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import datagen, jag

DEFAULT_H0 = 8
STOP_SCALE = 64.0


def recall_rows(ids, gt_ids, k):
    """Recall@k of each row: |ids & first min(k, #passing) exact ids| divided
    by that number; NaN for rows with no passing point."""
    ids = np.asarray(ids)[:, :k]
    gt = np.asarray(gt_ids)[:, :k]
    m = (gt >= 0).sum(1)
    hit = ((ids[:, :, None] == gt[:, None, :]) & (gt[:, None, :] >= 0) & (ids[:, :, None] >= 0)).any(2).sum(1)
    out = np.full(len(ids), np.nan)
    ok = m > 0
    out[ok] = hit[ok] / m[ok]
    return out


def exact_answers(index, qt, filters, aux, k):
    """Exact top-k by the GPU brute-force scan."""
    import torch
    ids, dist, _ = index.search(qt, filters, aux, k, k, flags=jag.JAG_SEARCH_SCAN_ALL)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dist.cpu().numpy()


@dataclass
class Traces:
    X: np.ndarray          # [nq][12] features at the decision hop
    recall: np.ndarray     # [nq][nl] recall@k per ladder beam
    cost: np.ndarray       # [nq][nl] distance computations per ladder beam
    hops: np.ndarray       # [nq][nl] hops per ladder beam
    last: np.ndarray       # [nq][nl] last hop that changed the first k entries
    ladder: tuple

    def labels(self, stop_margin=1.5, stop_extra=8, slack=0.0, target=None):
        """(y, t): the beam class and the stop target (margin * last change +
        extra hops) / STOP_SCALE of every query.  The class is the smallest
        beam whose recall reaches `target` (e.g. 0.95), or, for a query that
        no beam brings there and when target is None, the smallest beam
        reaching the best recall over the ladder (minus slack)."""
        rec = np.where(np.isnan(self.recall), -1.0, self.recall)
        best = rec.max(axis=1)
        ok = rec >= (best - slack - 1e-9)[:, None]
        if target is not None:
            hit = rec >= target - 1e-9
            ok = np.where(hit.any(axis=1)[:, None], hit, ok)
        y = np.argmax(ok, axis=1).astype(np.int32)
        last = self.last[np.arange(len(y)), y]
        t = ((stop_margin * last + stop_extra) / STOP_SCALE).astype(np.float32)
        return y, t


def collect_traces(index, qt, filters, aux, k, beam, gt_ids, ladder=jag.LADDER, h0=DEFAULT_H0):
    """Run every ladder beam as a FORCED policy (graph route only, s0 = 0)."""
    import torch
    nq = qt.shape[0]
    dev = qt.device
    nl = len(ladder)
    X = None
    rec = np.zeros((nq, nl))
    cost = np.zeros((nq, nl), np.int64)
    hops = np.zeros((nq, nl), np.int64)
    last = np.zeros((nq, nl), np.int64)
    for c, b in enumerate(ladder):
        forced = torch.tensor([[b, 0]], dtype=torch.int32, device=dev).repeat(nq, 1)
        feats = torch.zeros((nq, jag.MLP_FEATURES), dtype=torch.float32, device=dev)
        dec = torch.zeros((nq, 4), dtype=torch.int32, device=dev)
        pol = jag.Policy(jag.JAG_POLICY_FORCED, h0=h0, forced=forced, features=feats, decisions=dec, ladder=ladder)
        ids, _, cnt = index.search(qt, filters, aux, k, beam, counters=True, s0=0, policy=pol)
        torch.cuda.synchronize()
        rec[:, c] = recall_rows(ids.cpu().numpy(), gt_ids, k)
        cn = cnt.cpu().numpy()
        cost[:, c], hops[:, c] = cn[:, 2], cn[:, 0]
        last[:, c] = dec[:, 2].cpu().numpy()
        if X is None:
            X = feats.cpu().numpy()
    return Traces(X, rec, cost, hops, last, tuple(ladder))


def train(traces: Traces, epochs=60, batch=512, lr=2e-3, lam=0.5, seed=0, device="cuda", **label_kw):
    """Train the network on the traces (rows with no passing point are left
    out) with jag_mlp_train; returns (params tensor, loss trace)."""
    import torch
    y, t = traces.labels(**label_kw)
    keep = ~np.isnan(traces.recall).any(1)
    rng = np.random.Generator(np.random.PCG64(seed))
    order = rng.permutation(np.nonzero(keep)[0])
    X = torch.from_numpy(np.ascontiguousarray(traces.X[order])).to(device)
    yd = torch.from_numpy(y[order]).to(device)
    td = torch.from_numpy(t[order]).to(device)
    nl = len(traces.ladder)
    params = torch.from_numpy(datagen.mlp_init_params(nl, seed)).to(device)
    tr = jag.Trainer(nl, params)
    trace = tr.run(X, yd, td, epochs=epochs, batch=batch, lr=lr, lam=lam)
    return params, trace


def concat_traces(parts):
    """One Traces of several (for instance those of the two graphs of a
    mixed workload, searched separately)."""
    return Traces(np.concatenate([p.X for p in parts]), np.concatenate([p.recall for p in parts]),
                  np.concatenate([p.cost for p in parts]), np.concatenate([p.hops for p in parts]),
                  np.concatenate([p.last for p in parts]), parts[0].ladder)
