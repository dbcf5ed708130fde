"""Benchmark: QPS at recall@10 >= 0.95 per selectivity band, JAG filtered
search on one GB300 (N GPUs: one replica and one query batch per rank).

Headline workload (synthetic stand-in for the paper's label-filter datasets):
N=1,000,000 base vectors, d=128, fp32, from a 100-component Gaussian mixture
(centres N(0,4I), unit covariance); one label per point, Zipf(1.1) over 1,000
labels; 10,000 queries from the same mixture with labels from the same law;
k=10, graph degree R=32, build beam 64, thresholds {100%, 0%}, alpha 1.2;
labels with fewer than 16,384 points go to the exact scan (on the tensor
cores).

A step = one jag_search call over the whole 10,000-query batch: filter
preparation and routing, graph search (Algorithm 2) for graph-routed
queries, exact scan for the most selective ones.  The beam is the smallest of
16..256 for which recall@10 (against the exact scan of every query, itself
checked against the oracle's brute force on a sample) is >= 0.95 in every
selectivity band.  Inputs (640 MB of vectors + graph) exceed the L2 cache,
and L2 is also flushed between timed steps.

The same JSON line also carries the other forms: BF16 / FP8 rows and the
learned stop policy on the label workload; the learned beam / stop network
on the mixed range / boolean workload (two graphs, 100,000 training
queries); the precision form on subset filters (d = 100, fp32 / BF16 / FP8
rows); the 10M-point BF16 serving form, indexed at R = 32 and R = 64, with
the serve loop's p50 / p99; the
serve loop on the label index; and the oracle on the host cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QPS at recall@10=0.95 per selectivity band; plain FP32 vs BF16+learned; p99 ms"
BEAMS = [16, 24, 32, 48, 64, 96, 128, 160, 176, 192, 224, 256]
BANDS = [(0.0, 1e-4, "<1e-4"), (1e-4, 1e-3, "[1e-4,1e-3)"), (1e-3, 1e-2, "[1e-3,1e-2)"),
         (1e-2, 1e-1, "[1e-2,1e-1)"), (1e-1, 1.01, "[1e-1,1]")]
K = 10
R = 32
LB = 64
THRESHOLDS = (100, 0)
ALPHA = 1.2
S0 = 16384         # a label slice is scanned when it holds fewer rows than this and at most SCAN_CAP
SCAN_CAP = 16384
SERVE_S0 = 8192    # the serve loop scans a passing set with one warp (fp32 fma), so it takes smaller ones


def workload_desc(n, d, nq):
    return "label filter, Zipf(1.1) over 1000 labels, N=%d d=%d fp32 GMM-100, %d queries, k=10, R=32" % (n, d, nq)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def rank_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def recall_at_k(ids, gt_ids, gt_d=None, k=K):
    """Tie-tolerant recall@k: returned ids whose true distance is within the
    k-th true distance count as hits; divided by min(k, #passing)."""
    out = np.zeros(len(ids))
    for i in range(len(ids)):
        g = gt_ids[i][gt_ids[i] >= 0]
        m = min(k, len(g))
        if m == 0:
            out[i] = np.nan
            continue
        out[i] = len(set(ids[i][ids[i] >= 0].tolist()) & set(g[:m].tolist())) / m
    return out


def aggregate_timing(total_ms, steps, nq_per_rank, world, device):
    """Whole-job timing of a replicated run: the slowest rank's time (max over
    ranks) and the queries of all ranks divided by it."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / steps
    return ms_per_step, world * nq_per_rank / (ms_per_step / 1000.0)


def band_of(sel):
    b = np.full(len(sel), -1)
    for j, (lo, hi, _) in enumerate(BANDS):
        b[(sel >= lo) & (sel < hi)] = j
    return b


class Clocks:
    """nvidia-smi sampler for the timed region."""

    def __init__(self, gpu):
        self.gpu = gpu
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p is not None:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                out, _ = self.p.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        j = json.load(open(p))
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def profile_traffic(src_hash):
    """Per-launch DRAM bytes of the query kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "query_kernel_label_1m.md")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    h = re.search(r"source_hash:\s*([0-9a-f]+)", txt)
    t = re.search(r"traffic_bytes_per_full_launch:\s*([0-9.eE+]+)", txt)
    if not h or not t or h.group(1) != src_hash:
        return None
    return float(t.group(1))


# Sources the query path's kernels (graph search, scan, preparation) are
# compiled from; a profile summary is valid while their code is unchanged
# (the hash skips comments).
QUERY_SOURCES = ["paper_2602_10258_gb300/csrc/" + f for f in (
    "jag_internal.cuh", "launch.h", "launch_util.cuh", "plan.cuh", "query_graph.cuh", "search.cu",
    "search_core.cuh", "search_f32.cu")] + ["include/jag.h"]


def strip_comments(src):
    """C / C++ source without its comments (string literals kept)."""
    return re.sub(r'//[^\n]*|/\*.*?\*/|"(?:\\.|[^"\\])*"',
                  lambda m: m.group(0) if m.group(0).startswith('"') else " ", src, flags=re.S)


def kernel_source_hash():
    """sha256 (16 hex digits) of the query path's sources with comments
    removed and runs of white space made one space."""
    import hashlib
    hs = hashlib.sha256()
    for f in QUERY_SOURCES:
        code = strip_comments(open(os.path.join(ROOT, f), encoding="utf-8").read())
        hs.update(re.sub(r"\s+", " ", code).strip().encode())
    return hs.hexdigest()[:16]


def make_workload(args):
    from paper_2602_10258_gb300 import datagen as D
    return D.make_label_zipf(n=args.n, d=128, nq=args.nq, seed=args.seed)


def selectivity(w):
    counts = np.bincount(w.attr_i32, minlength=int(w.attr_i32.max()) + 1)
    lab = w.filters["payload"].astype(np.int64) & 0xFFFFFFFF
    return counts[np.minimum(lab, len(counts) - 1)] / w.n


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2602_10258_gb300 import jag

    rank, world, local = rank_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    w = make_workload(args)
    sel = selectivity(w)
    band = band_of(sel)
    t0 = time.time()
    idx = jag.Index.from_workload(w, R=R, l_b=LB, alpha=ALPHA, thresholds=THRESHOLDS, device=local)
    build_s = time.time() - t0
    info = idx.info()
    log("build: %.2f s (GPU %.2f s), entry %d" % (build_s, info["build_seconds"], info["entry"]))
    q = torch.from_numpy(w.q).to(dev)
    ft = jag.filters_to_device(w.filters, dev)
    at = jag.aux_to_device(w.aux, dev)
    nq = w.q.shape[0]
    stream = torch.cuda.current_stream(dev)

    # ground truth by the exact scan
    gt_ids = torch.empty((nq, K), dtype=torch.int32, device=dev)
    gt_d = torch.empty((nq, K), dtype=torch.float32, device=dev)
    jag.jag_search(idx.h, q, ft, at, K, K, gt_ids, gt_d, None, stream, flags=jag.JAG_SEARCH_SCAN_ALL)
    torch.cuda.synchronize()
    gt_ids, gt_d = gt_ids.cpu().numpy(), gt_d.cpu().numpy()

    ids = torch.empty((nq, K), dtype=torch.int32, device=dev)
    dd = torch.empty((nq, K), dtype=torch.float32, device=dev)
    cnt = torch.empty((nq, 4), dtype=torch.int32, device=dev)
    sweep = {}
    chosen = None
    band_min_beam = {}
    for beam in BEAMS:
        jag.jag_search(idx.h, q, ft, at, K, beam, ids, dd, None, stream, s0=S0, scan_cap=SCAN_CAP)
        torch.cuda.synchronize()
        rec = recall_at_k(ids.cpu().numpy(), gt_ids, gt_d)
        per = {}
        for j, (_, _, name) in enumerate(BANDS):
            m = (band == j) & ~np.isnan(rec)
            if m.any():
                per[name] = float(np.mean(rec[m]))
                if per[name] >= 0.95 and name not in band_min_beam:
                    band_min_beam[name] = beam
        sweep[beam] = per
        log("beam %d: %s" % (beam, {k: round(v, 4) for k, v in per.items()}))
        if chosen is None and all(v >= 0.95 for v in per.values()):
            chosen = beam
            if not args.full_sweep:
                break
    if chosen is None:
        chosen = BEAMS[-1]

    # counters pass: algorithmic bytes of one launch (untimed)
    jag.jag_search(idx.h, q, ft, at, K, chosen, ids, dd, cnt, stream, s0=S0, scan_cap=SCAN_CAP)
    torch.cuda.synchronize()
    c = cnt.cpu().numpy().astype(np.int64)
    graph_q = c[:, 3] == 0
    scan_q = c[:, 3] == 1
    row_bytes = 128 * 4
    # bytes the graph kernel executes, from its own counters (its visited set
    # forgets, so these include recomputation)
    exec_bytes_graph = int((c[graph_q, 0] * R * 4 + c[graph_q, 1] * 4 + c[graph_q, 2] * row_bytes).sum())
    bytes_scan = int((c[scan_q, 2] * (row_bytes + 4)).sum())

    # timed steps
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for s_ev, e_ev, kb, ke in ev:   # torch creates the CUDA event on first record
        kb.record(stream)
        ke.record(stream)
    for _ in range(args.warmup):
        flush.fill_(1.0)
        jag.jag_search(idx.h, q, ft, at, K, chosen, ids, dd, None, stream, s0=S0, scan_cap=SCAN_CAP)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))
            s_ev, e_ev, kb, ke = ev[i]
            s_ev.record(stream)
            jag.jag_search(idx.h, q, ft, at, K, chosen, ids, dd, None, stream, s0=S0, scan_cap=SCAN_CAP, ev_begin=kb, ev_end=ke)
            e_ev.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = np.array([s.elapsed_time(e) for s, e, _, _ in ev])
    kern_ms = np.array([a.elapsed_time(b) for _, _, a, b in ev])
    ms_per_step, value = aggregate_timing(float(step_ms.sum()), args.steps, nq, world, dev)

    # per-band QPS at each band's own smallest beam (informational)
    bands_out = {}
    for j, (_, _, name) in enumerate(BANDS):
        sel_q = np.nonzero(band == j)[0]
        if len(sel_q) == 0:
            continue
        beam_b = band_min_beam.get(name, chosen)
        qb = q[torch.from_numpy(sel_q).to(dev)]
        fb = jag.filters_to_device(w.filters[sel_q], dev)
        ib = torch.empty((len(sel_q), K), dtype=torch.int32, device=dev)
        db = torch.empty((len(sel_q), K), dtype=torch.float32, device=dev)
        ts = []
        for r in range(4):
            flush.fill_(2.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            jag.jag_search(idx.h, qb, fb, at, K, beam_b, ib, db, None, stream, s0=S0, scan_cap=SCAN_CAP)
            b.record(stream)
            torch.cuda.synchronize()
            if r:
                ts.append(a.elapsed_time(b))
        rec = recall_at_k(ib.cpu().numpy(), gt_ids[sel_q], gt_d[sel_q])
        bands_out[name] = {"queries": int(len(sel_q)), "beam": int(beam_b),
                           "recall": float(np.nanmean(rec)) if np.isfinite(rec).any() else None,
                           "qps": float(len(sel_q) / (np.median(ts) / 1000.0)),
                           "routed_to_scan": int((c[sel_q, 3] == 1).sum())}

    # end to end through the host-buffer entry point
    pin_q = torch.from_numpy(w.q).pin_memory()
    pin_f = torch.from_numpy(np.ascontiguousarray(w.filters).view(np.uint8).copy()).pin_memory()
    pin_ids = torch.empty((nq, K), dtype=torch.int32).pin_memory()
    pin_d = torch.empty((nq, K), dtype=torch.float32).pin_memory()
    for _ in range(2):
        jag.jag_search_host(idx.h, pin_q, pin_f, None, K, chosen, s0=S0, scan_cap=SCAN_CAP, out_ids=pin_ids, out_dist=pin_d)
    e2e_t = []
    for _ in range(max(3, min(args.steps, 10))):
        flush.fill_(3.0)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        jag.jag_search_host(idx.h, pin_q, pin_f, None, K, chosen, s0=S0, scan_cap=SCAN_CAP, out_ids=pin_ids, out_dist=pin_d)
        e2e_t.append(time.perf_counter() - t1)
    e2e_rec = recall_at_k(pin_ids.numpy(), gt_ids, gt_d)
    assert np.array_equal(pin_ids.numpy(), ids.cpu().numpy())

    # the same graph with BF16 / FP8 rows (searched in that format, fp32
    # re-rank of the top min(4k, beam)), swept and timed the same way
    graph_host, entry = idx.graph(), info["entry"]
    forms = {}
    for fname, fcode in (("bf16", jag.JAG_VEC_BF16), ("fp8", jag.JAG_VEC_FP8)):
        fidx = jag.Index.from_workload(w, R=R, graph=graph_host, entry=entry, storage=fcode, device=local)
        forms[fname] = measure_form(jag, fidx, q, ft, at, nq, band, gt_ids, gt_d, min(args.steps, 100), flush,
                                    stream)
        forms[fname]["distance_error_vs_fp64"] = stored_distance_error(fidx, w, gt_ids, fcode)
        fidx.close()
        log("%s: beam %s, %.0f QPS" % (fname, forms[fname]["beam"], forms[fname]["qps"]))
    forms["fp32"] = {"beam": chosen, "qps": round(value / world, 1), "recall": sweep[chosen],
                     "graph_kernel_ms": round(float(kern_ms.mean()), 3)}
    if not args.no_learned:
        forms["bf16_learned"] = measure_learned(jag, w, graph_host, entry, local, q, ft, at, nq, band, gt_ids, gt_d,
                                                flush, stream, steps=min(args.steps, 50))
        log("bf16+learned: %s" % {k: v for k, v in forms["bf16_learned"].items() if k in ("beam", "stop_scale", "qps")})
    serving = None
    if not args.no_serve:
        serving = measure_serving(jag, idx, w, chosen, band, gt_ids, gt_d, value / world)
        log("serving: %s" % {k: (v["p50_ms"], v["p99_ms"], v["achieved_qps"]) for k, v in serving.items() if isinstance(v, dict)})

    mixed = None
    if not args.no_mixed:
        mixed = measure_mixed(args, local, flush, stream)
    subset = None
    if not args.no_subset:
        subset = measure_subset(args, local, flush, stream)
    large = None
    if not args.no_large:
        large = measure_large(args, local)

    cpu, ocnt = None, None
    if rank == 0 and not args.no_cpu:
        cpu, ocnt = cpu_baseline(w, idx, chosen, gt_ids, gt_d, budget_s=args.cpu_seconds)
    # algorithmic bytes of the graph kernel per launch: H*R*4 + U*4 + U'*row
    # per graph-routed query, with H, U (first-seen neighbours) and U' (vector
    # distances) counted by the oracle's search, whose visited set is exact;
    # scaled to the whole batch when the oracle ran on a sample
    if ocnt is not None:
        og = ocnt[:, 3] == 0
        sample_bytes = int((ocnt[og, 0] * R * 4 + ocnt[og, 1] * 4 + ocnt[og, 2] * row_bytes).sum())
        alg_bytes = int(sample_bytes * graph_q.sum() / max(1, og.sum()))
        alg_source = "oracle counts (%d graph-routed queries)" % int(og.sum())
    else:
        alg_bytes = exec_bytes_graph
        alg_source = "kernel counters"
    peak, peak_kind = measured_peaks()
    kavg_s = float(kern_ms.mean()) / 1000.0
    achieved = alg_bytes / kavg_s / 1e9
    traffic = profile_traffic(kernel_source_hash())
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "kernel": "query_kernel (graph route)", "kernel_ms": round(kavg_s * 1000, 3),
                "algorithmic_bytes_per_launch": alg_bytes, "algorithmic_bytes_source": alg_source,
                "executed_bytes_per_launch": exec_bytes_graph, "peak_source": peak_kind,
                "scan_route_bytes_per_step": bytes_scan}

    recall_chosen = sweep[chosen]
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "queries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload_desc(w.n, w.d, nq), "beam": chosen, "k": K, "R": R,
                   "build": "GPU JAG build, l_b=%d, T=%s%%, alpha=%.1f" % (LB, list(THRESHOLDS), ALPHA),
                   "build_seconds": round(build_s, 2), "index_device_bytes": info["device_bytes"],
                   "scan_threshold_s0": S0, "scan_cap": SCAN_CAP, "l2": "inputs larger than L2 and L2 flushed between steps",
                   "recall_at_beam": recall_chosen, "bands": bands_out,
                   "beam_sweep": {str(b): v for b, v in sweep.items()},
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline,
        "e2e": {"value": round(nq / float(np.median(e2e_t)), 1), "unit": "queries/s",
                "h2d_bytes_per_step": int(w.q.nbytes + w.filters.nbytes),
                "d2h_bytes_per_step": int(nq * K * 8),
                "recall": float(np.nanmean(e2e_rec))},
        "cpu_baseline": cpu,
        "forms": forms,
        "learned_form_mixed": mixed,
        "precision_form_subset": subset,
        "serving_form_10m": large,
        "serving": serving,
        "clocks": clk.summary(),
        # per step (the launch list in profiles/): preparation, graph search, and
        # the tensor-core scan's count, two sums, offsets, fill, items, query
        # norms, contraction and selection
        "gpu_launches": int(args.steps * 11),
    }
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    idx.close()


def measure_form(jag, idx, q, ft, at, nq, band, gt_ids, gt_d, steps, flush, stream):
    """Smallest beam of the ladder with recall@10 >= 0.95 in every band, and
    the device time of a whole-batch search at that beam."""
    import torch
    dev = q.device
    ids = torch.empty((nq, K), dtype=torch.int32, device=dev)
    dd = torch.empty((nq, K), dtype=torch.float32, device=dev)
    chosen, per = None, None
    for beam in BEAMS:
        jag.jag_search(idx.h, q, ft, at, K, beam, ids, dd, None, stream, s0=S0, scan_cap=SCAN_CAP)
        torch.cuda.synchronize()
        rec = recall_at_k(ids.cpu().numpy(), gt_ids, gt_d)
        per = {}
        for j, (_, _, name) in enumerate(BANDS):
            m = (band == j) & ~np.isnan(rec)
            if m.any():
                per[name] = float(np.mean(rec[m]))
        if all(v >= 0.95 for v in per.values()):
            chosen = beam
            break
    if chosen is None:
        chosen = BEAMS[-1]
    cnt = torch.empty((nq, 4), dtype=torch.int32, device=dev)
    jag.jag_search(idx.h, q, ft, at, K, chosen, ids, dd, cnt, stream, s0=S0, scan_cap=SCAN_CAP)
    torch.cuda.synchronize()
    c = cnt.cpu().numpy()
    for _ in range(3):
        jag.jag_search(idx.h, q, ft, at, K, chosen, ids, dd, None, stream, s0=S0, scan_cap=SCAN_CAP)
    ts, ks = [], []
    for i in range(steps):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ka, kb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ka.record(stream)
        kb.record(stream)
        a.record(stream)
        jag.jag_search(idx.h, q, ft, at, K, chosen, ids, dd, None, stream, s0=S0, scan_cap=SCAN_CAP, ev_begin=ka, ev_end=kb)
        b.record(stream)
        ts.append((a, b, ka, kb))
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b, _, _ in ts]))
    kms = float(np.mean([ka.elapsed_time(kb) for _, _, ka, kb in ts]))
    info = idx.info()
    row_bytes = (info["d"] * 2 + 15) // 16 * 16 if info["storage"] == 1 else (info["d"] + 15) // 16 * 16 + 4
    gbytes = mixed_graph_bytes(c, row_bytes, 4, R)
    return {"beam": chosen, "qps": round(nq / (ms / 1000.0), 1), "ms_per_step": round(ms, 4),
            "graph_kernel_ms": round(kms, 3), "recall": per, "steps": steps,
            "graph_kernel_gather_bytes": gbytes,
            "graph_kernel_frac_of_hbm": round(gbytes / (kms / 1e3) / 1e9 / measured_peaks()[0], 4),
            "gather_bytes_source": "the kernel's counters (hops, first-seen neighbours, distances)"}


def measure_learned(jag, w, graph_host, entry, local, q, ft, at, nq, band, gt_ids, gt_d, flush, stream,
                    n_train=20000, steps=50):
    """BF16 rows + the learned stop hop.  Traces: n_train training queries
    (another query seed, same base set) searched at each base beam; the
    network learns the hop of each query's last change among its first k
    answers (plus 8 hops), in units of 1/64 hop.  Then the fastest (base beam,
    stop scale) whose recall@10 is >= 0.95 in every band, timed like the
    other forms; the fixed-beam BF16 form is its baseline."""
    import torch
    from paper_2602_10258_gb300 import datagen as D
    from paper_2602_10258_gb300 import policy as PL
    dev = q.device
    fidx = jag.Index.from_workload(w, R=R, graph=graph_host, entry=entry, storage=jag.JAG_VEC_BF16, device=local)
    wt = D.make_label_zipf(n=w.n, d=w.d, nq=n_train, seed=0, query_seed=101)
    qt = torch.from_numpy(wt.q).to(dev)
    ftt = jag.filters_to_device(wt.filters, dev)
    att = jag.aux_to_device(wt.aux, dev)
    nl = len(jag.LADDER)
    ids = torch.empty((nq, K), dtype=torch.int32, device=dev)
    dd = torch.empty((nq, K), dtype=torch.float32, device=dev)
    cnt = torch.empty((nq, 4), dtype=torch.int32, device=dev)
    t0 = time.time()
    cands, best_cnt = [], {}
    for base in (192, 224, 256):
        forced = torch.tensor([[base, 0]], dtype=torch.int32, device=dev).repeat(n_train, 1)
        feats = torch.zeros((n_train, 12), dtype=torch.float32, device=dev)
        dec = torch.zeros((n_train, 4), dtype=torch.int32, device=dev)
        pol = jag.Policy(jag.JAG_POLICY_FORCED, h0=32, forced=forced, features=feats, decisions=dec)
        fidx.search(qt, ftt, att, K, base, s0=0, policy=pol)
        torch.cuda.synchronize()
        X = feats
        y = torch.full((n_train,), nl - 1, dtype=torch.int32, device=dev)    # keep the base beam
        t = ((dec[:, 2].float() + 8.0) / 64.0).contiguous()
        params = torch.from_numpy(D.mlp_init_params(nl, 0)).to(dev)
        tr = jag.Trainer(nl, params)
        trace = tr.run(X, y, t, epochs=60, batch=512, lr=2e-3, lam=1.0)
        for scale in (64.0, 80.0, 96.0, 112.0, 128.0, 160.0, 192.0, 256.0):
            lp = jag.Policy.learned(params, h0=32, tau=0.0, stop_scale=scale)
            jag.jag_search(fidx.h, q, ft, at, K, base, ids, dd, cnt, stream, s0=S0, scan_cap=SCAN_CAP, policy=lp)
            torch.cuda.synchronize()
            rec = recall_at_k(ids.cpu().numpy(), gt_ids, gt_d)
            per = {name: float(np.mean(rec[(band == j) & ~np.isnan(rec)])) for j, (_, _, name) in enumerate(BANDS)
                   if ((band == j) & ~np.isnan(rec)).any()}
            c = cnt.cpu().numpy()
            g = c[:, 3] == 0
            best_cnt[(base, scale)] = c
            cands.append((base, scale, lp, per, float(c[g, 0].mean()), float(trace[-1])))
    ok = [cd for cd in cands if all(v >= 0.95 for v in cd[3].values())]
    train_s = time.time() - t0

    def timed(beam, pol):
        for _ in range(3):
            jag.jag_search(fidx.h, q, ft, at, K, beam, ids, dd, None, stream, s0=S0, scan_cap=SCAN_CAP, policy=pol)
        evs = []
        for i in range(steps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            jag.jag_search(fidx.h, q, ft, at, K, beam, ids, dd, None, stream, s0=S0, scan_cap=SCAN_CAP, policy=pol)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in evs]))

    best = None
    for base, scale, lp, per, hops, loss in ok:
        ms = timed(base, lp)
        if best is None or ms < best[0]:
            best = (ms, base, scale, per, hops, loss)
    fidx.close()
    if best is None:
        return {"qps": None, "note": "no (base, scale) reached recall 0.95 in every band",
                "train_seconds": round(train_s, 1)}
    ms, base, scale, per, hops, loss = best
    c = best_cnt[(base, scale)]
    gbytes = mixed_graph_bytes(c, (w.d * 2 + 15) // 16 * 16, 4, R)
    return {"beam": base, "stop_scale": scale, "h0": 32, "qps": round(nq / (ms / 1000.0), 1),
            "ms_per_step": round(ms, 4), "recall": per, "mean_hops_graph_route": round(hops, 1),
            "gather_bytes_per_step": gbytes,
            "gather_frac_of_hbm_over_step": round(gbytes / (ms / 1e3) / 1e9 / measured_peaks()[0], 4),
            "train": {"queries": n_train, "epochs": 60, "final_loss": round(loss, 4), "seconds": round(train_s, 1)},
            "steps": steps}


# ---------------------------------------------------------------------------
# the learned form's workload: float ranges and boolean filters
# ---------------------------------------------------------------------------

MIXED_R = 64                    # out-degree of both graphs of the mixed workload
MIXED_T_RANGE = (100, 10, 0)    # thresholds of the float-range graph
MIXED_T_BOOL = (100, 1, 0)      # thresholds of the mask graph (Hamming dist_A)
MIXED_LADDER = (32, 48, 64, 96, 128, 160, 192, 224, 256)
MIXED_H0 = 16


def mixed_selectivity(w, dev):
    """Exact selectivity of every filter of a mixed workload: float ranges by
    binary search in the sorted column, boolean filters by counting the
    points' 3-bit patterns on the GPU (torch; bookkeeping, not the path)."""
    import torch
    from paper_2602_10258_gb300 import datagen as D
    kind = w.filters["kind"]
    sel = np.zeros(len(w.q))
    rq = np.nonzero(kind == 3)[0]
    srt = np.sort(w.attr_f32)
    fl = D.filter_fields(w.filters)
    sel[rq] = (np.searchsorted(srt, fl["f_hi"][rq], "right") - np.searchsorted(srt, fl["f_lo"][rq], "left")) / w.n
    mt = torch.from_numpy(w.attr_mask.view(np.int64)).to(dev)
    for i in np.nonzero(kind == 5)[0]:
        vm = int(w.filters["payload"][i])
        bits = [b for b in range(64) if vm >> b & 1]
        pat = torch.zeros_like(mt)
        for j, b in enumerate(bits):
            pat |= ((mt >> b) & 1) << j
        h = torch.bincount(pat, minlength=1 << len(bits)).cpu().numpy()
        tt = w.aux[int(w.filters["aux_off"][i]):]
        sel[i] = sum(h[s_] for s_ in range(1 << len(bits)) if tt[s_ >> 3] >> (s_ & 7) & 1) / w.n
    return sel


class MixedIndex:
    """The two graphs of the mixed workload over one point set: float-range
    filters search a graph built on the float attribute, boolean filters one
    built on the bit mask (Hamming dist_A, Sec. 3.1), each query routed by its
    filter kind.  The two searches of a batch run on two streams."""

    def __init__(self, jag, w, storage, device, graphs=None):
        kw = dict(attr_f32=w.attr_f32, attr_mask=w.attr_mask, R=MIXED_R, l_b=64, alpha=ALPHA, storage=storage,
                  device=device)
        if graphs is None:
            self.ix = [jag.Index(w.x, dist_a=jag.JAG_F_RANGE_F32, thresholds=MIXED_T_RANGE, **kw),
                       jag.Index(w.x, dist_a=jag.JAG_F_BOOL, thresholds=MIXED_T_BOOL, **kw)]
        else:
            self.ix = [jag.Index(w.x, dist_a=da, graph=g, entry=e, **kw)
                       for da, (g, e) in zip((jag.JAG_F_RANGE_F32, jag.JAG_F_BOOL), graphs)]

    def graphs(self):
        return [(ix.graph(), ix.info()["entry"]) for ix in self.ix]

    def build_seconds(self):
        return [round(ix.info()["build_seconds"], 2) for ix in self.ix]

    def close(self):
        for ix in self.ix:
            ix.close()


class MixedBatch:
    """Device inputs and outputs of a mixed batch, split by filter kind."""

    def __init__(self, jag, w, dev):
        import torch
        kind = w.filters["kind"]
        self.rows = [np.nonzero(kind == jag.JAG_F_RANGE_F32)[0], np.nonzero(kind == jag.JAG_F_BOOL)[0]]
        self.q = [torch.from_numpy(np.ascontiguousarray(w.q[r])).to(dev) for r in self.rows]
        self.f = [jag.filters_to_device(w.filters[r], dev) for r in self.rows]
        self.aux = jag.aux_to_device(w.aux, dev)
        self.ids = [torch.empty((len(r), K), dtype=torch.int32, device=dev) for r in self.rows]
        self.dist = [torch.empty((len(r), K), dtype=torch.float32, device=dev) for r in self.rows]
        self.cnt = [torch.empty((len(r), 4), dtype=torch.int32, device=dev) for r in self.rows]
        self.streams = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
        self.n = len(w.q)

    def search(self, jag, mix, beams, policy=None, counters=False, stream=None, scan_all=False):
        """Both kinds' searches, forked from `stream` onto two streams and
        joined back (asynchronous)."""
        import torch
        stream = stream or torch.cuda.current_stream()
        fork = torch.cuda.Event()
        fork.record(stream)
        for g in range(2):
            st = self.streams[g]
            st.wait_event(fork)
            if len(self.rows[g]) == 0:
                continue
            kw = dict(flags=jag.JAG_SEARCH_SCAN_ALL) if scan_all else dict(s0=S0, scan_cap=SCAN_CAP, policy=policy)
            jag.jag_search(mix.ix[g].h, self.q[g], self.f[g], self.aux, K, K if scan_all else beams[g], self.ids[g],
                           self.dist[g], self.cnt[g] if counters else None, st, **kw)
            done = torch.cuda.Event()
            done.record(st)
            stream.wait_event(done)

    def gather(self, what):
        out = np.empty((self.n,) + tuple(what[0].shape[1:]), dtype=what[0].cpu().numpy().dtype)
        for g in range(2):
            out[self.rows[g]] = what[g].cpu().numpy()
        return out


def band_recalls(rec, band):
    return {name: float(np.mean(rec[(band == j) & ~np.isnan(rec)])) for j, (_, _, name) in enumerate(BANDS)
            if ((band == j) & ~np.isnan(rec)).any()}


def mixed_graph_bytes(cnt, row_bytes, attr_bytes, R_=MIXED_R):
    """Gather bytes of the graph searches from the kernels' own counters:
    hops * R * 4 + first-seen neighbours * attribute bytes + distances *
    row bytes, over graph-routed queries."""
    g = cnt[:, 3] == 0
    c = cnt[g].astype(np.int64)
    return int((c[:, 0] * R_ * 4 + c[:, 1] * attr_bytes + c[:, 2] * row_bytes).sum())


def measure_mixed(args, local, flush, stream):
    """The learned form's workload (float ranges and 3-of-32 boolean filters,
    N = 1M, d = 128): plain fixed-beam search (fp32 and BF16 rows; per graph
    the smallest beam with recall@10 >= 0.95 in every band of its queries)
    against BF16 rows with the learned beam / stop network, trained on the
    GPU on traces of 100,000 training queries labelled with the smallest
    ladder beam reaching recall 0.95; the same networks also run on the fp32
    rows."""
    import torch
    from paper_2602_10258_gb300 import datagen as D
    from paper_2602_10258_gb300 import jag
    from paper_2602_10258_gb300 import policy as PL
    dev = torch.device("cuda", local)
    t0 = time.time()
    w = D.make_mixed(n=args.n, d=128, nq=args.nq, seed=args.seed)
    wt = D.make_mixed(n=args.n, d=128, nq=args.mixed_train, seed=args.seed, query_seed=101)
    sel = mixed_selectivity(w, dev)
    band = band_of(sel)
    mix32 = MixedIndex(jag, w, jag.JAG_VEC_F32, local)
    graphs = mix32.graphs()
    mix16 = MixedIndex(jag, w, jag.JAG_VEC_BF16, local, graphs=graphs)
    prep_s = time.time() - t0
    hb = MixedBatch(jag, w, dev)
    hb.search(jag, mix32, (K, K), scan_all=True)
    torch.cuda.synchronize()
    gt_ids = hb.gather(hb.ids)
    out = {"workload": "float range (width log-uniform 1e-4..1) and boolean (AND/OR of 3 of 32 Bernoulli(0.3) bits) "
                       "filters, half each, N=%d d=128 fp32 GMM-100, %d queries, k=10" % (w.n, len(w.q)),
           "graphs": "float-range graph R=%d T=%s%%, mask graph R=%d T=%s%% (Hamming dist_A), GPU build %s s"
                     % (MIXED_R, list(MIXED_T_RANGE), MIXED_R, list(MIXED_T_BOOL), mix32.build_seconds()),
           "queries_by_kind": {"range": int(len(hb.rows[0])), "bool": int(len(hb.rows[1]))},
           "band_queries": {name: int((band == j).sum()) for j, (_, _, name) in enumerate(BANDS)}}

    def timed(mix, beams, pol, steps):
        for _ in range(3):
            hb.search(jag, mix, beams, pol, stream=stream)
        evs = []
        for i in range(steps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            hb.search(jag, mix, beams, pol, stream=stream)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in evs]))

    def evaluate(mix, beams, pol):
        hb.search(jag, mix, beams, pol, counters=True, stream=stream)
        torch.cuda.synchronize()
        ids, cnt = hb.gather(hb.ids), hb.gather(hb.cnt)
        rec = recall_at_k(ids, gt_ids, None)
        return band_recalls(rec, band), cnt

    steps = min(args.steps, 50)
    forms = {}
    for fname, mix, row_bytes in (("fp32", mix32, 512), ("bf16", mix16, 256)):
        beams = []
        for g in range(2):
            chosen = MIXED_LADDER[-1]
            for beam in MIXED_LADDER:
                bb = [MIXED_LADDER[-1], MIXED_LADDER[-1]]
                bb[g] = beam
                per, _ = evaluate(mix, bb, None)
                gb = band_of(sel[hb.rows[g]])
                rec_g = recall_at_k(hb.gather(hb.ids)[hb.rows[g]], gt_ids[hb.rows[g]], None)
                if all(v >= 0.95 for v in band_recalls(rec_g, gb).values()):
                    chosen = beam
                    break
            beams.append(chosen)
        per, cnt = evaluate(mix, beams, None)
        ms = timed(mix, beams, None, steps)
        gbytes = mixed_graph_bytes(cnt[hb.rows[0]], row_bytes, 4) + mixed_graph_bytes(cnt[hb.rows[1]], row_bytes, 8)
        forms["plain_" + fname] = {"beam_range": beams[0], "beam_bool": beams[1], "qps": round(hb.n / (ms / 1e3), 1),
                                   "ms_per_step": round(ms, 4), "recall": per,
                                   "mean_hops_graph_route": round(float(cnt[cnt[:, 3] == 0, 0].mean()), 1),
                                   "gather_bytes_per_step": gbytes,
                                   "gather_frac_of_hbm": round(gbytes / (ms / 1e3) / 1e9 / measured_peaks()[0], 4)}
        log("mixed plain %s: beams %s, %.0f QPS, %s" % (fname, beams, hb.n / (ms / 1e3), per))
    # learned policy: traces of the training queries on the BF16 graphs (the
    # graph-routed ones: scan-routed queries never reach the policy)
    t1 = time.time()
    tb = MixedBatch(jag, wt, dev)
    tb.search(jag, mix16, (K, K), scan_all=True)
    torch.cuda.synchronize()
    gt_train = [tb.ids[g].cpu().numpy() for g in range(2)]
    tb.search(jag, mix16, (MIXED_LADDER[-1], MIXED_LADDER[-1]), counters=True)
    torch.cuda.synchronize()
    base = (forms["plain_bf16"]["beam_range"], forms["plain_bf16"]["beam_bool"])
    tr = []
    for g in range(2):
        gq = np.nonzero(tb.cnt[g].cpu().numpy()[:, 3] == 0)[0]
        if len(gq) == 0:
            continue
        sel_q = torch.from_numpy(gq).to(dev)
        fg = tb.f[g].view(-1, 16)[sel_q].reshape(-1)
        # traced at the call beam the policy will run with (the features depend on it)
        tr.append(PL.collect_traces(mix16.ix[g], tb.q[g][sel_q], fg, tb.aux, K, base[g], gt_train[g][gq],
                                    ladder=MIXED_LADDER, h0=MIXED_H0))
    traces = PL.concat_traces(tr)
    trace_s = time.time() - t1
    nl = len(MIXED_LADDER)
    keep = ~np.isnan(traces.recall).any(1)
    order = np.random.default_rng(0).permutation(np.nonzero(keep)[0])
    X = torch.from_numpy(np.ascontiguousarray(traces.X[order])).to(dev)
    t2 = time.time()
    nets, cands = {}, []
    for shift in (0, 1, 2):
        # labels: the smallest ladder beam reaching recall 0.95, raised by
        # `shift` ladder steps as a margin; stop target from the label beam's
        # last change
        y, tt = traces.labels(target=0.95, stop_margin=1.25, stop_extra=8)
        y = np.minimum(y + shift, nl - 1).astype(np.int32)
        params = torch.from_numpy(D.mlp_init_params(nl, shift)).to(dev)
        loss = jag.Trainer(nl, params).run(X, torch.from_numpy(y[order]).to(dev),
                                           torch.from_numpy(tt[order]).to(dev), epochs=args.mixed_epochs, batch=1024,
                                           lr=2e-3, lam=0.25)
        nets[shift] = (params, float(loss[-1]), np.bincount(y[keep], minlength=nl))
        for tau in (0.0, 0.5, 1.0):
            for scale in (0.0, 96.0):
                pol = jag.Policy.learned(params, ladder=MIXED_LADDER, h0=MIXED_H0, tau=tau, stop_scale=scale)
                per, cnt = evaluate(mix16, base, pol)
                cands.append((shift, tau, scale, pol, per, cnt))
    torch.cuda.synchronize()
    train_s = time.time() - t2
    ok = [c for c in cands if all(v >= 0.95 for v in c[4].values())]
    best = None
    for shift, tau, scale, pol, per, cnt in ok:
        ms = timed(mix16, base, pol, steps)
        if best is None or ms < best[0]:
            best = (ms, shift, tau, scale, per, cnt)
    learned = {"train": {"queries": int(len(wt.q)), "traced_graph_queries": int(keep.sum()),
                         "label_beams": {str(MIXED_LADDER[c]): int(v) for c, v in enumerate(nets[0][2])},
                         "epochs": args.mixed_epochs, "final_loss_by_shift": {str(k_): round(v[1], 4)
                                                                           for k_, v in nets.items()},
                         "trace_seconds": round(trace_s, 1), "train_and_select_seconds": round(train_s, 1)},
               "candidates": [{"shift": c[0], "tau": c[1], "stop_scale": c[2],
                               "mean_hops": round(float(c[5][c[5][:, 3] == 0, 0].mean()), 1),
                               "min_band_recall": round(min(c[4].values()), 4)} for c in cands]}
    if best is None:
        learned["qps"] = None
        learned["note"] = "no (label shift, tau, stop scale) reached recall 0.95 in every band"
    else:
        ms, shift, tau, scale, per, cnt = best
        gbytes = mixed_graph_bytes(cnt[hb.rows[0]], 256, 4) + mixed_graph_bytes(cnt[hb.rows[1]], 256, 8)
        learned.update({"base_beam_range": base[0], "base_beam_bool": base[1], "h0": MIXED_H0, "label_shift": shift,
                        "tau": tau, "stop_scale": scale, "qps": round(hb.n / (ms / 1e3), 1),
                        "ms_per_step": round(ms, 4), "recall": per,
                        "mean_hops_graph_route": round(float(cnt[cnt[:, 3] == 0, 0].mean()), 1),
                        "gather_bytes_per_step": gbytes,
                        "gather_frac_of_hbm": round(gbytes / (ms / 1e3) / 1e9 / measured_peaks()[0], 4)})
    forms["bf16_learned"] = learned
    log("mixed learned: %s" % {k: v for k, v in learned.items() if k in ("label_shift", "tau", "stop_scale", "qps",
                                                                       "recall", "mean_hops_graph_route")})
    # the same networks on the fp32 rows, at the plain fp32 form's beams: the
    # fastest candidate that keeps recall >= 0.95 in every band
    base32 = (forms["plain_fp32"]["beam_range"], forms["plain_fp32"]["beam_bool"])
    best32 = None
    for shift, tau, scale, _, _, _ in cands:
        pol = jag.Policy.learned(nets[shift][0], ladder=MIXED_LADDER, h0=MIXED_H0, tau=tau, stop_scale=scale)
        per, cnt = evaluate(mix32, base32, pol)
        if not all(v >= 0.95 for v in per.values()):
            continue
        ms = timed(mix32, base32, pol, steps)
        if best32 is None or ms < best32[0]:
            best32 = (ms, shift, tau, scale, per, cnt)
    if best32 is None:
        forms["fp32_learned"] = {"qps": None, "note": "no candidate kept recall 0.95 in every band on fp32 rows"}
    else:
        ms, shift, tau, scale, per, cnt = best32
        gbytes = mixed_graph_bytes(cnt[hb.rows[0]], 512, 4) + mixed_graph_bytes(cnt[hb.rows[1]], 512, 8)
        forms["fp32_learned"] = {"base_beam_range": base32[0], "base_beam_bool": base32[1], "h0": MIXED_H0,
                                 "label_shift": shift, "tau": tau, "stop_scale": scale,
                                 "networks": "trained on the BF16 traces", "qps": round(hb.n / (ms / 1e3), 1),
                                 "ms_per_step": round(ms, 4), "recall": per,
                                 "mean_hops_graph_route": round(float(cnt[cnt[:, 3] == 0, 0].mean()), 1),
                                 "gather_bytes_per_step": gbytes,
                                 "gather_frac_of_hbm": round(gbytes / (ms / 1e3) / 1e9 / measured_peaks()[0], 4)}
    log("mixed learned fp32: %s" % {k: v for k, v in forms["fp32_learned"].items()
                                    if k in ("label_shift", "tau", "stop_scale", "qps", "recall")})
    out["forms"] = forms
    out["prep_seconds"] = round(prep_s, 1)
    mix32.close()
    mix16.close()
    return out


# ---------------------------------------------------------------------------
# the precision form's workload: subset filters over 64-bit label masks
# ---------------------------------------------------------------------------

SUBSET_R = 64
SUBSET_WEIGHTS = (0, 1, 5)      # Weight-JAG multipliers of the mask graph (Hamming dist_A)
SUBSET_BEAMS = (64, 96, 128, 160, 192, 256, 320, 384, 512)


def subset_selectivity(w, dev):
    """Exact selectivity of every subset filter (torch on the GPU; bookkeeping)."""
    import torch
    mt = torch.from_numpy(w.attr_mask.view(np.int64)).to(dev)
    req = w.filters["payload"].view(np.int64)
    sel = np.zeros(len(req))
    for i0 in range(0, len(req), 64):
        r = torch.from_numpy(np.ascontiguousarray(req[i0:i0 + 64])).to(dev)
        sel[i0:i0 + 64] = ((mt[None, :] & r[:, None]) == r[:, None]).sum(1).cpu().numpy() / w.n
    return sel


def measure_subset(args, local, flush, stream):
    """The precision form: N = 1M, d = 100 (200-component mixture), a 64-bit
    label mask per point (bit j with probability 0.5/(j+1)), 10,000 subset
    queries requiring 1-3 labels; rows stored as fp32, BF16 and FP8-E4M3 with
    a per-row scale (fp32 re-rank of the leading min(4k, beam) candidates).
    Per format: the smallest beam with recall@10 >= 0.95 in every band, its
    QPS, and the stored distance's error against fp64."""
    import torch
    from paper_2602_10258_gb300 import datagen as D
    from paper_2602_10258_gb300 import jag
    dev = torch.device("cuda", local)
    t0 = time.time()
    w = D.make_subset(n=args.n, d=100, nq=args.nq, seed=args.seed)
    sel = subset_selectivity(w, dev)
    band = band_of(sel)
    ix32 = jag.Index.from_workload(w, R=SUBSET_R, l_b=64, alpha=ALPHA, weights=SUBSET_WEIGHTS, device=local)
    info = ix32.info()
    graph, entry = ix32.graph(), info["entry"]
    prep_s = time.time() - t0
    nq = len(w.q)
    q = torch.from_numpy(w.q).to(dev)
    ft = jag.filters_to_device(w.filters, dev)
    at = jag.aux_to_device(w.aux, dev)
    gt_ids = torch.empty((nq, K), dtype=torch.int32, device=dev)
    gt_d = torch.empty((nq, K), dtype=torch.float32, device=dev)
    jag.jag_search(ix32.h, q, ft, at, K, K, gt_ids, gt_d, None, stream, flags=jag.JAG_SEARCH_SCAN_ALL)
    torch.cuda.synchronize()
    gt_ids, gt_d = gt_ids.cpu().numpy(), gt_d.cpu().numpy()
    out = {"workload": "subset filter, 64-bit masks with P(bit j) = 0.5/(j+1), 1-3 required labels "
                       "(selectivity 1e-4..0.5), N=%d d=100 fp32 GMM-200, %d queries, k=10" % (w.n, nq),
           "graph": "Weight-JAG R=%d, weights %s (Hamming dist_A), l_b=64, GPU build %.2f s"
                    % (SUBSET_R, list(SUBSET_WEIGHTS), info["build_seconds"]),
           "band_queries": {name: int((band == j).sum()) for j, (_, _, name) in enumerate(BANDS)},
           "prep_seconds": round(time.time() - t0, 1)}
    ids = torch.empty((nq, K), dtype=torch.int32, device=dev)
    dd = torch.empty((nq, K), dtype=torch.float32, device=dev)
    cnt = torch.empty((nq, 4), dtype=torch.int32, device=dev)
    steps = min(args.steps, 50)
    forms = {}
    for fname, fcode in (("fp32", jag.JAG_VEC_F32), ("bf16", jag.JAG_VEC_BF16), ("fp8", jag.JAG_VEC_FP8)):
        gi = ix32 if fcode == jag.JAG_VEC_F32 else jag.Index.from_workload(w, R=SUBSET_R, graph=graph, entry=entry,
                                                                            storage=fcode, device=local)
        chosen, per = None, None
        for beam in SUBSET_BEAMS:
            jag.jag_search(gi.h, q, ft, at, K, beam, ids, dd, None, stream, s0=S0, scan_cap=SCAN_CAP)
            torch.cuda.synchronize()
            per = band_recalls(recall_at_k(ids.cpu().numpy(), gt_ids), band)
            if all(v >= 0.95 for v in per.values()):
                chosen = beam
                break
        met = chosen is not None
        chosen = chosen or SUBSET_BEAMS[-1]
        jag.jag_search(gi.h, q, ft, at, K, chosen, ids, dd, cnt, stream, s0=S0, scan_cap=SCAN_CAP)
        torch.cuda.synchronize()
        c = cnt.cpu().numpy()
        for _ in range(3):
            jag.jag_search(gi.h, q, ft, at, K, chosen, ids, dd, None, stream, s0=S0, scan_cap=SCAN_CAP)
        evs = []
        for i in range(steps):
            flush.fill_(float(i))
            a, b, ka, kb = (torch.cuda.Event(enable_timing=True) for _ in range(4))
            ka.record(stream)
            kb.record(stream)
            a.record(stream)
            jag.jag_search(gi.h, q, ft, at, K, chosen, ids, dd, None, stream, s0=S0, scan_cap=SCAN_CAP, ev_begin=ka,
                           ev_end=kb)
            b.record(stream)
            evs.append((a, b, ka, kb))
        torch.cuda.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b, _, _ in evs]))
        kms = float(np.mean([ka.elapsed_time(kb) for _, _, ka, kb in evs]))
        row_bytes = 400 if fcode == jag.JAG_VEC_F32 else (208 if fcode == jag.JAG_VEC_BF16 else 116)
        gbytes = mixed_graph_bytes(c, row_bytes, 8, SUBSET_R)
        forms[fname] = {"beam": chosen, "recall_0.95_met": met, "qps": round(nq / (ms / 1e3), 1),
                        "ms_per_step": round(ms, 4), "graph_kernel_ms": round(kms, 3), "recall": per,
                        "routed_to_scan": int((c[:, 3] == 1).sum()),
                        "graph_kernel_gather_bytes": gbytes,
                        "graph_kernel_frac_of_hbm": round(gbytes / (kms / 1e3) / 1e9 / measured_peaks()[0], 4)}
        if fcode != jag.JAG_VEC_F32:
            forms[fname]["distance_error_vs_fp64"] = stored_distance_error(gi, w, gt_ids, fcode)
            gi.close()
        log("subset %s: beam %d, %.0f QPS, %s" % (fname, chosen, nq / (ms / 1e3), per))
    ix32.close()
    out["forms"] = forms
    return out


def serve_saturation(jag, idx, w, beam, batch_qps, n_req=2000, offered=(0.6, 1.0, 1.5)):
    """Saturated throughput of the serve loop: the largest QPS it achieves
    under Poisson arrivals of the request mix (sizes uniform in 1..256
    queries) offered at the given fractions of the batch path's QPS."""
    rng = np.random.default_rng(1)
    best = 0.0
    for frac in offered:
        sizes = rng.integers(1, 257, n_req).astype(np.int32)
        first = np.array([rng.integers(0, len(w.q) - s + 1) for s in sizes], np.int64)
        arrival = np.cumsum(rng.exponential(float(sizes.mean()) / (frac * batch_qps), n_req))
        srv = jag.Server(idx, K, beam, s0=SERVE_S0, scan_cap=SCAN_CAP, max_queries=1 << 17)
        t1 = time.perf_counter()
        srv.replay(arrival, sizes, first, w.q, w.filters, w.aux, timeout_s=300.0)
        wall = time.perf_counter() - t1
        srv.stop()
        best = max(best, float(sizes.sum()) / wall)
    return best


def measure_serving(jag, idx, w, beam, band, gt_ids, gt_d, batch_qps, n_req=2000, loads=(0.5, 0.8)):
    """The serve loop under open-loop Poisson arrivals: request sizes uniform
    in 1..256 queries (rows of the 10,000-query batch), arrival rate a
    fraction of the loop's own saturated throughput; p50 / p99 latency from
    arrival to completion, achieved QPS, and recall per band."""
    sat_qps = serve_saturation(jag, idx, w, beam, batch_qps)
    out = {"saturated_qps": round(sat_qps, 1), "s0": SERVE_S0}
    rng = np.random.default_rng(0)
    for load in loads:
        sizes = rng.integers(1, 257, n_req).astype(np.int32)
        first = np.array([rng.integers(0, len(w.q) - s + 1) for s in sizes], np.int64)
        rate = load * sat_qps / float(sizes.mean())            # requests per second
        arrival = np.cumsum(rng.exponential(1.0 / rate, n_req))
        srv = jag.Server(idx, K, beam, s0=SERVE_S0, scan_cap=SCAN_CAP, max_queries=1 << 17)
        t1 = time.perf_counter()
        ids, dist, lat, devs = srv.replay(arrival, sizes, first, w.q, w.filters, w.aux, timeout_s=300.0)
        wall = time.perf_counter() - t1
        info = srv.info()
        srv.stop()
        rows = np.unique(np.concatenate([np.arange(f, f + s) for f, s in zip(first, sizes)]))
        rec = recall_at_k(ids[rows], gt_ids[rows], gt_d[rows])
        per = {name: float(np.mean(rec[(band[rows] == j) & ~np.isnan(rec)])) for j, (_, _, name) in enumerate(BANDS)
               if ((band[rows] == j) & ~np.isnan(rec)).any()}
        out["load_%.1f" % load] = {
            "offered_qps": round(load * sat_qps, 1), "achieved_qps": round(float(sizes.sum()) / wall, 1),
            "p50_ms": round(1000 * float(np.percentile(lat, 50)), 3),
            "p99_ms": round(1000 * float(np.percentile(lat, 99)), 3),
            "device_p50_ms": round(1000 * float(np.percentile(devs, 50)), 3),
            "requests": n_req, "queries": int(sizes.sum()), "recall": per, "loop_launches": info["launches"]}
    return out


def stored_distance_error(idx, w, gt_ids, fcode, pairs=2000):
    """Relative error of the squared distance to the stored (dequantized)
    row against the fp64 distance to the fp32 row, over answer pairs."""
    rows, sc = idx.stored_rows()
    d = w.d
    rng = np.random.default_rng(0)
    qi = rng.integers(0, len(w.q), pairs)
    pi = gt_ids[qi, 0]
    ok = pi >= 0
    qi, pi = qi[ok], pi[ok]
    r = rows[pi]
    if fcode == 1:   # BF16: the upper half of an fp32 encoding
        xq = (r[:, :2 * d].copy().view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    else:            # FP8 E4M3: sign, 4-bit exponent (bias 7), 3-bit mantissa, times the row scale
        c = r[:, :d].astype(np.int64)
        e, m = (c >> 3) & 15, c & 7
        mag = np.where(e == 0, m / 8.0 * 2.0 ** -6, (1 + m / 8.0) * 2.0 ** (e - 7))
        xq = np.where(c >> 7, -mag, mag) * sc[pi][:, None].astype(np.float64)
    qq = w.q[qi].astype(np.float64)
    exact = ((qq - w.x[pi].astype(np.float64)) ** 2).sum(1)
    approx = ((qq - xq) ** 2).sum(1)
    rel = np.abs(approx - exact) / np.maximum(exact, 1e-30)
    return {"pairs": int(len(qi)), "max_rel": float(rel.max()), "mean_rel": float(rel.mean())}


def cpu_baseline(w, idx, beam, gt_ids, gt_d, budget_s=15.0):
    """The oracle's Query on the same graph and beam, all host cores, over a
    bounded sample of the batch (as many 200-query slices as fit the time
    budget)."""
    from oracle import jag_oracle as O
    graph = idx.graph()
    info = idx.info()
    ox = O.Index.from_workload(w, R=R, graph=graph, entry=info["entry"])
    cores = os.cpu_count() or 1
    done, t_total = 0, 0.0
    ids_all, cnt_all = [], []
    while done < len(w.q) and t_total < budget_s:
        sl = slice(done, min(done + 200, len(w.q)))
        t1 = time.perf_counter()
        ids, _, cn = O.query(ox, w.q[sl], w.filters[sl], w.aux, K, beam, s0=S0, scan_cap=SCAN_CAP, nthreads=cores)
        t_total += time.perf_counter() - t1
        ids_all.append(ids)
        cnt_all.append(cn)
        done = sl.stop
    ids = np.concatenate(ids_all)
    rec = recall_at_k(ids, gt_ids[:done], gt_d[:done])
    check = check_ground_truth(ox, w, gt_ids, gt_d, cores)
    return ({"value": round(done / t_total, 2), "unit": "queries/s", "cores": cores, "kind": "oracle",
             "sample": "first %d of the %d queries, beam %d, %.1f s" % (done, len(w.q), beam, t_total),
             "recall": float(np.nanmean(rec)), "ground_truth_check": check}, np.concatenate(cnt_all))


def check_ground_truth(ox, w, gt_ids, gt_d, cores, n_check=200, seed=5):
    """The recall ground truth (the GPU's exact scan of every query) against
    the oracle's brute-force filtered k-NN on a sample of queries (untimed):
    ids and fp32 distances must be identical, else the run fails."""
    from oracle import jag_oracle as O
    sample = np.sort(np.random.default_rng(seed).choice(len(w.q), min(n_check, len(w.q)), replace=False))
    bi, bd, _, _ = O.brute_force(ox, w.q[sample], w.filters[sample], w.aux, K, nthreads=cores)
    bad = sample[~((bi == gt_ids[sample]).all(axis=1) & (bd.view(np.uint32) == gt_d[sample].view(np.uint32)).all(axis=1))]
    if len(bad):
        raise RuntimeError("ground truth differs from the oracle's brute force on queries %s" % bad[:10].tolist())
    return {"queries": int(len(sample)), "mismatches": 0, "against": "oracle brute force (exact filtered k-NN)"}


def run_reference(args):
    """The oracle (plain C, host cores) as the reference arm: each step times
    Query on a bounded slice of the same batch over the same index."""
    rank, world, local = rank_env()
    if rank != 0:
        return
    import torch
    from paper_2602_10258_gb300 import jag
    from oracle import jag_oracle as O
    torch.cuda.set_device(local)
    w = make_workload(args)
    idx = jag.Index.from_workload(w, R=R, l_b=LB, alpha=ALPHA, thresholds=THRESHOLDS, device=local)
    graph, info = idx.graph(), idx.info()
    idx.close()
    ox = O.Index.from_workload(w, R=R, graph=graph, entry=info["entry"])
    cores = os.cpu_count() or 1
    beam = args.ref_beam
    per = max(50, args.ref_queries)
    times = []
    for i in range(args.warmup + args.steps):
        s = (i * per) % len(w.q)
        sl = slice(s, min(s + per, len(w.q)))
        t1 = time.perf_counter()
        O.query(ox, w.q[sl], w.filters[sl], w.aux, K, beam, s0=S0, scan_cap=SCAN_CAP, nthreads=cores)
        dt = time.perf_counter() - t1
        if i >= args.warmup:
            times.append((sl.stop - sl.start, dt))
    nq_t = sum(t[0] for t in times)
    t_t = sum(t[1] for t in times)
    value = nq_t / t_t
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": "queries/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(1000 * t_t / args.steps, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": workload_desc(w.n, w.d, len(w.q)), "beam": beam, "k": K, "R": R,
                      "index": "graph from the GPU build (index construction is not timed)"},
           "cpu_baseline": {"value": round(value, 2), "unit": "queries/s", "cores": cores, "kind": "oracle",
                            "sample": "%d queries per step, beam %d" % (per, beam)},
           "e2e": {"value": round(value, 2), "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


LARGE_BEAMS = (128, 192, 256, 320, 384, 448, 512)


def run_serve_large(args):
    print(json.dumps(measure_large(args, 0)))


def measure_large(args, local):
    """The serving form at its own scale: N = 10M, d = 100, BF16 rows (fp32
    re-rank), float attribute U[0,1), range filters of width log-uniform in
    [1e-4, 1].  The data are generated once and indexed at each degree of
    --large-r: R = 32 (the form's stated degree) and R = 64.  For each, the
    smallest beam with recall@10 >= 0.95 in every band on a ground-truth
    sample (else the largest beam, and says so), the batch search timed at
    that beam and at 256 (the serve loop's largest), then Poisson traffic
    replayed through the serve loop at beam <= 256.  Returns the R = 32
    result, with the others under "other_degrees"."""
    from paper_2602_10258_gb300 import datagen as D
    t0 = time.time()
    w = D.make_range_f32(n=args.large_n, d=100, nq=10000, seed=args.seed)
    gen_s = time.time() - t0
    srt = np.sort(w.attr_f32)
    fl = D.filter_fields(w.filters)
    sel = (np.searchsorted(srt, fl["f_hi"], "right") - np.searchsorted(srt, fl["f_lo"], "left")) / w.n
    band = band_of(sel)
    log("large: data %.1f s" % gen_s)
    outs = [measure_large_at(args, local, w, band, int(r)) for r in args.large_r.split(",")]
    out = outs[0]
    if len(outs) > 1:
        out["other_degrees"] = {"R%d" % o["config"]["R"]: o for o in outs[1:]}
    return out


def measure_large_at(args, local, w, band, degree):
    import torch
    from paper_2602_10258_gb300 import jag
    dev = torch.device("cuda", local)
    t0 = time.time()
    thr = tuple(int(v) for v in args.large_thresholds.split(","))
    idx = jag.Index.from_workload(w, R=degree, l_b=args.large_lb, alpha=args.large_alpha, thresholds=thr,
                                  storage=jag.JAG_VEC_BF16, device=local)
    build_s = time.time() - t0
    info = idx.info()
    log("large R=%d: build %.1f s (GPU %.1f s), %.2f GB on the device" % (
        degree, build_s, info["build_seconds"], info["device_bytes"] / 1e9))
    nq = len(w.q)
    q = torch.from_numpy(w.q).to(dev)
    ft = jag.filters_to_device(w.filters, dev)
    at = jag.aux_to_device(w.aux, dev)
    ns = min(args.large_gt, nq)
    t0 = time.time()
    gt = torch.empty((ns, K), dtype=torch.int32, device=dev)
    gd = torch.empty((ns, K), dtype=torch.float32, device=dev)
    jag.jag_search(idx.h, q[:ns], ft, at, K, K, gt, gd, None, None, flags=jag.JAG_SEARCH_SCAN_ALL)
    torch.cuda.synchronize()
    gt, gd = gt.cpu().numpy(), gd.cpu().numpy()
    gt_s = time.time() - t0
    ids = torch.empty((nq, K), dtype=torch.int32, device=dev)
    dd = torch.empty((nq, K), dtype=torch.float32, device=dev)
    chosen, per_chosen, sweep, per = None, None, {}, {}
    for beam in LARGE_BEAMS:
        jag.jag_search(idx.h, q, ft, at, K, beam, ids, dd, None, None, s0=S0, scan_cap=SCAN_CAP)
        torch.cuda.synchronize()
        rec = recall_at_k(ids.cpu().numpy()[:ns], gt, gd)
        per = {name: float(np.mean(rec[(band[:ns] == j) & ~np.isnan(rec)])) for j, (_, _, name) in enumerate(BANDS)
               if ((band[:ns] == j) & ~np.isnan(rec)).any()}
        sweep[beam] = {k: round(v, 4) for k, v in per.items()}
        log("large R=%d beam %d: %s" % (degree, beam, sweep[beam]))
        if all(v >= 0.95 for v in per.values()):
            chosen, per_chosen = beam, per
            break
    met = chosen is not None
    if not met:
        chosen, per_chosen = LARGE_BEAMS[-1], per
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def batch_ms(beam):
        for _ in range(3):
            jag.jag_search(idx.h, q, ft, at, K, beam, ids, dd, None, None, s0=S0, scan_cap=SCAN_CAP)
        evs = []
        for i in range(min(args.steps, 20)):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            jag.jag_search(idx.h, q, ft, at, K, beam, ids, dd, None, None, s0=S0, scan_cap=SCAN_CAP)
            b.record()
            evs.append((a, b))
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in evs]))

    ms = batch_ms(chosen)
    qps = nq / (ms / 1000.0)
    serve_beam = min(chosen, 256)
    ms_serve_beam = batch_ms(serve_beam) if serve_beam != chosen else ms
    gt_all = np.concatenate([gt, np.full((nq - ns, K), -1, np.int32)])
    gd_all = np.concatenate([gd, np.full((nq - ns, K), np.inf, np.float32)])
    serving = measure_serving(jag, idx, w, serve_beam, band, gt_all, gd_all, nq / (ms_serve_beam / 1000.0))
    serving["beam"] = serve_beam
    serving["recall_at_beam"] = sweep.get(serve_beam)
    idx.close()
    del flush, ids, dd, q
    torch.cuda.empty_cache()
    return {"metric": METRIC, "unit": "queries/s", "dtype": "bf16 rows, f32 re-rank",
            "data": "synthetic",
            "config": {"workload": "float range, width log-uniform 1e-4..1, N=%d d=100 GMM-200, 10000 queries, "
                                   "k=10, R=%d" % (w.n, degree), "R": degree, "beam": chosen, "recall_0.95_met": met,
                       "s0": S0, "scan_cap": SCAN_CAP,
                       "build": "GPU JAG build, l_b=%d, T=%s%%, alpha=%.2f" % (args.large_lb, list(thr),
                                                                                args.large_alpha),
                       "build_seconds": round(build_s, 1), "gpu_build_seconds": round(info["build_seconds"], 1),
                       "index_device_bytes": info["device_bytes"], "ground_truth_sample": ns,
                       "ground_truth_seconds": round(gt_s, 1), "beam_sweep": {str(b): v for b, v in sweep.items()}},
            "batch": {"qps": round(qps, 1), "ms_per_step": round(ms, 3), "recall": per_chosen,
                      "beam_256_qps": round(nq / (ms_serve_beam / 1000.0), 1)},
            "serving": serving}


def run_profile(args):
    """Build the index and run a few searches at a fixed beam (no sweep, no
    ground truth): the command profiled by ncu."""
    import torch
    from paper_2602_10258_gb300 import jag
    from paper_2602_10258_gb300 import datagen as D
    torch.cuda.set_device(0)
    if args.profile_workload == "subset":
        w = D.make_subset(n=args.n, d=100, nq=args.nq, seed=args.seed)
    else:
        w = make_workload(args)
    idx = jag.Index.from_workload(w, R=R, l_b=LB, alpha=ALPHA, thresholds=THRESHOLDS, storage=args.storage)
    q = torch.from_numpy(w.q).cuda()
    ft = jag.filters_to_device(w.filters, q.device)
    ids = torch.empty((len(w.q), K), dtype=torch.int32, device=q.device)
    dd = torch.empty((len(w.q), K), dtype=torch.float32, device=q.device)
    for _ in range(args.steps):
        jag.jag_search(idx.h, q, ft, jag.aux_to_device(w.aux, q.device), K, args.beam, ids, dd, None, None, s0=S0,
                       scan_cap=SCAN_CAP)
    torch.cuda.synchronize()
    log("profile run done: %d searches of %d queries at beam %d, storage %d" % (args.steps, len(w.q), args.beam,
                                                                               args.storage))
    idx.close()


def main():
    global S0, SCAN_CAP
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--nq", type=int, default=10_000)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--full-sweep", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the learned form's mixed range / boolean workload")
    ap.add_argument("--no-subset", action="store_true", help="skip the precision form's subset workload")
    ap.add_argument("--subset-only", action="store_true", help="only the precision form's subset workload")
    ap.add_argument("--mixed-train", type=int, default=100_000, help="training queries of the learned form")
    ap.add_argument("--mixed-epochs", type=int, default=40)
    ap.add_argument("--mixed-only", action="store_true", help="only the mixed workload's forms (prints its JSON)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-beam", type=int, default=192)
    ap.add_argument("--ref-queries", type=int, default=200)
    ap.add_argument("--profile", action="store_true", help="fixed-beam searches only (for ncu)")
    ap.add_argument("--serve-large", action="store_true", help="only the 10M BF16 serving form")
    ap.add_argument("--no-large", action="store_true", help="skip the 10M BF16 serving form")
    ap.add_argument("--large-n", type=int, default=10_000_000)
    ap.add_argument("--large-gt", type=int, default=2000, help="queries with ground truth in the large form")
    ap.add_argument("--large-thresholds", default="100,10,0", help="threshold percentiles of the large form's build")
    ap.add_argument("--large-lb", type=int, default=128, help="build beam of the large form")
    ap.add_argument("--large-alpha", type=float, default=ALPHA, help="pruning alpha of the large form")
    ap.add_argument("--large-r", default="32,64", help="graph degrees of the large form (the first is reported)")
    ap.add_argument("--beam", type=int, default=192)
    ap.add_argument("--profile-workload", default="label", choices=["label", "subset"],
                    help="workload of the --profile run: the label workload or the precision form's subset one")
    ap.add_argument("--storage", type=int, default=0, help="row storage of the --profile run: 0 fp32, 1 BF16, 2 FP8")
    ap.add_argument("--s0", type=int, default=None, help="scan route threshold (default %d)" % S0)
    ap.add_argument("--scan-cap", type=int, default=None, help="largest scanned set (default %d)" % SCAN_CAP)
    args = ap.parse_args()
    if args.s0 is not None:
        S0 = args.s0
    if args.scan_cap is not None:
        SCAN_CAP = args.scan_cap
    if args.warmup < 3:
        args.warmup = 3
    if args.subset_only:
        import torch
        torch.cuda.set_device(0)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        print(json.dumps(measure_subset(args, 0, flush, torch.cuda.current_stream())))
    elif args.mixed_only:
        import torch
        torch.cuda.set_device(0)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        print(json.dumps(measure_mixed(args, 0, flush, torch.cuda.current_stream())))
    elif args.profile:
        run_profile(args)
    elif args.serve_large:
        run_serve_large(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
