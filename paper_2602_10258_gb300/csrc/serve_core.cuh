// Device-resident request loop (serving with continuous batching).
//
// A persistent kernel: each warp repeatedly claims the next published query
// (a global index over all requests, in publication order, handed out as
// tickets; see serve_claim), finds its
// request through the query map, answers it exactly as the batched search
// does (the plan of plan_query, then the exact scan or GreedySearch of
// Algorithm 1 with D_F, then the fp32 re-rank for BF16 / FP8 rows) and writes
// the answers straight into the request's output rows in mapped host memory.
// The warp that finishes a request's last query writes its completion record.
// Requests, their inputs and outputs live in pinned host memory the host
// writes and reads directly; the only device-side state is the claim counter,
// the published count last read from the host, and per-slot completion
// counters.
//
// Every wait is bounded: a warp with nothing to claim backs off with
// __nanosleep and exits after idle_ns without work or once the host sets
// stop; the host launches the loop again when new work arrives.
#pragma once

#include "plan.cuh"
#include "search_core.cuh"

namespace jag {

// One request, written by the host before it publishes the request's
// queries (mapped host memory).
struct ServeReq {
  uint64_t ticket;
  int64_t qbase;        // global index of its first query
  int32_t nq, pad0;
  int64_t q_off, f_off, aux_off, aux_bytes, ids_off, dist_off;   // arena byte offsets
  int64_t lut_off;      // byte offset of its boolean tables in the device scratch
};

// Completion record of the request in a slot (mapped host memory, device
// writes; ticket last).
struct ServeDone {
  unsigned long long ticket;
  unsigned long long t_first, t_end;   // %globaltimer, ns
  uint32_t status, pad;
};

// Host-written control words (mapped host memory).
struct ServeCtl {
  unsigned long long published;   // queries published so far
  unsigned int stop;
  unsigned int pad;
};

// Device-memory state of a server.
struct ServeDev {
  unsigned long long claimed;        // queries claimed so far
  unsigned long long queries_done;
  unsigned long long pub_seen;       // the largest published count a warp has read from the host
  unsigned long long bad_claims;     // claimed queries whose map entry named another request (skipped)
};

struct ServeArgs {
  DevIndex ix;
  int d, k, ls, hbits;
  int64_t s0, cap;
  const ServeCtl *ctl;
  const ServeReq *ring;
  ServeDone *done;
  const uint32_t *qmap;             // slot of global query c at c % qcap
  int64_t qcap;
  uint8_t *arena;                   // device view of the host arena
  uint8_t *lut;                     // device scratch for boolean tables
  ServeDev *dev;
  int32_t *done_cnt;                // [slots] queries finished per slot
  uint32_t *req_status;             // [slots]
  unsigned long long *t_first;      // [slots]
  unsigned long long idle_ns;
  jag_policy pol;
  int has_policy;
  int nslots;                       // request slots (ring, done, done_cnt, ... entries)
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned int ld_volatile_u32(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_sys(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void max_release_gpu(unsigned long long *p, unsigned long long v) {
  asm volatile("red.release.gpu.global.max.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_gpu(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Claim the next query (lane 0 only): returns 1 with its index in *c0, 0 to
// exit (stop, or idle for longer than idle_ns).
//
// A claim is a ticket from one atomicAdd on the claim counter, taken once
// the warp has seen published work nobody claimed; with many warps some
// tickets run ahead of what is published, and their holders wait, in ticket
// order, for the host to publish them.  (A compare-and-swap claim never runs
// ahead, but under contention only one succeeds per round trip to L2, which
// caps dispatch near two million queries a second.)  The holder of the
// oldest unpublished ticket reads the host's published count (acquire,
// system scope) and passes it on in device memory (release / acquire, GPU
// scope), which carries the host's writes along; the others read only that
// copy.  A holder idle for idle_ns gives its ticket back when it is the
// newest one (one compare-and-swap), so tickets return in the reverse order
// of their claims and none is lost or handed out twice.
__device__ inline int serve_claim(const ServeArgs &a, unsigned long long *c0) {
  unsigned long long t0 = global_ns();
  unsigned int nap = 64;
  for (;;) {   // no ticket yet
    unsigned long long p = ld_acquire_gpu(&a.dev->pub_seen);
    const unsigned long long c = ld_relaxed_gpu(&a.dev->claimed);
    if (c >= p) {
      const unsigned long long h = ld_acquire_sys(&a.ctl->published);
      if (h > p) {
        max_release_gpu(&a.dev->pub_seen, h);
        p = h;
      }
    }
    if (c < p) break;
    if (ld_volatile_u32(&a.ctl->stop)) return 0;
    if (global_ns() - t0 > a.idle_ns) return 0;
    __nanosleep(nap);
    if (nap < 8192) nap <<= 1;
  }
  const unsigned long long t = atomicAdd(&a.dev->claimed, 1ull);
  t0 = global_ns();
  nap = 32;
  for (;;) {   // holding ticket t
    const unsigned long long p = ld_acquire_gpu(&a.dev->pub_seen);
    if (t < p) {
      *c0 = t;
      return 1;
    }
    if (t == p) {   // the oldest unpublished ticket
      const unsigned long long h = ld_acquire_sys(&a.ctl->published);
      if (h > p) {
        max_release_gpu(&a.dev->pub_seen, h);
        continue;
      }
    }
    if (ld_volatile_u32(&a.ctl->stop)) return 0;
    if (global_ns() - t0 > a.idle_ns && atomicCAS(&a.dev->claimed, t + 1, t) == t + 1) return 0;
    __nanosleep(nap);
    if (nap < 4096) nap <<= 1;
  }
}

// Merge the exact fp32 distances of nc candidates ids[0..nc) into the sorted
// top-k list of S (count cnt); returns the new count.
template <int CAP, int PF, int CPLF>
__device__ __forceinline__ int scan_merge(const DevIndex &ix, const QChunks<CPLF, JAG_VEC_F32> &qf,
                                          const WarpSmem &S, const uint32_t *ids, int nc, int cnt, int k) {
  const int lane = threadIdx.x & 31;
  const bool full = cnt == k;
  const uint64_t tkey = full ? S.bkey[k - 1] : kNoKey;
  const uint32_t tid = full ? (S.bid[k - 1] & ~kExpanded) : kEmptySlot;
  const float dist = candidate_distances<PF, CPLF, 4, JAG_VEC_F32, true>(ix, qf, ids, nc);
  uint64_t ck = kNoKey;
  uint32_t cv = kEmptySlot;
  if (lane < nc) {
    ck = make_key(0u, dist);
    cv = ids[lane];
    if (full && !key_less(ck, cv, tkey, tid)) { ck = kNoKey; cv = kEmptySlot; }
  }
  int r0;
  return merge_candidates<CAP, false>(S.bkey, S.bid, cnt, k, ck, cv, r0);
}

// Exact top-k over the ids of a sorted-column slice (the scan route of
// label / range filters).
template <int CAP, int PF, int CPLF>
__device__ int scan_slice(const DevIndex &ix, const QChunks<CPLF, JAG_VEC_F32> &qf, const WarpSmem &S,
                          const int32_t *ids, int64_t m, int k) {
  const int lane = threadIdx.x & 31;
  int cnt = 0;
  for (int64_t b = 0; b < m; b += 32) {
    const int nc = (int)min64(32, m - b);
    __syncwarp();
    if (lane < nc) S.cid[lane] = (uint32_t)ids[b + lane];
    __syncwarp();
    cnt = scan_merge<CAP, PF, CPLF>(ix, qf, S, S.cid, nc, cnt, k);
  }
  return cnt;
}

// The scan route of subset / boolean filters: one pass over the mask column
// collects the passing points (64-entry buffer S.cid .. S.ck1) and ranks
// them 32 at a time.  If more than cap points pass, *over is set and the
// query goes to the graph search, as in the batched path.
template <int CAP, int PF, int CPLF>
__device__ int scan_masks(const DevIndex &ix, const QChunks<CPLF, JAG_VEC_F32> &qf, const WarpSmem &S,
                          const jag_filter &f, const uint8_t *tt, int64_t cap, int k, bool *over) {
  constexpr int U = 8;   // mask loads in flight per lane
  const int lane = threadIdx.x & 31;
  uint32_t *buf = S.cid;
  int cnt = 0, held = 0;
  int64_t total = 0;
  *over = false;
  for (int64_t base = 0; base < ix.n; base += 32 * U) {
    uint64_t a[U];
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int64_t u = base + j * 32 + lane;
      a[j] = u < ix.n ? __ldg(ix.a_mask + u) : 0ull;
    }
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int64_t u = base + j * 32 + lane;
      bool pass = false;
      if (u < ix.n) {
        if (f.kind == JAG_F_SUBSET) pass = (f.payload & a[j]) == f.payload;
        else { const uint32_t s = compress_bits(a[j], f.payload); pass = (tt[s >> 3] >> (s & 7)) & 1; }
      }
      const uint32_t m = __ballot_sync(kFull, pass);
      if (!m) continue;
      total += __popc(m);
      if (total > cap) { *over = true; return 0; }
      if (pass) buf[held + __popc(m & lanemask_lt())] = (uint32_t)u;
      held += __popc(m);
      __syncwarp();
      if (held >= 32) {
        cnt = scan_merge<CAP, PF, CPLF>(ix, qf, S, buf, 32, cnt, k);
        __syncwarp();
        const uint32_t rest = lane < held - 32 ? buf[32 + lane] : 0u;
        __syncwarp();
        if (lane < held - 32) buf[lane] = rest;
        held -= 32;
        __syncwarp();
      }
    }
  }
  if (held > 0) cnt = scan_merge<CAP, PF, CPLF>(ix, qf, S, buf, held, cnt, k);
  return cnt;
}

__device__ __forceinline__ void pad_rows(int k, int32_t *oid, float *od) {
  for (int j = threadIdx.x & 31; j < k; j += 32) { oid[j] = -1; od[j] = __int_as_float(0x7F800000); }
}

// One query, answered as the batched search answers it.  P / CPL: lane
// mapping of the stored rows (format FMT); CPLF: chunks per lane of the fp32
// rows with 32 lanes per row (the exact scan and the re-rank).
template <int CAP, int P, int CPL, int FMT, bool POL, int CPLF>
__device__ void serve_query(const ServeArgs &a, const WarpSmem &S, const jag_filter &f,
                            const float *qv, const uint8_t *aux, int64_t aux_bytes, uint8_t *lut_base,
                            int32_t *oid, float *od, uint32_t *status) {
  const int lane = threadIdx.x & 31;
  const DevIndex &ix = a.ix;
  QueryPlan pl;
  if (!plan_query(ix, f, aux, aux_bytes, a.s0, a.cap, 0, POL ? 1 : 0, lut_base, pl)) {
    pad_rows(a.k, oid, od);
    if (lane == 0) atomicOr(status, kErrBadFilter);
    return;
  }
  QChunks<CPLF, JAG_VEC_F32> qf;
  load_point<32, CPLF, JAG_VEC_F32>(qv, a.d, qf);
  if (pl.route == kRouteSlice) {
    const int32_t *ids = (f.kind == JAG_F_RANGE_F32 ? ix.sf32_id : ix.si32_id) + pl.begin;
    const int cnt = scan_slice<CAP, 32, CPLF>(ix, qf, S, ids, pl.end - pl.begin, a.k);
    write_answers(S, cnt, 0, a.k, oid, od);
    return;
  }
  if (pl.route == kRouteList) {
    bool over;
    const uint8_t *tt = f.kind == JAG_F_BOOL ? aux + f.aux_off : nullptr;
    const int cnt = scan_masks<CAP, 32, CPLF>(ix, qf, S, f, tt, a.cap, a.k, &over);
    if (!over) {
      write_answers(S, cnt, 0, a.k, oid, od);
      return;
    }
  }
  // graph route: GreedySearch with D_F
  QChunks<CPL, FMT> q;
  load_point<P, CPL, FMT>(qv, a.d, q);
  const QueryKey key{f.kind, f.payload, pl.lut_off >= 0 ? lut_base + pl.lut_off : nullptr};
  NoSink sink;
  SearchStats st;
  int cnt;
  if constexpr (POL) {
    const int64_t sample = ix.n < 4096 ? ix.n : 4096;
    const int64_t est = (f.kind == JAG_F_SUBSET || f.kind == JAG_F_BOOL) ? (int64_t)pl.est * ix.n / sample
                        : (f.kind == JAG_F_NONE ? ix.n : (int64_t)pl.est);
    // as the batch path: the plain loop up to h0, the decision outside it
    // (scratch: the free candidate arrays), the loop re-entered
    SearchCursor cur{0, 0};
    int lsq = a.ls, lim = a.pol.mode != JAG_POLICY_PLAIN ? a.pol.h0 : 0x7FFFFFFF;
    bool decided = false;
    for (;;) {
      cnt = greedy_search<CAP, P, CPL, FMT, 0, true>(ix, key, q, lsq, a.hbits, S, sink, st, lim, &cur);
      if (decided || st.hops < lim) break;
      __syncwarp();
      const PolicyOut o = policy_decide(a.pol, S, reinterpret_cast<float *>(S.cid), cnt, a.k, est, f.kind, a.ls,
                                        nullptr, nullptr);
      __syncwarp();
      decided = true;
      lsq = o.beam;
      if (cnt > lsq) cnt = lsq;
      if (o.stop > 0 && st.hops >= o.stop) break;
      lim = o.stop > 0 ? o.stop : 0x7FFFFFFF;
      cur.cnt = cnt;
    }
  } else {
    cnt = greedy_search<CAP, P, CPL, FMT, 0>(ix, key, q, a.ls, a.hbits, S, sink, st);
  }
  if (FMT == JAG_VEC_F32) {
    write_answers(S, cnt, 0, a.k, oid, od);
    return;
  }
  // BF16 / FP8 rows: the leading min(4k, l_s) passing entries of L, ranked
  // again by exact fp32 distance (their ids parked in the visited table)
  const int rr = 4 * a.k < a.ls ? 4 * a.k : a.ls;
  int np = 0;
  for (int b = 0; b < rr && b < cnt; b += 32) {
    const int j = b + lane;
    const bool ok = j < rr && j < cnt && (S.bkey[j] >> 32) == 0;
    const uint32_t m = __ballot_sync(kFull, ok);
    if (ok) S.hash[j] = S.bid[j] & ~kExpanded;
    np += __popc(m);
    if (m != kFull) break;   // passing entries form a prefix of L
  }
  __syncwarp();
  int c2 = 0;
  for (int b = 0; b < np; b += 32) c2 = scan_merge<CAP, 32, CPLF>(ix, qf, S, S.hash + b, min(32, np - b), c2, a.k);
  write_answers(S, c2, 0, a.k, oid, od);
}

// Rows of one chunk per lane (d <= 128 fp32): 6 CTAs per SM (at most 85
// registers, no spill), 24 warps.  Measured on the 1M label index: 4 / 6 / 8
// CTAs saturate at 4.18 / 5.71 / 6.36 M QPS with request p99 at 0.8 of that
// of 1.9 / 2.0 / 3.0 ms (8 CTAs spill at 64 registers).
template <int CAP, int P, int CPL, int FMT, bool POL, int CPLF>
__global__ void __launch_bounds__(kSearchWarps * 32, CPLF == 1 ? 6 : 1)
serve_kernel(const __grid_constant__ ServeArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lcap = list_slots(a.ls);
  const size_t wbytes = warp_smem_bytes(lcap, a.hbits);
  uint8_t *wb = smem + warp * wbytes;
  const WarpSmem S = carve_warp_smem(wb, lcap, a.hbits);
  for (;;) {
    unsigned long long c = 0;
    int got = 0;
    if (lane == 0) got = serve_claim(a, &c);
    got = __shfl_sync(kFull, got, 0);
    c = __shfl_sync(kFull, c, 0);
    if (!got) return;
    const uint32_t slot = a.qmap[(unsigned long long)c % (unsigned long long)a.qcap];
    const ServeReq rq = a.ring[slot < (uint32_t)a.nslots ? slot : 0u];
    const int64_t i = c - rq.qbase;
    // cannot happen while the host keeps the map's window; never read out of range
    if (slot >= (uint32_t)a.nslots || i < 0 || i >= rq.nq) {
      if (lane == 0) atomicAdd(&a.dev->bad_claims, 1ull);
      __syncwarp();
      continue;
    }
    if (i == 0 && lane == 0) a.t_first[slot] = global_ns();
    const jag_filter f = reinterpret_cast<const jag_filter *>(a.arena + rq.f_off)[i];
    const float *qv = reinterpret_cast<const float *>(a.arena + rq.q_off) + i * a.d;
    int32_t *oid = reinterpret_cast<int32_t *>(a.arena + rq.ids_off) + i * a.k;
    float *od = reinterpret_cast<float *>(a.arena + rq.dist_off) + i * a.k;
    serve_query<CAP, P, CPL, FMT, POL, CPLF>(a, S, f, qv, a.arena + rq.aux_off, rq.aux_bytes,
                                             a.lut + rq.lut_off, oid, od, a.req_status + slot);
    // answers visible system-wide before the count that may complete the request
    __threadfence_system();
    __syncwarp();
    if (lane == 0) {
      __threadfence_system();
      const int old = atomicAdd(a.done_cnt + slot, 1);
      atomicAdd(&a.dev->queries_done, 1ull);
      if (old == rq.nq - 1) {
        __threadfence();
        ServeDone *dn = a.done + slot;
        dn->t_first = a.t_first[slot];
        dn->t_end = global_ns();
        dn->status = a.req_status[slot];
        a.done_cnt[slot] = 0;
        a.req_status[slot] = 0;
        __threadfence_system();
        st_release_sys(&dn->ticket, rq.ticket);
      }
    }
    __syncwarp();
  }
}

// Launch of the loop for one row format (instantiated in serve_*.cu).
template <int FMT>
cudaError_t launch_serve_fmt(const ServeArgs &a, int ctas, cudaStream_t stream, int *grid_out);

}  // namespace jag
