// Query path kernels: filter preparation and routing, attribute gather for
// routed subset/boolean filters, the query kernel (graph search or exact scan
// per query) and the brute-force scan.
#include <algorithm>
#include <mutex>

#include "launch.h"
#include "launch_util.cuh"
#include "plan.cuh"
#include "search_core.cuh"

namespace jag {

constexpr int kPrepWarps = 8;
constexpr int kGatherTile = 4096;
constexpr int kGatherQPB = 64;   // queries per gather CTA

__device__ __forceinline__ void pad_outputs(int64_t qi, int k, int32_t *out_ids, float *out_dist) {
  const int lane = threadIdx.x & 31;
  for (int j = lane; j < k; j += 32) {
    out_ids[qi * k + j] = -1;
    out_dist[qi * k + j] = __int_as_float(0x7F800000);
  }
}

// K0: validate each filter, build boolean tables, and route the query:
// label/range filters count their passing set exactly (binary search in the
// sorted column); subset/boolean filters are estimated on the fixed sample of
// S = min(4096, n) points with ids floor(j n / S).  A query whose count
// (estimate) is below s0 goes to the exact scan.
__global__ void __launch_bounds__(kPrepWarps * 32)
prep_kernel(DevIndex ix, const jag_filter *filters, const uint8_t *aux, int64_t aux_bytes, int64_t nq,
            int64_t s0, int64_t cap, int scan_all, int need_est, QueryPlan *plans, uint8_t *lut_base,
            int32_t *list_counts, int k,
            int32_t *out_ids, float *out_dist, int32_t *counters, uint32_t *status) {
  const int lane = threadIdx.x & 31;
  const int64_t wstride = (int64_t)gridDim.x * kPrepWarps;
  for (int64_t qi = (int64_t)blockIdx.x * kPrepWarps + (threadIdx.x >> 5); qi < nq; qi += wstride) {
    const jag_filter f = filters[qi];
    QueryPlan pl;
    pl.route = kRouteGraph; pl.lut_off = -1; pl.begin = 0; pl.end = 0; pl.count = 0; pl.est = 0;
    const bool ok = plan_query(ix, f, aux, aux_bytes, s0, cap, scan_all, need_est, lut_base, pl);
    if (!ok) {
      if (lane == 0) {
        plans[qi] = pl;
        atomicOr(status, kErrBadFilter);
        if (counters) { counters[qi * 4 + 0] = 0; counters[qi * 4 + 1] = 0; counters[qi * 4 + 2] = 0; counters[qi * 4 + 3] = 0; }
      }
      pad_outputs(qi, k, out_ids, out_dist);
      continue;
    }
    if (pl.route == kRouteList && lane == 0) list_counts[qi] = 0;
    if (lane == 0) plans[qi] = pl;
  }
}

// Exact key of a list-routed filter, shared by identical filters: a subset
// filter's required bits (below bit 62), or a boolean filter over m <= 4 bits
// as its m, bit positions and truth table.  false: no shareable key (the
// query gathers a list of its own).
__device__ __forceinline__ bool list_key(const jag_filter &f, const uint8_t *aux, uint64_t *key) {
  if (f.kind == JAG_F_SUBSET) {
    if (f.payload >> 62) return false;
    *key = (1ull << 62) | f.payload;
    return true;
  }
  if (f.kind != JAG_F_BOOL) return false;
  const int m = __popcll(f.payload);
  if (m > 4) return false;
  uint64_t pos = 0;
  int j = 0;
  for (uint64_t v = f.payload; v; v &= v - 1, ++j) pos |= (uint64_t)(__ffsll((long long)v) - 1) << (6 * j);
  uint64_t t = aux[f.aux_off];
  if (m == 4) t |= (uint64_t)aux[f.aux_off + 1] << 8;
  if (m < 3) t &= (1ull << (1 << m)) - 1;   // the 2^m bits of the table
  *key = (1ull << 63) | ((uint64_t)m << 56) | (t << 24) | pos;
  return true;
}

__device__ __forceinline__ uint64_t mix64(uint64_t v) {
  v ^= v >> 33; v *= 0xFF51AFD7ED558CCDull; v ^= v >> 33; v *= 0xC4CEB9FE1A85EC53ull; v ^= v >> 33;
  return v;
}

// K1a: list-routed queries with the same filter join one hash slot; the
// slot's leader is its lowest query index (lslot[qi] = slot, -1 if the
// filter has no shareable key).
__global__ void list_group_kernel(const QueryPlan *plans, const jag_filter *filters, const uint8_t *aux, int64_t nq,
                                  uint64_t *hkey, int32_t *hlead, uint32_t hmask, int32_t *lslot) {
  const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (qi >= nq) return;
  if (plans[qi].route != kRouteList) return;
  uint64_t key;
  if (!list_key(filters[qi], aux, &key)) { lslot[qi] = -1; return; }
  uint32_t h = (uint32_t)mix64(key) & hmask;
  for (uint32_t probe = 0; probe <= hmask; ++probe) {   // at least 2 nq slots
    const unsigned long long old = atomicCAS((unsigned long long *)&hkey[h], ~0ull, (unsigned long long)key);
    if (old == ~0ull || old == key) break;
    h = (h + 1) & hmask;
  }
  atomicMin(&hlead[h], (int32_t)qi);
  lslot[qi] = (int32_t)h;
}

// K1b: every list-routed query records its leader in plan.begin (the query
// whose gathered list it reads); leaders are listed for the gather: subset
// filters with a required bit (gathered from a posting list) from the front
// of `leaders`, the others (a pass over the mask column) from the back.
__global__ void list_leader_kernel(QueryPlan *plans, const jag_filter *filters, int64_t nq, const int32_t *hlead,
                                   const int32_t *lslot, int32_t *leaders, unsigned long long *nlead) {
  const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (qi >= nq) return;
  if (plans[qi].route != kRouteList) return;
  const int32_t s = lslot[qi];
  const int64_t lead = s < 0 ? qi : hlead[s];
  plans[qi].begin = lead;
  if (lead != qi) return;
  const jag_filter f = filters[qi];
  if (f.kind == JAG_F_SUBSET && f.payload != 0) leaders[atomicAdd(&nlead[0], 1ull)] = (int32_t)qi;
  else leaders[nq - 1 - (int64_t)atomicAdd(&nlead[1], 1ull)] = (int32_t)qi;
}

// K2a: kPostParts CTAs per subset leader walk the posting list of its rarest
// required bit, one part each, and keep the points that hold every required
// bit (in any order: the scan's answers do not depend on it); each lane
// keeps kPostUnroll loads in flight.  Past cap points the list is full and
// the count only has to exceed cap (the query then goes to the graph).
constexpr int kPostWarps = 8;
constexpr int kPostUnroll = 4;
constexpr int kPostParts = 8;   // CTAs per leader, each over one part of its posting list

__global__ void __launch_bounds__(kPostWarps * 32)
gather_postings_kernel(DevIndex ix, const jag_filter *filters, const int32_t *leaders,
                       const unsigned long long *nlead, int64_t cap, int32_t *lists, int32_t *counts) {
  const int64_t w = blockIdx.x;
  if (w >= (int64_t)nlead[0]) return;
  const int lane = threadIdx.x & 31;
  const int64_t qi = leaders[w];
  const uint64_t f = filters[qi].payload;
  int jb = 0;
  int64_t best = INT64_MAX;
  for (uint64_t v = f; v; v &= v - 1) {
    const int j = __ffsll((long long)v) - 1;
    const int64_t len = ix.bit_off[j + 1] - ix.bit_off[j];
    if (len < best) { best = len; jb = j; }
  }
  // this CTA's part of the list; positions come from the leader's count
  // (zeroed by the preparation kernel), so the parts fill one list
  const int64_t l0 = ix.bit_off[jb], len = ix.bit_off[jb + 1] - l0;
  const int64_t b0 = l0 + len * blockIdx.y / kPostParts, b1 = l0 + len * (blockIdx.y + 1) / kPostParts;
  constexpr int kStep = kPostWarps * 32 * kPostUnroll;
  int seen = 0;   // the leader's count as this warp last saw it
  for (int64_t b = b0 + (threadIdx.x >> 5) * 32 * kPostUnroll; b < b1; b += kStep) {
    if (seen > cap) break;   // full: the count is already past cap
    int32_t u[kPostUnroll];
    uint64_t a[kPostUnroll];
#pragma unroll
    for (int r = 0; r < kPostUnroll; ++r) {
      const int64_t e = b + r * 32 + lane;
      u[r] = e < b1 ? ix.bit_ids[e] : -1;
    }
#pragma unroll
    for (int r = 0; r < kPostUnroll; ++r) a[r] = u[r] >= 0 ? ix.a_mask[u[r]] : 0ull;
#pragma unroll
    for (int r = 0; r < kPostUnroll; ++r) {
      const bool pass = u[r] >= 0 && (a[r] & f) == f;
      const uint32_t m = __ballot_sync(kFull, pass);
      if (!m) continue;
      int off = 0;
      if (lane == 0) off = atomicAdd(counts + qi, __popc(m));
      off = __shfl_sync(kFull, off, 0);
      seen = off + __popc(m);
      if (pass) {
        const int64_t pos = off + __popc(m & lanemask_lt());
        if (pos < cap) lists[qi * cap + pos] = u[r];
      }
    }
  }
}

// The leader's count past cap is only known to exceed it: it reads cap + 1.
__global__ void clamp_counts_kernel(const int32_t *leaders, const unsigned long long *nlead, int64_t cap,
                                    int32_t *counts) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= (int64_t)nlead[0]) return;
  const int64_t qi = leaders[w];
  if (counts[qi] > cap) counts[qi] = (int32_t)cap + 1;
}

// K2b: one pass over a tile of masks evaluates the predicates of up to
// kGatherQPB other leaders (boolean filters, or subset filters with no
// required bit) and appends the passing ids to their lists.
__global__ void __launch_bounds__(256)
gather_list_kernel(DevIndex ix, const jag_filter *filters, const uint8_t *aux, const int32_t *leaders, int64_t nq,
                   const unsigned long long *nlead, int64_t cap, int32_t *lists, int32_t *counts) {
  __shared__ uint64_t sm[kGatherTile];
  const int64_t t0 = (int64_t)blockIdx.x * kGatherTile;
  const int64_t t1 = min64(ix.n, t0 + kGatherTile);
  const int64_t q0 = (int64_t)blockIdx.y * kGatherQPB;
  const int64_t nl = (int64_t)*nlead;   // the leaders at leaders[0 .. nl) (the back of the array)
  if (q0 >= nl) return;
  for (int64_t i = t0 + threadIdx.x; i < t1; i += blockDim.x) sm[i - t0] = ix.a_mask[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int qq = warp; qq < kGatherQPB; qq += nw) {
    if (q0 + qq >= nl) break;
    const int64_t qi = leaders[nq - 1 - (q0 + qq)];
    const jag_filter f = filters[qi];
    const uint8_t *tt = f.kind == JAG_F_BOOL ? aux + f.aux_off : nullptr;
    for (int64_t b = t0; b < t1; b += 32) {
      const int64_t u = b + lane;
      bool pass = false;
      if (u < t1) {
        const uint64_t a = sm[u - t0];
        if (f.kind == JAG_F_SUBSET) pass = (f.payload & a) == f.payload;
        else { const uint32_t s = compress_bits(a, f.payload); pass = (tt[s >> 3] >> (s & 7)) & 1; }
      }
      const uint32_t m = __ballot_sync(kFull, pass);
      if (!m) continue;
      int off = 0;
      if (lane == 0) off = atomicAdd(&counts[qi], __popc(m));
      off = __shfl_sync(kFull, off, 0);
      if (pass) {
        const int64_t pos = off + __popc(m & lanemask_lt());
        if (pos < cap) lists[qi * cap + pos] = (int32_t)u;
      }
    }
  }
}

// A list-routed query takes its leader's passing count; one whose passing
// set exceeds the scan capacity goes back to the graph search.
__global__ void finalize_routes_kernel(QueryPlan *plans, const int32_t *counts, int64_t nq, int64_t cap) {
  const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (qi >= nq) return;
  if (plans[qi].route != kRouteList) return;
  const int32_t c = counts[plans[qi].begin];
  plans[qi].count = c;
  if (c > cap) plans[qi].route = kRouteGraph;
}

// Rows of the nc candidates cid[0..nc) copied into shared memory with
// asynchronous 16-byte copies, issued as one commit group (not waited for).
__device__ __forceinline__ void stage_rows_issue(const DevIndex &ix, const uint32_t *cid, int nc, float *rows) {
  const int lane = threadIdx.x & 31;
  const int nch = ix.nchunks;
  const int total = nc * nch;
  for (int i = lane; i < total; i += 32) {
    const int c = i / nch, ch = i - c * nch;
    const float *src = ix.x + (int64_t)cid[c] * ix.xs + ch * 4;
    const unsigned dst = (unsigned)__cvta_generic_to_shared(rows + (size_t)c * ix.xs + ch * 4);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// Distances from the lane-held chunks q to nc rows staged in shared memory,
// in the same lane mapping and rounding order as candidate_distances.
template <int P, int CPL>
__device__ __forceinline__ float staged_distances(const QChunks<CPL, JAG_VEC_F32> &q, const float *rows, int64_t xs,
                                                  int nchunks, int nc) {
  constexpr int VPW = 32 / P;
  constexpr int U = 4;   // rows reduced together
  const int lane = threadIdx.x & 31;
  const int grp = lane / P, lig = lane % P;
  float mine = 0.f;
  for (int base = 0; base < nc; base += U * VPW) {
    float acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int c = base + u * VPW + grp;
      acc[u] = 0.f;
      if (c < nc) {
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
          const int ch = lig + j * 32;
          if (ch < nchunks)
            acc[u] = chunk_accumulate(acc[u], q.v[j][0], *reinterpret_cast<const float4 *>(rows + c * xs + ch * 4));
        }
      }
    }
    const float tot = group_reduce_spread<P, U>(acc);
    const int rel = lane - base;
    const bool mine_here = rel >= 0 && rel < VPW * U;
    const float v = __shfl_sync(kFull, tot, mine_here ? spread_source<P, U>(rel / VPW, rel % VPW) : 0);
    if (mine_here) mine = v;
  }
  return mine;
}

__device__ __forceinline__ void routed_candidates(const DevIndex &ix, const jag_filter *filters,
                                                  const QueryPlan &pl, int64_t qi, const int32_t *lists,
                                                  int64_t cap, const int32_t **ids, int64_t *m) {
  if (pl.route == kRouteSlice) {
    const int32_t kind = filters[qi].kind;
    *ids = (kind == JAG_F_RANGE_F32 ? ix.sf32_id : ix.si32_id) + pl.begin;
    *m = pl.end - pl.begin;
  } else {
    *ids = lists + pl.begin * cap;   // the list of the query's leader (the same filter)
    *m = pl.count;
  }
}

// K3: exact scan of the scan-routed queries.  A warp takes one tile of one
// query's passing set (a slice of the sorted column for label and range
// filters, the gathered list for subset and boolean ones), stages its rows
// in shared memory round by round, and leaves the tile's top k in a partial
// list; merge_scan_kernel combines a query's partial lists.
// Warps per CTA of the exact scan: two, so that a scan CTA fits on an SM as
// soon as little of the graph search's last wave has left it.
constexpr int kScanWarps = 2;

template <int CAP, int P, int CPL>
__global__ void __launch_bounds__(kScanWarps * 32)
scan_tile_kernel(DevIndex ix, const float *queries, int d, const jag_filter *filters, const QueryPlan *plans,
                 const int32_t *lists, int64_t cap, int k, int64_t tile, int ntiles, int rpr, const uint64_t *items,
                 const unsigned long long *nitems, unsigned long long *work, uint64_t *part_key,
                 uint32_t *part_id) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lcap = list_slots(k);
  const size_t head = warp_smem_bytes(lcap, 5) + 32 * 4;   // list, small arrays, second id slot
  uint8_t *wb = smem + warp * (head + 2 * (size_t)rpr * ix.xs * 4);
  const WarpSmem S = carve_warp_smem(wb, lcap, 5);
  uint32_t *cids[2] = {S.cid, reinterpret_cast<uint32_t *>(wb + warp_smem_bytes(lcap, 5))};
  float *rows[2] = {reinterpret_cast<float *>(wb + head), reinterpret_cast<float *>(wb + head) + (size_t)rpr * ix.xs};
  const unsigned long long total = *nitems;
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(work, 1ull);
    it = __shfl_sync(kFull, it, 0);
    if (it >= total) return;
    const uint64_t item = items[it];
    const int64_t qi = (int64_t)(item >> 20);
    const int t = (int)(item & 0xFFFFF);
    const QueryPlan pl = plans[qi];
    const int32_t *ids;
    int64_t m;
    routed_candidates(ix, filters, pl, qi, lists, cap, &ids, &m);
    const int64_t b0 = (int64_t)t * tile;
    const int64_t b1 = min64(m, b0 + tile);
    QChunks<CPL, JAG_VEC_F32> q;
    load_point<P, CPL>(queries + qi * d, d, q);
    int cnt = 0;
    // round r covers [b0 + r*rpr, ...); round r+1 is in flight while r is reduced
    const int nr = (int)((b1 - b0 + rpr - 1) / rpr);
    {
      const int nc0 = (int)min64(rpr, b1 - b0);
      if (lane < nc0) cids[0][lane] = (uint32_t)ids[b0 + lane];
      __syncwarp();
      stage_rows_issue(ix, cids[0], nc0, rows[0]);
    }
    for (int r = 0; r < nr; ++r) {
      const int cur = r & 1;
      const int64_t b = b0 + (int64_t)r * rpr;
      const int nc = (int)min64(rpr, b1 - b);
      if (r + 1 < nr) {
        const int64_t bn = b + rpr;
        const int ncn = (int)min64(rpr, b1 - bn);
        if (lane < ncn) cids[cur ^ 1][lane] = (uint32_t)ids[bn + lane];
        __syncwarp();
        stage_rows_issue(ix, cids[cur ^ 1], ncn, rows[cur ^ 1]);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
      }
      __syncwarp();
      const bool full = cnt == k;
      const uint64_t tkey = full ? S.bkey[k - 1] : kNoKey;
      const uint32_t tid = full ? S.bid[k - 1] : kEmptySlot;
      const float dist = staged_distances<P, CPL>(q, rows[cur], ix.xs, ix.nchunks, nc);
      uint64_t ck = kNoKey;
      uint32_t cv = kEmptySlot;
      if (lane < nc) {
        ck = make_key(0u, dist);
        cv = cids[cur][lane];
        if (full && !key_less(ck, cv, tkey, tid)) { ck = kNoKey; cv = kEmptySlot; }
      }
      int r0;
      cnt = merge_candidates<CAP, false>(S.bkey, S.bid, cnt, k, ck, cv, r0);
      __syncwarp();   // rows[cur] and cids[cur] are reused by round r + 2
    }
    uint64_t *pk = part_key + (qi * ntiles + t) * k;
    uint32_t *pi = part_id + (qi * ntiles + t) * k;
    for (int j = lane; j < k; j += 32) {
      pk[j] = j < cnt ? S.bkey[j] : kNoKey;
      pi[j] = j < cnt ? S.bid[j] : kEmptySlot;
    }
    __syncwarp();
  }
}

// (query, tile) work items of the scan route, compacted so that every scan
// warp gets a real tile: items[i] = (query << 20) | tile.
__global__ void scan_items_kernel(const DevIndex ix, const jag_filter *filters, const QueryPlan *plans,
                                  const int32_t *lists, int64_t cap, int64_t nq, int64_t tile, uint64_t *items,
                                  unsigned long long *nitems) {
  const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (qi >= nq) return;
  const QueryPlan pl = plans[qi];
  if (pl.route != kRouteSlice && pl.route != kRouteList) return;
  const int32_t *ids;
  int64_t m;
  routed_candidates(ix, filters, pl, qi, lists, cap, &ids, &m);
  const int64_t nt = (m + tile - 1) / tile;
  if (nt == 0) return;
  const unsigned long long base = atomicAdd(nitems, (unsigned long long)nt);
  for (int64_t t = 0; t < nt; ++t) items[base + t] = ((uint64_t)qi << 20) | (uint64_t)t;
}

template <int CAP>
__global__ void __launch_bounds__(kSearchWarps * 32)
merge_scan_kernel(const DevIndex ix, const jag_filter *filters, const QueryPlan *plans, const int32_t *lists,
                  int64_t cap, int64_t nq, int k, int64_t tile, int ntiles, const uint64_t *part_key,
                  const uint32_t *part_id, int32_t *out_ids, float *out_dist, int32_t *counters) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lcap = list_slots(k);
  const WarpSmem S = carve_warp_smem(smem + warp * warp_smem_bytes(lcap, 5), lcap, 5);
  const int64_t qi = (int64_t)blockIdx.x * kSearchWarps + warp;
  if (qi >= nq) return;
  const QueryPlan pl = plans[qi];
  if (pl.route != kRouteSlice && pl.route != kRouteList) return;
  const int32_t *ids;
  int64_t m;
  routed_candidates(ix, filters, pl, qi, lists, cap, &ids, &m);
  const int nt = (int)((m + tile - 1) / tile);
  int cnt = 0;
  for (int t = 0; t < nt; ++t) {
    for (int b = 0; b < k; b += 32) {
      uint64_t ck = kNoKey;
      uint32_t cv = kEmptySlot;
      if (b + lane < k) {
        ck = part_key[(qi * ntiles + t) * k + b + lane];
        cv = part_id[(qi * ntiles + t) * k + b + lane];
      }
      if (cnt == k && ck != kNoKey && !key_less(ck, cv, S.bkey[k - 1], S.bid[k - 1])) { ck = kNoKey; cv = kEmptySlot; }
      int r0;
      cnt = merge_candidates<CAP, false>(S.bkey, S.bid, cnt, k, ck, cv, r0);
    }
  }
  write_answers(S, cnt, qi, k, out_ids, out_dist);
  if (counters && lane == 0) {
    int32_t *c = counters + qi * 4;
    c[0] = 0; c[1] = 0; c[2] = (int32_t)m; c[3] = 1;
  }
}

// Brute force: every point of a tile is tested against the filter and the
// passing ones ranked exactly; partial lists are merged per query afterwards.
template <int CAP, int P, int CPL>
__global__ void __launch_bounds__(kSearchWarps * 32)
brute_tile_kernel(DevIndex ix, const float *queries, int d, const jag_filter *filters, const uint8_t *aux,
                  const QueryPlan *plans, int64_t nq, int k, int64_t tile, int ntiles, uint64_t *part_key,
                  uint32_t *part_id) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const WarpSmem S = carve_warp_smem(smem + warp * warp_smem_bytes(CAP, 5), CAP, 5);
  const int64_t qi = (int64_t)blockIdx.y * kSearchWarps + warp;
  if (qi >= nq) return;
  const int t = blockIdx.x;
  uint64_t *pk = part_key + (qi * ntiles + t) * k;
  uint32_t *pi = part_id + (qi * ntiles + t) * k;
  if (plans[qi].route != kRouteSkip + 1) {
    for (int j = lane; j < k; j += 32) { pk[j] = kNoKey; pi[j] = kEmptySlot; }
    return;
  }
  const jag_filter f = filters[qi];
  const uint8_t *tt = f.kind == JAG_F_BOOL ? aux + f.aux_off : nullptr;
  QChunks<CPL, JAG_VEC_F32> q;
  load_point<P, CPL>(queries + qi * d, d, q);
  const int64_t b0 = (int64_t)t * tile, b1 = min64(ix.n, b0 + tile);
  int cnt = 0;
  for (int64_t b = b0; b < b1; b += 32) {
    const int64_t u = b + lane;
    const bool pass = u < b1 && passes(ix, u, f.kind, f.payload, tt);
    const uint32_t pm = __ballot_sync(kFull, pass);
    if (!pm) continue;
    const int nc = __popc(pm);
    if (pass) S.cid[__popc(pm & lanemask_lt())] = (uint32_t)u;
    __syncwarp();
    const bool full = cnt == k;
    const uint64_t tkey = full ? S.bkey[k - 1] : kNoKey;
    const uint32_t tid = full ? S.bid[k - 1] : kEmptySlot;
    const float dist = candidate_distances<P, CPL, 4, JAG_VEC_F32, true>(ix, q, S.cid, nc);
    uint64_t ck = kNoKey;
    uint32_t cv = kEmptySlot;
    if (lane < nc) {
      ck = make_key(0u, dist);
      cv = S.cid[lane];
      if (full && !key_less(ck, cv, tkey, tid)) { ck = kNoKey; cv = kEmptySlot; }
    }
    int r0;
    cnt = merge_candidates<CAP, false>(S.bkey, S.bid, cnt, k, ck, cv, r0);
  }
  for (int j = lane; j < k; j += 32) {
    pk[j] = j < cnt ? S.bkey[j] : kNoKey;
    pi[j] = j < cnt ? S.bid[j] : kEmptySlot;
  }
}

template <int CAP>
__global__ void __launch_bounds__(kSearchWarps * 32)
merge_parts_kernel(const QueryPlan *plans, int64_t nq, int k, int ntiles, const uint64_t *part_key,
                   const uint32_t *part_id, int32_t *out_ids, float *out_dist, int32_t *counters) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const WarpSmem S = carve_warp_smem(smem + warp * warp_smem_bytes(CAP, 5), CAP, 5);
  const int64_t qi = (int64_t)blockIdx.x * kSearchWarps + warp;
  if (qi >= nq) return;
  if (plans[qi].route != kRouteSkip + 1) return;   // padded by the preparation kernel
  int cnt = 0;
  for (int t = 0; t < ntiles; ++t) {
    for (int b = 0; b < k; b += 32) {
      uint64_t ck = kNoKey;
      uint32_t cv = kEmptySlot;
      if (b + lane < k) {
        ck = part_key[(qi * ntiles + t) * k + b + lane];
        cv = part_id[(qi * ntiles + t) * k + b + lane];
      }
      if (cnt == k && ck != kNoKey && !key_less(ck, cv, S.bkey[k - 1], S.bid[k - 1])) { ck = kNoKey; cv = kEmptySlot; }
      int r0;
      cnt = merge_candidates<CAP, false>(S.bkey, S.bid, cnt, k, ck, cv, r0);
    }
  }
  write_answers(S, cnt, qi, k, out_ids, out_dist);
  if (counters && lane == 0) {
    int32_t *c = counters + qi * 4;
    c[0] = 0; c[1] = 0; c[2] = 0; c[3] = 2;
  }
}

// K5: fp32 re-rank for BF16 / FP8 storage.  The graph kernel leaves the ids
// of the leading rr passing entries of each final list (-1 padded); their
// canonical fp32 distances are computed from the fp32 rows and the best k,
// by (distance, id), are the answers.
template <int CAP, int P, int CPL>
__global__ void __launch_bounds__(kSearchWarps * 32)
rerank_kernel(DevIndex ix, const float *queries, int d, const QueryPlan *plans, int64_t nq, int k, int rr,
              const int32_t *rr_ids, int32_t *out_ids, float *out_dist) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lcap = list_slots(k);
  const WarpSmem S = carve_warp_smem(smem + warp * warp_smem_bytes(lcap, 5), lcap, 5);
  const int64_t qi = (int64_t)blockIdx.x * kSearchWarps + warp;
  if (qi >= nq) return;
  if (plans[qi].route != kRouteGraph) return;
  QChunks<CPL, JAG_VEC_F32> q;
  load_point<P, CPL>(queries + qi * d, d, q);
  int cnt = 0;
  for (int b = 0; b < rr; b += 32) {
    const int32_t id = b + lane < rr ? rr_ids[qi * rr + b + lane] : -1;
    const int nc = __popc(__ballot_sync(kFull, id >= 0));   // valid ids form a prefix
    if (nc == 0) break;
    if (lane < nc) S.cid[lane] = (uint32_t)id;
    __syncwarp();
    const bool full = cnt == k;
    const uint64_t tkey = full ? S.bkey[k - 1] : kNoKey;
    const uint32_t tid = full ? S.bid[k - 1] : kEmptySlot;
    const float dist = candidate_distances<P, CPL, 4, JAG_VEC_F32, true>(ix, q, S.cid, nc);
    uint64_t ck = kNoKey;
    uint32_t cv = kEmptySlot;
    if (lane < nc) {
      ck = make_key(0u, dist);
      cv = S.cid[lane];
      if (full && !key_less(ck, cv, tkey, tid)) { ck = kNoKey; cv = kEmptySlot; }
    }
    int r0;
    cnt = merge_candidates<CAP, false>(S.bkey, S.bid, cnt, k, ck, cv, r0);
  }
  write_answers(S, cnt, qi, k, out_ids, out_dist);
}

// Edge attribute tables: the attribute of every edge's target, [n][R].
__global__ void edge_attr_kernel(DevIndex ix, int32_t *ea_i32, float *ea_f32, uint64_t *ea_mask) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ix.n * ix.R) return;
  const int32_t u = ix.graph[e];
  const int64_t v = u >= 0 ? u : 0;
  if (ea_i32) ea_i32[e] = u >= 0 ? ix.a_i32[v] : 0;
  if (ea_f32) ea_f32[e] = u >= 0 ? ix.a_f32[v] : 0.f;
  if (ea_mask) ea_mask[e] = u >= 0 ? ix.a_mask[v] : 0ull;
}

cudaError_t build_edge_attrs(const DevIndex &ix, int32_t *ea_i32, float *ea_f32, uint64_t *ea_mask,
                             cudaStream_t stream) {
  const int64_t ne = ix.n * ix.R;
  edge_attr_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, stream>>>(ix, ea_i32, ea_f32, ea_mask);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

size_t tc_slots(int64_t nq) {
  size_t h = 64;
  while (h < (size_t)std::max<int64_t>(nq, 1) * 2) h <<= 1;
  return h;
}

int list_capacity(int ls) {
  if (ls <= 64) return 64;
  if (ls <= 128) return 128;
  if (ls <= 256) return 256;
  if (ls <= 512) return 512;
  return 0;
}

bool row_mapping(int nchunks, int *P, int *CPL) {
  if (nchunks <= 8) { *P = 8; *CPL = 1; }
  else if (nchunks <= 16) { *P = 16; *CPL = 1; }
  else if (nchunks <= 32) { *P = 32; *CPL = 1; }
  else if (nchunks <= 64) { *P = 32; *CPL = 2; }
  else if (nchunks <= 128) { *P = 32; *CPL = 4; }
  else if (nchunks <= 256) { *P = 32; *CPL = 8; }
  else return false;
  return true;
}

static size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

void scan_tiling(int64_t n, int scan_all, int64_t s0, int64_t cap, int32_t *ntiles, int64_t *tile) {
  if (scan_all) {
    *tile = 65536;
    *ntiles = (int32_t)std::max<int64_t>(1, (n + *tile - 1) / *tile);
  } else {
    *tile = 1024;
    const int64_t most = std::max<int64_t>(std::max<int64_t>(s0, cap), 1);
    *ntiles = (int32_t)std::max<int64_t>(1, (most + *tile - 1) / *tile);
  }
}

// Rows per round of the staged scan: two rounds of rows (double buffer)
// take 8 KB of shared memory per warp, so that a scan CTA fits beside the
// graph kernel as soon as a few of its warps have left an SM -- the scan then
// runs inside the graph search's last wave.  (16 KB per warp: 3.32 M against
// 3.59 M QPS on the 1M label batch; 4 KB: within 1 %.)
int scan_rows_per_round(int64_t xs) {
  const int64_t r = 4096 / (xs * 4);
  return (int)std::max<int64_t>(1, std::min<int64_t>(32, r));
}

SearchScratch search_scratch_layout(const DevIndex &ix, int64_t nq, int64_t aux_bytes, int64_t cap, int32_t k,
                                    int32_t ls, int scan_all, int64_t s0, int tc) {
  SearchScratch s{};
  const size_t q1 = (size_t)std::max<int64_t>(nq, 1);
  scan_tiling(ix.n, scan_all, s0, cap, &s.ntiles, &s.tile);
  const bool lists = !scan_all && s0 > 0 && ix.a_mask != nullptr;
  s.tc = (!scan_all && s0 > 0 && tc) ? 1 : 0;
  // a slice of at most cap rows touches at most cap / 128 + 2 tiles; the
  // tile lists are indexed with int32, else the fp32 scan kernels run
  const size_t tc_entries = q1 * ((size_t)cap / 128 + 2);
  if (tc_entries + q1 >= ((size_t)1 << 31)) s.tc = 0;
  const bool parts_needed = scan_all || (s0 > 0 && !s.tc);
  size_t off = 0;
  s.plans = off; off += align256(sizeof(QueryPlan) * q1);
  s.lut = off; off += align256((size_t)std::max<int64_t>(aux_bytes, 1) * 8);
  s.lists = off; off += lists ? align256(q1 * (size_t)cap * 4) : 256;
  s.lslots = lists ? tc_slots(nq) : 1;
  s.lhkey = off; off += align256(s.lslots * 8);
  s.lhlead = off; off += align256(s.lslots * 4);
  s.lslot = off; off += align256((lists ? q1 : 1) * 4);
  s.leaders = off; off += align256((lists ? q1 : 1) * 4);
  s.list_counts = off; off += align256(q1 * 4);
  s.work = off; off += 256;
  s.status = off; off += 256;
  const size_t parts = parts_needed ? q1 * (size_t)s.ntiles * (size_t)k : 1;
  s.part_key = off; off += align256(parts * 8);
  s.part_id = off; off += align256(parts * 4);
  s.scan_items = off; off += (!scan_all && s0 > 0 && !s.tc) ? align256(q1 * (size_t)s.ntiles * 8) : 256;
  s.rr = ix.fmt != JAG_VEC_F32 ? rerank_count(k, ls) : 0;
  s.rr_ids = off; off += align256(q1 * (size_t)std::max(s.rr, 1) * 4);
  if (s.tc) {
    const size_t T0 = (size_t)tc_column_tiles(ix.n), U = 2 * T0 + q1;
    // work items: column tiles at most 2 T0 + (entries) / 64; leaders' lists
    // at most (cap / 128 + 1) per listed query and one more per leader
    const size_t items = 2 * T0 + tc_entries / kTcItemQueries + 2 * q1 * ((size_t)cap / 128 + 1);
    s.approx = off; off += align256(q1 * (size_t)cap * 4);
    s.qnorm = off; off += align256(q1 * 4);
    s.tcnt = off; off += align256(U * 4);
    s.tfill = off; off += align256(U * 4);
    s.toff = off; off += align256(U * 4);
    s.tq = off; off += align256((tc_entries + q1) * 4);
    s.item_unit = off; off += align256(items * 4);
    s.ioff = off; off += align256(U * 8);
    s.bsum = off; off += align256(((U + 1023) / 1024) * 16);
  }
  s.total = off;
  return s;
}

void bind_scratch(SearchLaunch &L, const SearchScratch &s, uint8_t *base) {
  L.plans = reinterpret_cast<QueryPlan *>(base + s.plans);
  L.lut = base + s.lut;
  L.lists = reinterpret_cast<int32_t *>(base + s.lists);
  L.lgroup.hkey = reinterpret_cast<uint64_t *>(base + s.lhkey);
  L.lgroup.hlead = reinterpret_cast<int32_t *>(base + s.lhlead);
  L.lgroup.lslot = reinterpret_cast<int32_t *>(base + s.lslot);
  L.lgroup.leaders = reinterpret_cast<int32_t *>(base + s.leaders);
  L.lgroup.slots = s.lslots;
  L.list_counts = reinterpret_cast<int32_t *>(base + s.list_counts);
  L.work = reinterpret_cast<unsigned long long *>(base + s.work);
  L.status = reinterpret_cast<uint32_t *>(base + s.status);
  L.part_key = reinterpret_cast<uint64_t *>(base + s.part_key);
  L.part_id = reinterpret_cast<uint32_t *>(base + s.part_id);
  L.scan_items = reinterpret_cast<uint64_t *>(base + s.scan_items);
  L.ntiles = s.ntiles;
  L.tile = s.tile;
  L.rr = s.rr;
  L.rr_ids = reinterpret_cast<int32_t *>(base + s.rr_ids);
  L.tc = TcScratch{};
  if (s.tc) {
    L.tc.approx = reinterpret_cast<float *>(base + s.approx);
    L.tc.qnorm = reinterpret_cast<float *>(base + s.qnorm);
    L.tc.item_unit = reinterpret_cast<int32_t *>(base + s.item_unit);
    L.tc.tcnt = reinterpret_cast<int32_t *>(base + s.tcnt);
    L.tc.tfill = reinterpret_cast<int32_t *>(base + s.tfill);
    L.tc.toff = reinterpret_cast<int32_t *>(base + s.toff);
    L.tc.tq = reinterpret_cast<int32_t *>(base + s.tq);
    L.tc.ioff = reinterpret_cast<int64_t *>(base + s.ioff);
    L.tc.bsum = reinterpret_cast<int64_t *>(base + s.bsum);
  }
}

template <int CAP, int P, int CPL>
static cudaError_t launch_scan(const SearchLaunch &L) {
  const int64_t want = std::max<int64_t>((L.nq + kSearchWarps - 1) / kSearchWarps, 1);
  // the exact scan for the routed queries (k <= ls <= CAP)
  const int rpr = scan_rows_per_round(L.ix.xs);
  const size_t ssm = (size_t)kScanWarps * (warp_smem_bytes(list_slots(L.k), 5) + 32 * 4 + 2 * (size_t)rpr * L.ix.xs * 4);
  auto sk = scan_tile_kernel<CAP, P, CPL>;
  // work items in their own scratch region; counters in work[2..3]
  uint64_t *items = L.scan_items;
  scan_items_kernel<<<(unsigned)((L.nq + 255) / 256), 256, 0, L.stream>>>(L.ix, L.filters, L.plans, L.lists, L.cap,
                                                                          L.nq, L.tile, items, L.work + 3);
  const int sbps = blocks_per_sm(sk, ssm, kScanWarps);
  if (sbps == 0) return cudaErrorInvalidConfiguration;
  const int64_t sgrid = std::min<int64_t>((int64_t)sbps * num_sms(),
                                          std::max<int64_t>(1, (L.nq * L.ntiles + kScanWarps - 1) / kScanWarps));
  sk<<<(unsigned)sgrid, kScanWarps * 32, ssm, L.stream>>>(L.ix, L.queries, L.d, L.filters, L.plans, L.lists, L.cap,
                                                           L.k, L.tile, L.ntiles, rpr, items, L.work + 3, L.work + 2,
                                                           L.part_key, L.part_id);
  const size_t msm = (size_t)kSearchWarps * warp_smem_bytes(list_slots(L.k), 5);
  auto mk = merge_scan_kernel<CAP>;
  if (blocks_per_sm(mk, msm) == 0) return cudaErrorInvalidConfiguration;
  mk<<<(unsigned)want, kSearchWarps * 32, msm, L.stream>>>(L.ix, L.filters, L.plans, L.lists, L.cap, L.nq, L.k,
                                                          L.tile, L.ntiles, L.part_key, L.part_id, L.out_ids,
                                                          L.out_dist, L.counters);
  return cudaGetLastError();
}

template <int CAP, int P, int CPL>
static cudaError_t launch_rerank(const SearchLaunch &L) {
  const int64_t want = std::max<int64_t>((L.nq + kSearchWarps - 1) / kSearchWarps, 1);
  const size_t sm = (size_t)kSearchWarps * warp_smem_bytes(list_slots(L.k), 5);
  auto rk = rerank_kernel<CAP, P, CPL>;
  if (blocks_per_sm(rk, sm) == 0) return cudaErrorInvalidConfiguration;
  rk<<<(unsigned)want, kSearchWarps * 32, sm, L.stream>>>(L.ix, L.queries, L.d, L.plans, L.nq, L.k, L.rr, L.rr_ids,
                                                         L.out_ids, L.out_dist);
  return cudaGetLastError();
}

template <int CAP, int P, int CPL>
static cudaError_t launch_brute(const SearchLaunch &L) {
  const size_t smem = (size_t)kSearchWarps * warp_smem_bytes(CAP, 5);
  auto kern = brute_tile_kernel<CAP, P, CPL>;
  if (blocks_per_sm(kern, smem) == 0) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)L.ntiles, (unsigned)((L.nq + kSearchWarps - 1) / kSearchWarps));
  kern<<<grid, kSearchWarps * 32, smem, L.stream>>>(L.ix, L.queries, L.d, L.filters, L.aux, L.plans, L.nq, L.k,
                                                     L.tile, L.ntiles, L.part_key, L.part_id);
  auto mk = merge_parts_kernel<CAP>;
  if (blocks_per_sm(mk, smem) == 0) return cudaErrorInvalidConfiguration;
  mk<<<(unsigned)((L.nq + kSearchWarps - 1) / kSearchWarps), kSearchWarps * 32, smem, L.stream>>>(
      L.plans, L.nq, L.k, L.ntiles, L.part_key, L.part_id, L.out_ids, L.out_dist, L.counters);
  return cudaGetLastError();
}

enum Job { kJobScan, kJobBrute, kJobRerank };

template <int CAP>
static cudaError_t dispatch_rows(const SearchLaunch &L, int P, int CPL, Job job) {
#define JAG_CASE(PP, CC)                                                    \
  if (P == PP && CPL == CC) {                                               \
    if (job == kJobBrute) return launch_brute<CAP, PP, CC>(L);              \
    if (job == kJobRerank) return launch_rerank<CAP, PP, CC>(L);            \
    return launch_scan<CAP, PP, CC>(L);                                     \
  }
  JAG_CASE(8, 1)
  JAG_CASE(16, 1)
  JAG_CASE(32, 1)
  JAG_CASE(32, 2)
  JAG_CASE(32, 4)
  JAG_CASE(32, 8)
#undef JAG_CASE
  return cudaErrorInvalidValue;
}

static cudaError_t dispatch_job(const SearchLaunch &L, int P, int CPL, Job job, int cap_of) {
  switch (list_capacity(cap_of)) {
    case 64: return dispatch_rows<64>(L, P, CPL, job);
    case 128: return dispatch_rows<128>(L, P, CPL, job);
    case 256: return dispatch_rows<256>(L, P, CPL, job);
    default: return cudaErrorInvalidValue;
  }
}

// Per-device stream on which the exact scan runs beside the graph search.
static cudaStream_t side_stream() {
  static std::mutex mu;
  static cudaStream_t streams[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> g(mu);
  if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess)
    streams[dev] = nullptr;
  return streams[dev];
}

cudaError_t run_search(const SearchLaunch &L) {
  if (L.nq == 0) return cudaSuccess;
  int P, CPL;
  if (!row_mapping(L.ix.nchunks, &P, &CPL)) return cudaErrorInvalidValue;
  cudaError_t e;
  if ((e = cudaMemsetAsync(L.work, 0, 256, L.stream)) != cudaSuccess) return e;
  {
    int64_t blocks = std::min<int64_t>((L.nq + kPrepWarps - 1) / kPrepWarps, (int64_t)num_sms() * 16);
    prep_kernel<<<(unsigned)blocks, kPrepWarps * 32, 0, L.stream>>>(
        L.ix, L.filters, L.aux, L.aux_bytes, L.nq, L.s0, L.cap, L.scan_all, L.has_policy, L.plans, L.lut,
        L.list_counts, L.k,
        L.out_ids, L.out_dist, L.counters, L.status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (L.scan_all) return dispatch_job(L, P, CPL, kJobBrute, L.k);
  if (L.s0 > 0 && L.ix.a_mask) {
    // identical list-routed filters share one gathered list (their leader's)
    const unsigned qb = (unsigned)((L.nq + 255) / 256);
    if ((e = cudaMemsetAsync(L.lgroup.hkey, 0xFF, L.lgroup.slots * 8, L.stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(L.lgroup.hlead, 0x7F, L.lgroup.slots * 4, L.stream)) != cudaSuccess) return e;
    list_group_kernel<<<qb, 256, 0, L.stream>>>(L.plans, L.filters, L.aux, L.nq, L.lgroup.hkey, L.lgroup.hlead,
                                                (uint32_t)(L.lgroup.slots - 1), L.lgroup.lslot);
    list_leader_kernel<<<qb, 256, 0, L.stream>>>(L.plans, L.filters, L.nq, L.lgroup.hlead, L.lgroup.lslot,
                                                 L.lgroup.leaders, L.work + 8);
    gather_postings_kernel<<<dim3((unsigned)L.nq, kPostParts), kPostWarps * 32, 0, L.stream>>>(
        L.ix, L.filters, L.lgroup.leaders, L.work + 8, L.cap, L.lists, L.list_counts);
    clamp_counts_kernel<<<(unsigned)((L.nq + 255) / 256), 256, 0, L.stream>>>(L.lgroup.leaders, L.work + 8, L.cap,
                                                                           L.list_counts);
    // the other leaders sit at the back of the array, in reverse order: the
    // mask pass reads them as leaders[nq - 1 - i]
    dim3 grid((unsigned)((L.ix.n + kGatherTile - 1) / kGatherTile), (unsigned)((L.nq + kGatherQPB - 1) / kGatherQPB));
    gather_list_kernel<<<grid, 256, 0, L.stream>>>(L.ix, L.filters, L.aux, L.lgroup.leaders, L.nq, L.work + 9,
                                                   L.cap, L.lists, L.list_counts);
    finalize_routes_kernel<<<(unsigned)((L.nq + 255) / 256), 256, 0, L.stream>>>(L.plans, L.list_counts, L.nq,
                                                                                 L.cap);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // The exact scan of the routed queries and the graph search of the others
  // touch disjoint queries.  The graph search is enqueued first, so that its
  // persistent CTAs take the SMs; the scan follows on a side stream and fills
  // the SMs that the graph search's last wave leaves idle; the two join
  // before the call's work ends.
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  if (L.s0 > 0 && L.fork_scan) {
    side = side_stream();
    if (!side || cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming) != cudaSuccess) {
      side = nullptr;
    } else if (cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming) != cudaSuccess) {
      cudaEventDestroy(ev_fork);
      side = nullptr;
    } else if ((e = cudaEventRecord(ev_fork, L.stream)) != cudaSuccess) {
      cudaEventDestroy(ev_fork);
      cudaEventDestroy(ev_join);
      return e;
    }
  }
  // graph search in the stored format, then the fp32 re-rank when the rows
  // are BF16 / FP8
  switch (L.ix.fmt) {
    case JAG_VEC_F32: e = launch_graph_fmt<JAG_VEC_F32>(L); break;
    case JAG_VEC_BF16: e = launch_graph_fmt<JAG_VEC_BF16>(L); break;
    case JAG_VEC_FP8: e = launch_graph_fmt<JAG_VEC_FP8>(L); break;
    default: e = cudaErrorInvalidValue;
  }
  if (e == cudaSuccess && L.ix.fmt != JAG_VEC_F32) e = dispatch_job(L, P, CPL, kJobRerank, L.k);
  if (side) {
    SearchLaunch S = L;
    S.stream = side;
    S.ev_begin = S.ev_end = nullptr;
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev_fork, 0);
    if (e == cudaSuccess) e = L.tc.approx ? launch_scan_tc(S) : dispatch_job(S, P, CPL, kJobScan, L.k);
    if (e == cudaSuccess) e = cudaEventRecord(ev_join, side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(L.stream, ev_join, 0);
    cudaEventDestroy(ev_fork);
    cudaEventDestroy(ev_join);
    return e;
  }
  if (e != cudaSuccess) return e;
  if (L.s0 > 0) return L.tc.approx ? launch_scan_tc(L) : dispatch_job(L, P, CPL, kJobScan, L.k);
  return cudaSuccess;
}

}  // namespace jag
