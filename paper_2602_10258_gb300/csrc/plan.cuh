// Per-query preparation shared by the batched search and the serve loop:
// filter validation, the boolean filter-distance table and the routing
// decision (graph search or exact scan).
#pragma once

#include "jag_internal.cuh"

namespace jag {

__device__ __forceinline__ int64_t lower_bound_i32(const int32_t *v, int64_t n, int32_t x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) { int64_t m = (lo + hi) >> 1; if (v[m] < x) lo = m + 1; else hi = m; }
  return lo;
}
__device__ __forceinline__ int64_t upper_bound_i32(const int32_t *v, int64_t n, int32_t x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) { int64_t m = (lo + hi) >> 1; if (v[m] <= x) lo = m + 1; else hi = m; }
  return lo;
}
__device__ __forceinline__ int64_t lower_bound_f32(const float *v, int64_t n, float x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) { int64_t m = (lo + hi) >> 1; if (v[m] < x) lo = m + 1; else hi = m; }
  return lo;
}
__device__ __forceinline__ int64_t upper_bound_f32(const float *v, int64_t n, float x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) { int64_t m = (lo + hi) >> 1; if (v[m] <= x) lo = m + 1; else hi = m; }
  return lo;
}

// Boolean distance table of one filter (Sec. 3.1, boolean example):
// lut[s] = least Hamming distance from assignment s of the m involved bits to
// an assignment where the truth table is 1 (255 if there is none).  Computed
// one dimension at a time: the Hamming metric is a sum over bits, so relaxing
// each pair (s, s ^ 2^j) once per bit j gives the exact distances.
__device__ inline void build_bool_lut(const uint8_t *tt, int m, uint8_t *lut) {
  const int lane = threadIdx.x & 31;
  const uint32_t S = 1u << m;
  for (uint32_t s = lane; s < S; s += 32) lut[s] = ((tt[s >> 3] >> (s & 7)) & 1) ? 0 : 255;
  __syncwarp();
  for (int j = 0; j < m; ++j) {
    const uint32_t low = (1u << j) - 1;
    for (uint32_t i = lane; i < (S >> 1); i += 32) {
      const uint32_t s = ((i & ~low) << 1) | (i & low);
      const uint32_t t = s | (1u << j);
      const int a = lut[s], b = lut[t];
      lut[s] = (uint8_t)min(a, b + 1);
      lut[t] = (uint8_t)min(b, a + 1);
    }
    __syncwarp();
  }
}

// Plan of one query by the calling warp (every lane returns the same):
// validate the filter (false: bad filter, route kRouteSkip); build the
// boolean table at lut_base + 8 * aux_off; label/range filters count their
// passing set exactly (binary search in the sorted column), subset/boolean
// filters estimate it on the fixed sample of S = min(4096, n) points with
// ids floor(j n / S).  With s0 > 0 a query whose count (estimate) is below s0
// goes to the exact scan (a slice of a sorted column, or, for subset/boolean
// filters, a list gathered by a pass over the mask column).  need_est: fill
// pl.est even when s0 = 0 (the learned policy's feature).
__device__ inline bool plan_query(const DevIndex &ix, const jag_filter &f, const uint8_t *aux, int64_t aux_bytes,
                                  int64_t s0, int64_t cap, int scan_all, int need_est, uint8_t *lut_base,
                                  QueryPlan &pl) {
  const int lane = threadIdx.x & 31;
  pl.route = kRouteGraph; pl.lut_off = -1; pl.begin = 0; pl.end = 0; pl.count = 0; pl.est = 0;
  bool ok;
  int m = 0;
  switch (f.kind) {
    case JAG_F_NONE: ok = true; break;
    case JAG_F_LABEL: case JAG_F_RANGE_I32: ok = ix.a_i32 != nullptr; break;
    case JAG_F_RANGE_F32: ok = ix.a_f32 != nullptr; break;
    case JAG_F_SUBSET: ok = ix.a_mask != nullptr; break;
    case JAG_F_BOOL: {
      m = __popcll(f.payload);
      ok = ix.a_mask != nullptr && aux != nullptr && m <= 16 && f.aux_off >= 0;
      if (ok) {
        const int64_t tbytes = ((int64_t)1 << m) / 8 > 0 ? ((int64_t)1 << m) / 8 : 1;
        ok = (int64_t)f.aux_off + tbytes <= aux_bytes;
      }
      break;
    }
    default: ok = false;
  }
  if (!ok) {
    pl.route = kRouteSkip;
    return false;
  }
  const uint8_t *tt = nullptr;
  if (f.kind == JAG_F_BOOL) {
    tt = aux + f.aux_off;
    pl.lut_off = f.aux_off * 8;
    build_bool_lut(tt, m, lut_base + pl.lut_off);
  }
  if (scan_all) {
    pl.route = kRouteSkip + 1;   // brute-force scan
  } else if (s0 > 0 || need_est) {
    if (f.kind == JAG_F_LABEL || f.kind == JAG_F_RANGE_I32 || f.kind == JAG_F_RANGE_F32) {
      int64_t b = 0, e = 0;
      if (lane == 0) {
        if (f.kind == JAG_F_LABEL) {
          b = lower_bound_i32(ix.si32_val, ix.n, lo32(f.payload));
          e = upper_bound_i32(ix.si32_val, ix.n, lo32(f.payload));
        } else if (f.kind == JAG_F_RANGE_I32) {
          const int32_t lo = lo32(f.payload), hi = hi32(f.payload);
          if (lo <= hi) { b = lower_bound_i32(ix.si32_val, ix.n, lo); e = upper_bound_i32(ix.si32_val, ix.n, hi); }
        } else {
          const float lo = u2f((uint32_t)lo32(f.payload)), hi = u2f((uint32_t)hi32(f.payload));
          if (lo <= hi) { b = lower_bound_f32(ix.sf32_val, ix.n, lo); e = upper_bound_f32(ix.sf32_val, ix.n, hi); }
        }
      }
      b = __shfl_sync(kFull, b, 0);
      e = __shfl_sync(kFull, e, 0);
      pl.begin = b; pl.end = e;
      pl.est = (int32_t)min64(e - b, 0x7FFFFFFF);
      if (s0 > 0 && e - b < s0 && e - b <= cap) pl.route = kRouteSlice;
    } else if (f.kind == JAG_F_SUBSET || f.kind == JAG_F_BOOL) {
      const int64_t S = ix.n < 4096 ? ix.n : 4096;
      int hits = 0;
      for (int64_t j = lane; j < S; j += 32) hits += passes(ix, j * ix.n / S, f.kind, f.payload, tt) ? 1 : 0;
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) hits += __shfl_xor_sync(kFull, hits, o);
      pl.est = hits;
      if (s0 > 0 && (int64_t)hits * ix.n < s0 * S) pl.route = kRouteList;
    }
  }
  return true;
}

}  // namespace jag
