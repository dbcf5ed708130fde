// Internal device-side definitions of the JAG search library (sm_103a).
//
// Data layout in device memory (one index):
//   x        fp32 rows, stride xs floats (d rounded up to a multiple of 4,
//            zero padded) so that every row starts on a 16-byte boundary and
//            is read as 16-byte chunks;
//   graph    int32 [n][R] out-lists, -1 padded (one 128-byte row at R = 32);
//   a_i32 / a_f32 / a_mask   per-point attribute columns (structure of arrays);
//   s*_val / s*_id           the int32 / float32 column sorted by (value, id):
//            label and range filters read their passing set as one slice.
//
// Ordered keys.  Candidates are compared lexicographically by
// (first component, squared distance, id) (Sec. 3.2, "Unified comparison
// rule"; the id is a final tie-break).  The first component is dist_F for a
// query and the capped dist_A for the build, kept as a 32-bit unsigned: an
// integer distance, or the bit pattern of a non-negative float, which orders
// like the value.  (first, distance bits) form one 64-bit key.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "jag.h"

namespace jag {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr uint32_t kExpanded = 0x80000000u;   // beam id flag: vertex expanded
constexpr uint32_t kEmptySlot = 0xFFFFFFFFu;  // visited-set empty slot
constexpr uint64_t kNoKey = ~0ull;

enum Route : int32_t { kRouteGraph = 0, kRouteSlice = 1, kRouteList = 2, kRouteSkip = 3 };

struct DevIndex {
  int64_t n;
  int32_t d;
  int32_t nchunks;      // 16-byte chunks per stored fp32 row = xs / 4
  int64_t xs;           // row stride in floats
  const float *x;
  const int32_t *graph;
  int32_t R;
  int32_t entry;
  int32_t dist_a;
  int32_t pad0;
  const int32_t *a_i32;
  const float *a_f32;
  const uint64_t *a_mask;
  const int32_t *si32_val;
  const int32_t *si32_id;
  const float *sf32_val;
  const int32_t *sf32_id;
  // attribute of each edge's target, laid out like the graph ([n][R]), so a
  // hop reads neighbour ids and their attributes in one wave of loads
  const int32_t *ea_i32;
  const float *ea_f32;
  const uint64_t *ea_mask;
  // rows in the storage format the search reads (BF16 / FP8); fp32 rows (x)
  // stay for the build, the exact scan and the fp32 re-rank
  const uint8_t *xq;
  const float *qscale;      // per-row scale of FP8 rows
  int32_t fmt;              // jag_vec_format
  int32_t qbytes;           // bytes per stored row (multiple of 16)
  int32_t qchunks;          // 16-byte chunks per stored row
  int32_t pad1;
  // |x|^2 of every fp32 row (any summation order) and the largest of them:
  // the exact scan's approximate distances and their error bound
  const float *xnorm;
  float xnorm_max;
  int32_t pad2;
  // posting lists of the mask column: the ids of the points with bit j set
  // are bit_ids[bit_off[j] .. bit_off[j + 1]), in increasing order
  const int64_t *bit_off;
  const int32_t *bit_ids;
};

// Elements of one 16-byte chunk of a stored row, per format.
template <int FMT>
struct RowFmt {
  static constexpr int E = FMT == JAG_VEC_F32 ? 4 : (FMT == JAG_VEC_BF16 ? 8 : 16);
  static constexpr int Q4 = E / 4;   // float4 registers of query per chunk
};

// Per-query plan written by the preparation kernel.
struct QueryPlan {
  int32_t route;        // Route
  int32_t lut_off;      // byte offset of the boolean distance table, -1 if none
  int64_t begin, end;   // passing slice of a sorted column (kRouteSlice)
  int32_t count;        // passing points gathered for kRouteList
  int32_t est;          // estimated / exact passing count used by the router
};

__device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint32_t f2u(float f) { return __float_as_uint(f); }
__device__ __forceinline__ float u2f(uint32_t u) { return __uint_as_float(u); }

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ int32_t lo32(uint64_t p) { return (int32_t)(uint32_t)(p & 0xFFFFFFFFu); }
__device__ __forceinline__ int32_t hi32(uint64_t p) { return (int32_t)(uint32_t)(p >> 32); }

// Compress the bits of a selected by vars into the low bits, lowest first.
__device__ __forceinline__ uint32_t compress_bits(uint64_t a, uint64_t vars) {
  uint32_t s = 0;
  int j = 0;
  while (vars) {
    int pos = __ffsll((long long)vars) - 1;
    s |= (uint32_t)((a >> pos) & 1ull) << j;
    ++j;
    vars &= vars - 1;
  }
  return s;
}

// g(a, f) of Sec. 2 for point u.  tt: the boolean filter's truth table.
__device__ __forceinline__ bool passes(const DevIndex &ix, int64_t u, int32_t kind, uint64_t pay,
                                       const uint8_t *tt) {
  switch (kind) {
    case JAG_F_NONE: return true;
    case JAG_F_LABEL: return ix.a_i32[u] == lo32(pay);
    case JAG_F_RANGE_I32: {
      int32_t a = ix.a_i32[u];
      return lo32(pay) <= a && a <= hi32(pay);
    }
    case JAG_F_RANGE_F32: {
      float a = ix.a_f32[u];
      return u2f((uint32_t)lo32(pay)) <= a && a <= u2f((uint32_t)hi32(pay));
    }
    case JAG_F_SUBSET: return (pay & ix.a_mask[u]) == pay;
    case JAG_F_BOOL: {
      uint32_t s = compress_bits(ix.a_mask[u], pay);
      return (tt[s >> 3] >> (s & 7)) & 1;
    }
    default: return false;
  }
}

// dist_F(a, f) in ordered 32-bit form (Sec. 3.1, "Examples") from the raw
// attribute word a (int32 or float32 bit pattern in the low 32 bits, or the
// 64-bit mask).  lut: the per-query boolean table (least flips per
// assignment of the involved bits).
__device__ __forceinline__ uint32_t filter_distance_raw(int32_t kind, uint64_t pay, const uint8_t *lut,
                                                        uint64_t raw) {
  // an if-chain on the (warp-uniform) kind: cheaper than a jump table
  if (kind == JAG_F_LABEL) return (int32_t)(uint32_t)raw != lo32(pay) ? 1u : 0u;
  if (kind == JAG_F_RANGE_I32) {
    const int64_t a = (int32_t)(uint32_t)raw, lo = lo32(pay), hi = hi32(pay);
    return a < lo ? (uint32_t)(lo - a) : (a > hi ? (uint32_t)(a - hi) : 0u);
  }
  if (kind == JAG_F_RANGE_F32) {
    const float a = u2f((uint32_t)raw);
    const float lo = u2f((uint32_t)lo32(pay)), hi = u2f((uint32_t)hi32(pay));
    if (a < lo) return f2u(__fsub_rn(lo, a));
    if (a > hi) return f2u(__fsub_rn(a, hi));
    if (lo <= a && a <= hi) return 0u;
    return 0x7F800000u;  // NaN bound: never satisfied
  }
  if (kind == JAG_F_SUBSET) return (uint32_t)__popcll(pay & ~raw);
  if (kind == JAG_F_BOOL) return lut[compress_bits(raw, pay)];
  if (kind == JAG_F_NONE) return 0u;
  return 0x7F800000u;
}

// The raw attribute word a filter kind reads, for point u.
__device__ __forceinline__ uint64_t point_attr(const DevIndex &ix, int64_t u, int32_t kind) {
  switch (kind) {
    case JAG_F_LABEL: case JAG_F_RANGE_I32: return (uint32_t)ix.a_i32[u];
    case JAG_F_RANGE_F32: return f2u(ix.a_f32[u]);
    case JAG_F_SUBSET: case JAG_F_BOOL: return ix.a_mask[u];
    default: return 0;
  }
}

__device__ __forceinline__ uint32_t ld_word(const void *p) {
  uint32_t v;
  asm volatile("ld.global.nc.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ uint64_t ld_dword(const void *p) {
  uint64_t v;
  asm volatile("ld.global.nc.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}

// Ask L2 for the 128-byte lines of [p, p + bytes) (no register is written;
// a later load of the bytes finds them in L2 or already on their way).
__device__ __forceinline__ void prefetch_l2(const void *p, int bytes) {
  const uint64_t a1 = ((uint64_t)p + (uint64_t)bytes - 1) & ~127ull;
  for (uint64_t a = (uint64_t)p & ~127ull; a <= a1; a += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

// The same word for the target of edge e (= p * R + r) from the edge table;
// issued where it is written, next to the load of the neighbour id.
__device__ __forceinline__ uint64_t edge_attr(const DevIndex &ix, int64_t e, int32_t kind) {
  switch (kind) {
    case JAG_F_LABEL: case JAG_F_RANGE_I32: return ld_word(ix.ea_i32 + e);
    case JAG_F_RANGE_F32: return ld_word(ix.ea_f32 + e);
    case JAG_F_SUBSET: case JAG_F_BOOL: return ld_dword(ix.ea_mask + e);
    default: return 0;
  }
}

__device__ __forceinline__ uint32_t filter_distance(const DevIndex &ix, int64_t u, int32_t kind,
                                                    uint64_t pay, const uint8_t *lut) {
  return filter_distance_raw(kind, pay, lut, point_attr(ix, u, kind));
}

// dist_A(a_i, a_j) in ordered form (Sec. 3.1) for the build's attribute.
__device__ __forceinline__ uint32_t attribute_distance(const DevIndex &ix, int64_t i, int64_t j) {
  switch (ix.dist_a) {
    case JAG_F_LABEL: return ix.a_i32[i] != ix.a_i32[j] ? 1u : 0u;
    case JAG_F_RANGE_I32: {
      int64_t t = (int64_t)ix.a_i32[i] - (int64_t)ix.a_i32[j];
      return (uint32_t)(t < 0 ? -t : t);
    }
    case JAG_F_RANGE_F32: return f2u(fabsf(__fsub_rn(ix.a_f32[i], ix.a_f32[j])));
    default: return (uint32_t)__popcll(ix.a_mask[i] ^ ix.a_mask[j]);
  }
}

// dist_A(.,.; t) = max(dist_A - t, 0) (Sec. 3.2, "Capped attribute distance").
__device__ __forceinline__ uint32_t capped_distance(int32_t dist_a, uint32_t da, uint32_t t) {
  if (dist_a == JAG_F_RANGE_F32) {
    float fa = u2f(da), ft = u2f(t);
    return fa > ft ? f2u(__fsub_rn(fa, ft)) : 0u;
  }
  return da > t ? da - t : 0u;
}

__device__ __forceinline__ bool key_less(uint64_t ak, uint32_t aid, uint64_t bk, uint32_t bid) {
  return (ak < bk) | ((ak == bk) & (aid < bid));   // no short circuit: no branch
}

__device__ __forceinline__ uint64_t make_key(uint32_t first, float dist) {
  return ((uint64_t)first << 32) | (uint64_t)f2u(dist);
}

// 16-byte read-only gather of one chunk of a stored row.
__device__ __forceinline__ float4 ld_chunk(const float *p) {
  float4 v;
  asm volatile("ld.global.nc.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

// acc <- fma(t, t, acc) over the four elements of one chunk, in order, with
// t = q - x rounded to fp32.  Element order and rounding are part of the
// distance's definition; no contraction beyond these explicit fmas.
__device__ __forceinline__ float chunk_accumulate(float acc, float4 q, float4 x) {
  float t;
  t = __fsub_rn(q.x, x.x); acc = __fmaf_rn(t, t, acc);
  t = __fsub_rn(q.y, x.y); acc = __fmaf_rn(t, t, acc);
  t = __fsub_rn(q.z, x.z); acc = __fmaf_rn(t, t, acc);
  t = __fsub_rn(q.w, x.w); acc = __fmaf_rn(t, t, acc);
  return acc;
}

__device__ __forceinline__ uint4 ld_chunk_u4(const void *p) {
  uint4 v;
  asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

__device__ __forceinline__ float acc_elem(float acc, float q, float x) {
  const float t = __fsub_rn(q, x);
  return __fmaf_rn(t, t, acc);
}

// One 16-byte chunk of a stored row in format FMT: elements in increasing
// order, each as acc = fma(t, t, acc), t = q_i - x_i; BF16 elements are exact
// in fp32; FP8 elements are decoded exactly and multiplied by the row's
// scale s (rounded to fp32) first.
template <int FMT>
__device__ __forceinline__ float chunk_acc(float acc, const float4 (&q)[RowFmt<FMT>::Q4], uint4 raw, float s) {
  if constexpr (FMT == JAG_VEC_F32) {
    return chunk_accumulate(acc, q[0], make_float4(u2f(raw.x), u2f(raw.y), u2f(raw.z), u2f(raw.w)));
  } else if constexpr (FMT == JAG_VEC_BF16) {
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 qq = q[i >> 1];
      const float q0 = (i & 1) ? qq.z : qq.x, q1 = (i & 1) ? qq.w : qq.y;
      acc = acc_elem(acc, q0, u2f(w[i] << 16));
      acc = acc_elem(acc, q1, u2f(w[i] & 0xFFFF0000u));
    }
    return acc;
  } else {
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[i] & 0xFFFFu), __NV_E4M3);
      const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[i] >> 16), __NV_E4M3);
      const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&lo));
      const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&hi));
      const float4 qq = q[i];
      acc = acc_elem(acc, qq.x, __fmul_rn(s, a.x));
      acc = acc_elem(acc, qq.y, __fmul_rn(s, a.y));
      acc = acc_elem(acc, qq.z, __fmul_rn(s, b.x));
      acc = acc_elem(acc, qq.w, __fmul_rn(s, b.y));
    }
    return acc;
  }
}

// Butterfly over the P lanes of a group: acc_l + acc_(l xor o), o = P/2..1.
template <int P>
__device__ __forceinline__ float group_reduce(float acc) {
#pragma unroll
  for (int o = P / 2; o >= 1; o >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(kFull, acc, o));
  return acc;
}

// The same butterfly for U accumulators (U a power of two, U <= P), with the
// rows spread over the lanes as they are reduced: at each of the first
// log2(U) levels a lane keeps half of its rows (the lower half if bit o of
// its lane index is clear) and trades the other half with lane l xor o, so
// one shuffle moves two partial rows.  Every row still receives the sums
// acc_l + acc_(l xor o) of the plain butterfly (fp32 addition is
// commutative), in the same tree, with U - 1 + log2(P/U) shuffles instead of
// U log2(P).  On return lane l of a group holds the total of row
// (l mod P) / (P/U); spread_source gives the lane holding row s of group g.
template <int P, int U>
__device__ __forceinline__ float group_reduce_spread(float (&acc)[U]) {
  static_assert(U >= 1 && (U & (U - 1)) == 0 && U <= P, "rows per lane");
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = U / 2, o = P / 2; h >= 1; h >>= 1, o >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float send = upper ? acc[i] : acc[i + h];
      const float keep = upper ? acc[i + h] : acc[i];
      acc[i] = __fadd_rn(keep, __shfl_xor_sync(kFull, send, o));
    }
  }
  float v = acc[0];
#pragma unroll
  for (int o = P / (2 * U); o >= 1; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

template <int P, int U>
__device__ __forceinline__ int spread_source(int s, int g) {
  return g * P + s * (P / U);
}

// Status word bits written by kernels (read back by the host where needed).
enum : uint32_t {
  kErrVisitedOverflow = 1u,
  kErrCandOverflow = 2u,
  kErrBadFilter = 4u,
  kErrTcTimeout = 16u,   // the tensor-core scan gave up waiting for its MMAs
  kErrTcBound = 32u,     // a scan candidate broke the approximation bound (its query was rescanned exactly)
};

}  // namespace jag
