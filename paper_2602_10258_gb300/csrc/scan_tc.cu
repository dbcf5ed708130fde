// Exact pre-filter scan on the tensor cores (the Pre-Filtering baseline of
// the experiments, for the queries routed to the scan).
//
// Queries routed to the scan that share rows -- every query of one label
// shares its whole slice of the sorted column, overlapping ranges share part
// of theirs -- form dense contractions: rows x queries over the dimension.
// The scan runs in three steps:
//
//  1. grouping   the sorted columns are cut into tiles of 128 positions;
//                every slice-routed query is listed at each tile its slice
//                touches (a counting sort by tile); list-routed queries are
//                listed at their leader (the query that gathered the passing
//                set of their filter), whose list is cut into tiles of 128;
//  2. contract   a CTA takes one tile (128 rows) and up to 64 of the queries
//                listed there, gathers the fp32 rows and queries into shared
//                memory in the tensor core's K-major layout, and computes all
//                dot products with tcgen05.mma (kind::tf32, accumulators in
//                tensor memory); the epilogue writes the approximate squared
//                distance a = |x|^2 + |q|^2 - 2 q.x of every row inside the
//                query's slice;
//  3. select     one warp per query finds a threshold tau that at least k
//                rows reach (the k-th smallest of a sample of the a values),
//                computes the canonical fp32 distance of every row with
//                a <= tau + 2 eps, and keeps the best k by (distance, id).
//
// eps bounds |a - d| for the canonical fp32 distance d of any row:
//   eps = (2^-8 + dim 2^-20) (|q|^2 + max_x |x|^2) + 2^-100.
// TF32 operands carry 10 fraction bits (relative error < 2^-10 each, so a
// product is within 2^-8.99 of q_i x_i); the fp32 accumulation of dim + 8
// terms adds at most (dim + 8) 2^-22 of sum |q_i x_i| even if every addition
// is off by two units in the last place; |x|^2, |q|^2, the canonical
// distance and the final two operations add (3 dim + 8) 2^-24 of
// (|q|^2 + |x|^2); and sum |q_i x_i| <= (|q|^2 + |x|^2) / 2.  The bound is
// twice that sum.  Any row among the exact top k then has a <= tau + 2 eps:
// at least k rows have d <= tau + eps, so the k-th distance is at most
// tau + eps.  The answers are therefore the exact top k whatever the
// approximation, provided the bound holds; the select step checks it on
// every candidate and, should it ever fail, takes every row as a candidate.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "launch.h"
#include "launch_util.cuh"
#include "search_core.cuh"

namespace jag {

namespace {

constexpr int kTcRows = 128;         // rows per tile: the MMA's M
constexpr int kTcQueries = kTcItemQueries;   // queries per item at most: the MMA's N (padded to 16)
constexpr int kTcK = 128;            // fp32 elements of a row per pass (K chunk)
constexpr int kTcThreads = 128;      // four warps: one per 32-lane quarter of tensor memory
constexpr int kTcCols = 64;          // tensor-memory columns allocated (>= kTcQueries, a power of two >= 32)
constexpr uint32_t kTcSbo = kTcK * 32;                       // bytes between 8-row groups of an operand
constexpr size_t kTcSmemA = (size_t)kTcRows * kTcK * 4;      // 64 KB
constexpr size_t kTcSmemB = (size_t)kTcQueries * kTcK * 4;   // 32 KB
constexpr size_t kTcSmem = kTcSmemA + kTcSmemB + 1024;      // + alignment slack

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major operand without swizzling:
// 8-row x 16-byte core matrices, adjacent along K at lbo bytes, 8-row groups
// at sbo bytes; version bits 46-48 = 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::tf32: fp32 accumulator (bits 4-5 = 1), A and
// B in TF32 (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at
// bit 24.
__device__ __forceinline__ uint32_t tf32_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Bounded wait for the phase `parity` of an mbarrier (about a second at
// most); false if it did not complete.
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 24); ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (it >= 16) __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

__device__ __forceinline__ bool scan_routed(int32_t route) { return route == kRouteSlice || route == kRouteList; }

// The sorted column a slice-routed query reads: 0 = int32, 1 = float32.
__device__ __forceinline__ int slice_column(int32_t kind) { return kind == JAG_F_RANGE_F32 ? 1 : 0; }

// Work units of the scan: U = 2 T0 column tiles (T0 = ceil(n / 128) per
// column), then one unit per query: the list of a leader (the queries that
// read that leader's gathered list are listed there).
struct TcUnits {
  int64_t T0, U;
};

// The unit a scan-routed query is listed at for tile t of its slice, or its
// leader's list unit.
__device__ __forceinline__ int64_t list_unit(const TcUnits &tu, const QueryPlan &pl) { return 2 * tu.T0 + pl.begin; }

// (1a) each scan-routed query counts itself at every unit it is listed at
// (one warp per query, lanes over the tiles of a slice).
__global__ void tc_count_kernel(const QueryPlan *plans, const jag_filter *filters, int64_t nq, TcUnits tu,
                                int32_t *tcnt) {
  const int64_t qi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (qi >= nq) return;
  const QueryPlan pl = plans[qi];
  if (pl.route == kRouteList) {
    if (lane == 0) atomicAdd(&tcnt[list_unit(tu, pl)], 1);
    return;
  }
  if (pl.route != kRouteSlice || pl.end <= pl.begin) return;
  const int64_t base = slice_column(filters[qi].kind) * tu.T0;
  for (int64_t t = pl.begin / kTcRows + lane; t <= (pl.end - 1) / kTcRows; t += 32) atomicAdd(&tcnt[base + t], 1);
}

// Per unit: (listed queries, work items).  A column tile has one item per
// chunk of up to 64 listed queries; a leader's list one per (128 rows of the
// list, chunk of up to 64 listed queries).
__device__ __forceinline__ void unit_sizes(int64_t u, const TcUnits &tu, const int32_t *tcnt, const QueryPlan *plans,
                                           int64_t *entries, int64_t *items) {
  const int64_t c = u < tu.U ? tcnt[u] : 0;
  *entries = c;
  if (u < 2 * tu.T0 || c == 0) {
    *items = (c + kTcQueries - 1) / kTcQueries;
  } else {
    const int64_t rows = plans[u - 2 * tu.T0].count;
    *items = ((rows + kTcRows - 1) / kTcRows) * ((c + kTcQueries - 1) / kTcQueries);
  }
}

constexpr int kTcScanBlock = 1024;

// Inclusive block-wide sum of v over kTcScanBlock threads.
__device__ __forceinline__ int64_t block_scan_incl(int64_t v, int64_t *wsum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t t = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) wsum[warp] = v;
  __syncthreads();
  if (warp == 0) {
    int64_t w = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t t = __shfl_up_sync(kFull, w, o);
      if (lane >= o) w += t;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  const int64_t r = v + (warp > 0 ? wsum[warp - 1] : 0);
  __syncthreads();
  return r;
}

// (1b) exclusive prefix sums of (entries, items) over the units, in three
// passes: block totals, a scan of the block totals, block-local scans.
__global__ void __launch_bounds__(kTcScanBlock)
tc_sum_kernel(TcUnits tu, const int32_t *tcnt, const QueryPlan *plans, int64_t *bsum) {
  __shared__ int64_t wsum[32];
  const int64_t u = (int64_t)blockIdx.x * kTcScanBlock + threadIdx.x;
  int64_t e = 0, i = 0;
  if (u < tu.U) unit_sizes(u, tu, tcnt, plans, &e, &i);
  const int64_t es = block_scan_incl(e, wsum);
  const int64_t is = block_scan_incl(i, wsum);
  if (threadIdx.x == kTcScanBlock - 1) { bsum[2 * blockIdx.x] = es; bsum[2 * blockIdx.x + 1] = is; }
}

__global__ void __launch_bounds__(kTcScanBlock)
tc_sum_blocks_kernel(int64_t nblk, int64_t *bsum, unsigned long long *counters) {
  __shared__ int64_t wsum[32];
  int64_t ce = 0, ci = 0;
  for (int64_t b0 = 0; b0 < nblk; b0 += kTcScanBlock) {
    const int64_t b = b0 + threadIdx.x;
    const int64_t e = b < nblk ? bsum[2 * b] : 0, i = b < nblk ? bsum[2 * b + 1] : 0;
    const int64_t es = block_scan_incl(e, wsum);
    const int64_t is = block_scan_incl(i, wsum);
    __syncthreads();
    if (b < nblk) { bsum[2 * b] = ce + es - e; bsum[2 * b + 1] = ci + is - i; }
    __shared__ int64_t tot[2];
    if (threadIdx.x == kTcScanBlock - 1) { tot[0] = es; tot[1] = is; }
    __syncthreads();
    ce += tot[0];
    ci += tot[1];
    __syncthreads();
  }
  if (threadIdx.x == 0) { counters[0] = (unsigned long long)ce; counters[1] = (unsigned long long)ci; }
}

__global__ void __launch_bounds__(kTcScanBlock)
tc_offsets_kernel(TcUnits tu, const int32_t *tcnt, const QueryPlan *plans, const int64_t *bsum, int32_t *toff,
                  int64_t *ioff) {
  __shared__ int64_t wsum[32];
  const int64_t u = (int64_t)blockIdx.x * kTcScanBlock + threadIdx.x;
  int64_t e = 0, i = 0;
  if (u < tu.U) unit_sizes(u, tu, tcnt, plans, &e, &i);
  const int64_t es = block_scan_incl(e, wsum);
  const int64_t is = block_scan_incl(i, wsum);
  if (u < tu.U) {
    toff[u] = (int32_t)(bsum[2 * blockIdx.x] + es - e);
    ioff[u] = bsum[2 * blockIdx.x + 1] + is - i;
  }
}

// (1c) each scan-routed query enters the list of every unit it counted at.
__global__ void tc_fill_kernel(const QueryPlan *plans, const jag_filter *filters, int64_t nq, TcUnits tu,
                               const int32_t *toff, int32_t *tfill, int32_t *tq) {
  const int64_t qi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (qi >= nq) return;
  const QueryPlan pl = plans[qi];
  if (pl.route == kRouteList) {
    if (lane == 0) {
      const int64_t u = list_unit(tu, pl);
      tq[toff[u] + atomicAdd(&tfill[u], 1)] = (int32_t)qi;
    }
    return;
  }
  if (pl.route != kRouteSlice || pl.end <= pl.begin) return;
  const int64_t base = slice_column(filters[qi].kind) * tu.T0;
  for (int64_t t = pl.begin / kTcRows + lane; t <= (pl.end - 1) / kTcRows; t += 32) {
    const int32_t pos = atomicAdd(&tfill[base + t], 1);
    tq[toff[base + t] + pos] = (int32_t)qi;
  }
}

// (1d) the unit of every work item, and |q|^2 of every scan-routed query
// (one warp per query).
__global__ void tc_items_kernel(TcUnits tu, const int32_t *tcnt, const QueryPlan *plans, const int64_t *ioff,
                                int32_t *item_unit) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= tu.U) return;
  int64_t e, n;
  unit_sizes(u, tu, tcnt, plans, &e, &n);
  for (int64_t j = 0; j < n; ++j) item_unit[ioff[u] + j] = (int32_t)u;
}

__global__ void tc_qnorm_kernel(const QueryPlan *plans, const float *queries, int d, int64_t nq, float *qnorm) {
  const int64_t qi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (qi >= nq) return;
  const int32_t r = plans[qi].route;
  if (r != kRouteSlice && r != kRouteList) return;
  float acc = 0.f;
  for (int e = lane; e < d; e += 32) { const float t = queries[qi * d + e]; acc = __fmaf_rn(t, t, acc); }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(kFull, acc, o));
  if (lane == 0) qnorm[qi] = acc;
}

// (2) the contraction.  Persistent CTAs of four warps claim work items; per
// item: the rows and queries go to shared memory (rows by 16-byte cp.async
// from the fp32 rows, queries by plain loads, both zero padded), one thread
// issues the MMAs of each 128-element K chunk into tensor memory, and after
// the MMAs' commit the four warps read their 32 rows each and write the
// approximate distances approx[q][position of the row in q's passing set].
__global__ void __launch_bounds__(kTcThreads, 1)
tc_contract_kernel(DevIndex ix, const float *queries, int d, const jag_filter *filters, const QueryPlan *plans,
                   const int32_t *lists, int64_t cap, TcUnits tu, const int32_t *tcnt, const int32_t *toff,
                   const int32_t *tq, const int64_t *ioff, const int32_t *item_unit, const float *qnorm,
                   unsigned long long *counters, float *approx, uint32_t *status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float *sa = reinterpret_cast<float *>(smem);
  float *sb = reinterpret_cast<float *>(smem + kTcSmemA);
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t s_taddr;
  __shared__ int64_t s_item;
  __shared__ int32_t s_qid[kTcQueries];
  __shared__ int32_t s_qb[kTcQueries];   // first position of the row set in the query's own passing set
  __shared__ int32_t s_qm[kTcQueries];   // rows of the query's passing set
  __shared__ float s_qn[kTcQueries];
  __shared__ int32_t s_rid[kTcRows];
  __shared__ int s_abort;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t mbar_addr = smem_u32(&mbar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_addr) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_taddr)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = s_taddr;
  const uint32_t sa_addr = smem_u32(sa), sb_addr = smem_u32(sb);
  const unsigned long long ni = counters[1];
  uint32_t phase = 0;
  const int nkc = (d + kTcK - 1) / kTcK;
  for (;;) {
    if (tid == 0) s_item = (int64_t)atomicAdd(counters + 2, 1ull);
    __syncthreads();
    const int64_t item = s_item;
    __syncthreads();   // every thread has read s_item before the next claim overwrites it
    if (item >= (int64_t)ni) break;
    const int64_t lo = item_unit[item];
    const int64_t local = item - ioff[lo];
    int nrow, nqc;
    if (lo < 2 * tu.T0) {
      // a tile of a sorted column and a chunk of the queries listed there;
      // row r of the tile is position t * 128 + r of the column, which is
      // position t * 128 + r - begin of a query's own slice
      const int col = (int)(lo / tu.T0);
      const int64_t t = lo - col * tu.T0;
      const int32_t *sid = col ? ix.sf32_id : ix.si32_id;
      nrow = (int)min64(kTcRows, ix.n - t * kTcRows);
      nqc = (int)min64(kTcQueries, (int64_t)tcnt[lo] - local * kTcQueries);
      if (tid < nqc) {
        const int32_t qi = tq[toff[lo] + local * kTcQueries + tid];
        const QueryPlan pl = plans[qi];
        s_qid[tid] = qi;
        s_qb[tid] = (int32_t)(t * kTcRows - pl.begin);
        s_qm[tid] = (int32_t)(pl.end - pl.begin);
        s_qn[tid] = qnorm[qi];
      }
      s_rid[tid] = tid < nrow ? sid[t * kTcRows + tid] : -1;
    } else {
      // 128 rows of a leader's gathered list and a chunk of the queries that
      // share it (row r is position tile * 128 + r of each one's passing set)
      const int64_t lead = lo - 2 * tu.T0;
      const int32_t cnt = plans[lead].count;
      const int64_t nchunk = ((int64_t)tcnt[lo] + kTcQueries - 1) / kTcQueries;
      const int64_t tile = local / nchunk, chunk = local - tile * nchunk;
      nrow = (int)min64(kTcRows, (int64_t)cnt - tile * kTcRows);
      nqc = (int)min64(kTcQueries, (int64_t)tcnt[lo] - chunk * kTcQueries);
      if (tid < nqc) {
        const int32_t qi = tq[toff[lo] + chunk * kTcQueries + tid];
        s_qid[tid] = qi;
        s_qb[tid] = (int32_t)(tile * kTcRows);
        s_qm[tid] = cnt;
        s_qn[tid] = qnorm[qi];
      }
      s_rid[tid] = tid < nrow ? lists[lead * cap + tile * kTcRows + tid] : -1;
    }
    const int N = (nqc + 15) & ~15;
    __syncthreads();
    for (int kc = 0; kc < nkc; ++kc) {
      const int k0 = kc * kTcK;
      const int kw = min(kTcK, ((d - k0) + 7) & ~7);   // elements of this chunk, a multiple of 8
      const int c4n = kw / 4;                          // 16-byte chunks per row
      // rows: lane -> (row % 8, chunk), so a warp writes 8 rows x 4 chunks of 16 bytes
      for (int blk = warp; blk < (kTcRows / 8) * ((c4n + 3) / 4); blk += kTcThreads / 32) {
        const int rg = blk % (kTcRows / 8), cg = blk / (kTcRows / 8);
        const int r = rg * 8 + (lane & 7), c4 = cg * 4 + (lane >> 3);
        if (c4 < c4n) {
          const int kk = k0 + 4 * c4;
          const int32_t id = s_rid[r];
          const bool ok = id >= 0 && kk < ix.xs;
          const float *src = ok ? ix.x + (int64_t)id * ix.xs + kk : ix.x;
          cp_async16(sa_addr + rg * kTcSbo + c4 * 128 + (r & 7) * 16, src, ok ? 16u : 0u);
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      // queries: plain loads (rows of d floats need not be 16-byte aligned)
      for (int e = tid; e < N * c4n; e += kTcThreads) {
        const int n = e / c4n, c4 = e - n * c4n;
        const int kk = k0 + 4 * c4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n < nqc) {
          const float *qr = queries + (int64_t)s_qid[n] * d;
          v.x = kk + 0 < d ? qr[kk + 0] : 0.f;
          v.y = kk + 1 < d ? qr[kk + 1] : 0.f;
          v.z = kk + 2 < d ? qr[kk + 2] : 0.f;
          v.w = kk + 3 < d ? qr[kk + 3] : 0.f;
        }
        *reinterpret_cast<float4 *>(reinterpret_cast<uint8_t *>(sb) + (n >> 3) * kTcSbo + c4 * 128 + (n & 7) * 16) = v;
      }
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      if (tid == 0) {
        const uint32_t idesc = tf32_idesc(kTcRows, N);
        for (int s = 0; s < kw / 8; ++s) {
          const uint64_t ad = smem_desc(sa_addr + s * 256, 128, kTcSbo);
          const uint64_t bd = smem_desc(sb_addr + s * 256, 128, kTcSbo);
          const uint32_t accum = (kc > 0 || s > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\t"
              "setp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
              "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
              : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_addr)
                     : "memory");
      }
      const bool ok = __syncthreads_and(mbar_wait(mbar_addr, phase) ? 1 : 0) != 0;
      phase ^= 1u;
      tc_fence_after();
      if (!ok) {
        // the MMAs did not complete in time: give them a second bounded wait
        // before tensor memory is released, flag the error and stop
        if (tid == 0) { atomicOr(status, kErrTcTimeout); s_abort = 1; }
        mbar_wait(mbar_addr, phase ^ 1u);
        break;
      }
    }
    __syncthreads();
    if (s_abort) break;
    // epilogue: warp w holds rows 32w + lane in tensor-memory lanes 32w..32w+31
    const int r = warp * 32 + lane;
    const int32_t rid = s_rid[r];
    const float xn = rid >= 0 ? ix.xnorm[rid] : 0.f;
    for (int c0 = 0; c0 < N; c0 += 16) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int n = c0 + j;
        const int pos = s_qb[n < kTcQueries ? n : 0] + r;   // the row's position in the query's passing set
        if (n < nqc && r < nrow && pos >= 0 && pos < s_qm[n]) {
          const float a = __fsub_rn(__fadd_rn(xn, s_qn[n]), __fmul_rn(2.f, u2f(v[j])));
          approx[(int64_t)s_qid[n] * cap + pos] = a;
        }
      }
    }
    tc_fence_before();
    __syncthreads();   // shared memory and tensor memory are reused by the next item
    tc_fence_after();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTcCols) : "memory");
}

__device__ __forceinline__ void group_rows(const DevIndex &ix, const jag_filter *filters, const QueryPlan &pl,
                                           int64_t qi, const int32_t *lists, int64_t cap, const int32_t **ids,
                                           int64_t *m) {
  if (pl.route == kRouteSlice) {
    *ids = (slice_column(filters[qi].kind) ? ix.sf32_id : ix.si32_id) + pl.begin;
    *m = pl.end - pl.begin;
  } else {
    *ids = lists + pl.begin * cap;   // the leader's list
    *m = pl.count;
  }
}

// (3) selection per scan-routed query (one warp each), see the file comment.
constexpr int kSelUnroll = 8;   // approximations read per lane per round
template <int CAP, int P, int CPL>
__global__ void __launch_bounds__(kSearchWarps * 32)
tc_select_kernel(DevIndex ix, const float *queries, int d, const jag_filter *filters, const QueryPlan *plans,
                 const int32_t *lists, int64_t cap, int64_t nq, int k, const float *approx, int32_t *out_ids,
                 float *out_dist, int32_t *counters, uint32_t *status) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lcap = list_slots(k);
  const WarpSmem S = carve_warp_smem(smem + warp * warp_smem_bytes(lcap, 5), lcap, 5);
  const int64_t qi = (int64_t)blockIdx.x * kSearchWarps + warp;
  if (qi >= nq) return;
  const QueryPlan pl = plans[qi];
  if (!scan_routed(pl.route)) return;
  const int32_t *ids;
  int64_t m;
  group_rows(ix, filters, pl, qi, lists, cap, &ids, &m);
  const float *a = approx + qi * cap;
  QChunks<CPL, JAG_VEC_F32> q;
  load_point<P, CPL>(queries + qi * d, d, q);
  // eps from |q|^2 and the largest |x|^2 of the index
  float qn = 0.f;
  for (int e = lane; e < d; e += 32) { const float t = queries[qi * d + e]; qn = __fmaf_rn(t, t, qn); }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) qn = __fadd_rn(qn, __shfl_xor_sync(kFull, qn, o));
  const float eps = __fmaf_rn(__fadd_rn(0.00390625f, __fmul_rn((float)d, 9.5367431640625e-07f)),
                              __fadd_rn(qn, ix.xnorm_max), 7.888609052210118e-31f);
  // tau: the k-th smallest of the four smallest a values of every lane (at
  // least k rows have a <= tau); every row is a candidate when m <= 4k or k > 128
  float thr = INFINITY;
  if (m > 4 * (int64_t)k && k <= 128) {
    float r0 = INFINITY, r1 = INFINITY, r2 = INFINITY, r3 = INFINITY;
    for (int64_t b = 0; b < m; b += 32 * kSelUnroll) {
      float vv[kSelUnroll];   // kSelUnroll independent loads in flight per lane
#pragma unroll
      for (int r = 0; r < kSelUnroll; ++r) {
        const int64_t j = b + r * 32 + lane;
        vv[r] = j < m ? a[j] : INFINITY;
      }
#pragma unroll
      for (int r = 0; r < kSelUnroll; ++r) {
        const float v = vv[r];
        if (v < r3) {
          r3 = v;
          if (r3 < r2) { const float t = r2; r2 = r3; r3 = t; }
          if (r2 < r1) { const float t = r1; r1 = r2; r2 = t; }
          if (r1 < r0) { const float t = r0; r0 = r1; r1 = t; }
        }
      }
    }
    float tau = INFINITY;
    for (int i = 0; i < k; ++i) {
      float v = r0;
      int who = lane;
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        const float ov = __shfl_xor_sync(kFull, v, o);
        const int ow = __shfl_xor_sync(kFull, who, o);
        if (ov < v || (ov == v && ow < who)) { v = ov; who = ow; }
      }
      tau = v;
      if (lane == who) { r0 = r1; r1 = r2; r2 = r3; r3 = INFINITY; }
    }
    thr = __fadd_rn(tau, __fmul_rn(2.f, eps));
  }
  int cnt = 0, ncand = 0;
  for (int pass = 0; pass < 2; ++pass) {
    bool broken = false;
    cnt = 0;
    ncand = 0;
    for (int64_t b0 = 0; b0 < m; b0 += 32 * kSelUnroll) {
      float vv[kSelUnroll];
      uint32_t any = 0;
#pragma unroll
      for (int r = 0; r < kSelUnroll; ++r) {
        const int64_t j = b0 + r * 32 + lane;
        vv[r] = j < m ? a[j] : INFINITY;
        any |= (j < m && !(vv[r] > thr)) ? (1u << r) : 0u;
      }
      if (!__any_sync(kFull, any != 0)) continue;
      for (int r = 0; r < kSelUnroll; ++r) {
        const int64_t b = b0 + r * 32;
        if (b >= m) break;
        const bool cand = (any >> r) & 1u;
        const uint32_t cm = __ballot_sync(kFull, cand);
        if (!cm) continue;
        float v = vv[0];   // vv[r] by selection, so that vv stays in registers
#pragma unroll
        for (int i = 1; i < kSelUnroll; ++i) v = r == i ? vv[i] : v;
        const int nc = __popc(cm);
        ncand += nc;
        if (cand) {
          const int pos = __popc(cm & lanemask_lt());
          S.cid[pos] = (uint32_t)ids[b + lane];
          S.ck1[pos] = f2u(v);   // its approximation, for the bound check
        }
        __syncwarp();
        const bool full = cnt == k;
        const uint64_t tkey = full ? S.bkey[k - 1] : kNoKey;
        const uint32_t tid = full ? S.bid[k - 1] : kEmptySlot;
        const float dist = candidate_distances<P, CPL, 4, JAG_VEC_F32, true>(ix, q, S.cid, nc);
        uint64_t ck = kNoKey;
        uint32_t cv = kEmptySlot;
        if (lane < nc) {
          if (thr != INFINITY && !(fabsf(__fsub_rn(u2f(S.ck1[lane]), dist)) <= eps)) broken = true;
          ck = make_key(0u, dist);
          cv = S.cid[lane];
          if (full && !key_less(ck, cv, tkey, tid)) { ck = kNoKey; cv = kEmptySlot; }
        }
        int r0;
        cnt = merge_candidates<CAP, false>(S.bkey, S.bid, cnt, k, ck, cv, r0);
      }
    }
    if (!__any_sync(kFull, broken)) break;
    if (lane == 0) atomicOr(status, kErrTcBound);
    thr = INFINITY;   // the bound failed on a candidate: every row is a candidate
  }
  write_answers(S, cnt, qi, k, out_ids, out_dist);
  if (counters && lane == 0) {
    int32_t *c = counters + qi * 4;
    c[0] = 0; c[1] = ncand; c[2] = (int32_t)m; c[3] = 1;
  }
}

__global__ void row_norms_kernel(DevIndex ix, float *xn, unsigned int *xmax) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ix.n) return;
  const float *r = ix.x + i * ix.xs;
  float acc = 0.f;
  for (int e = 0; e < ix.d; ++e) acc = __fmaf_rn(r[e], r[e], acc);
  xn[i] = acc;
  atomicMax(xmax, f2u(acc));   // non-negative floats order as their bit patterns
}

template <int CAP, int P, int CPL>
cudaError_t launch_select(const SearchLaunch &L) {
  const size_t sm = (size_t)kSearchWarps * warp_smem_bytes(list_slots(L.k), 5);
  auto kern = tc_select_kernel<CAP, P, CPL>;
  if (blocks_per_sm(kern, sm) == 0) return cudaErrorInvalidConfiguration;
  kern<<<(unsigned)((L.nq + kSearchWarps - 1) / kSearchWarps), kSearchWarps * 32, sm, L.stream>>>(
      L.ix, L.queries, L.d, L.filters, L.plans, L.lists, L.cap, L.nq, L.k, L.tc.approx, L.out_ids, L.out_dist,
      L.counters, L.status);
  return cudaGetLastError();
}

}  // namespace

cudaError_t row_norms(const DevIndex &ix, float *xn, unsigned int *dmax, float *xmax_host, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(dmax, 0, sizeof(unsigned int), stream);
  if (e != cudaSuccess) return e;
  row_norms_kernel<<<(unsigned)((ix.n + 255) / 256), 256, 0, stream>>>(ix, xn, dmax);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  unsigned int hmax = 0;
  if ((e = cudaMemcpyAsync(&hmax, dmax, sizeof(unsigned int), cudaMemcpyDeviceToHost, stream)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return e;
  float f;
  memcpy(&f, &hmax, sizeof(f));
  *xmax_host = f;
  return cudaSuccess;
}

int64_t tc_column_tiles(int64_t n) { return (n + kTcRows - 1) / kTcRows; }

cudaError_t launch_scan_tc(const SearchLaunch &L) {
  const TcScratch &T = L.tc;
  const int64_t nq = L.nq;
  cudaError_t e;
  TcUnits tu;
  tu.T0 = tc_column_tiles(L.ix.n);
  tu.U = 2 * tu.T0 + nq;
  const int64_t nblk = (tu.U + kTcScanBlock - 1) / kTcScanBlock;
  if ((e = cudaMemsetAsync(T.tcnt, 0, sizeof(int32_t) * (size_t)tu.U, L.stream)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(T.tfill, 0, sizeof(int32_t) * (size_t)tu.U, L.stream)) != cudaSuccess) return e;
  const unsigned wb = (unsigned)((nq * 32 + 255) / 256);   // one warp per query
  tc_count_kernel<<<wb, 256, 0, L.stream>>>(L.plans, L.filters, nq, tu, T.tcnt);
  tc_sum_kernel<<<(unsigned)nblk, kTcScanBlock, 0, L.stream>>>(tu, T.tcnt, L.plans, T.bsum);
  tc_sum_blocks_kernel<<<1, kTcScanBlock, 0, L.stream>>>(nblk, T.bsum, L.work + 4);
  tc_offsets_kernel<<<(unsigned)nblk, kTcScanBlock, 0, L.stream>>>(tu, T.tcnt, L.plans, T.bsum, T.toff, T.ioff);
  tc_fill_kernel<<<wb, 256, 0, L.stream>>>(L.plans, L.filters, nq, tu, T.toff, T.tfill, T.tq);
  tc_items_kernel<<<(unsigned)((tu.U + 255) / 256), 256, 0, L.stream>>>(tu, T.tcnt, L.plans, T.ioff, T.item_unit);
  tc_qnorm_kernel<<<wb, 256, 0, L.stream>>>(L.plans, L.queries, L.d, nq, T.qnorm);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int bps = blocks_per_sm(tc_contract_kernel, kTcSmem, kTcThreads / 32);
  if (bps == 0) return cudaErrorInvalidConfiguration;
  {
    // CTAs that fit an SM by shared memory (the occupancy query can report
    // fewer for this kernel); the CTAs only claim items from a counter and
    // never wait on one another, so more of them than fit at once is safe
    int dev = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const int by_smem = per_sm / (int)(kTcSmem + 4096);
    bps = std::max(bps, std::min(by_smem, 2));
  }
  tc_contract_kernel<<<(unsigned)(bps * num_sms()), kTcThreads, kTcSmem, L.stream>>>(
      L.ix, L.queries, L.d, L.filters, L.plans, L.lists, L.cap, tu, T.tcnt, T.toff, T.tq, T.ioff, T.item_unit,
      T.qnorm, L.work + 4, T.approx, L.status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int P, CPL;
  if (!row_mapping(L.ix.nchunks, &P, &CPL)) return cudaErrorInvalidValue;
#define JAG_SCASE(CC, PP, QQ) \
  if (list_capacity(L.k) == CC && P == PP && CPL == QQ) return launch_select<CC, PP, QQ>(L);
#define JAG_SROWS(CC) JAG_SCASE(CC, 8, 1) JAG_SCASE(CC, 16, 1) JAG_SCASE(CC, 32, 1) JAG_SCASE(CC, 32, 2) \
  JAG_SCASE(CC, 32, 4) JAG_SCASE(CC, 32, 8)
  JAG_SROWS(64)
  JAG_SROWS(128)
  JAG_SROWS(256)
#undef JAG_SROWS
#undef JAG_SCASE
  return cudaErrorInvalidValue;
}

}  // namespace jag
