// K1: the graph-search kernel of a query batch, for rows stored in format FMT
// (one translation unit per format keeps compile units small).
#pragma once

#include <algorithm>

#include "launch.h"
#include "launch_util.cuh"
#include "search_core.cuh"

namespace jag {

// Each warp takes queries from a global counter and runs GreedySearch with
// D_F (Algorithm 2) for the graph-routed ones.  With fp32 rows it writes the
// answers; with BF16 / FP8 rows it leaves the ids of the leading rr passing
// entries of the final list for the fp32 re-rank.
// Lanes per row of the graph search for rows of 17..32 chunks (a 128-d fp32
// row is 32 chunks).
constexpr int kGraphLanes = 32;

// Warps (searches) per CTA of the graph kernel: 2, so that CTAs leave an SM
// in finer steps during the last wave and the exact scan's CTAs fit sooner;
// 4 for a traced policy search, whose 64-byte policy context per warp would
// otherwise cost a CTA per SM.
__host__ __device__ constexpr int graph_warps(int POL) { return POL == 2 ? 4 : 2; }

// CTAs per SM the graph kernel is compiled for (its register budget): one
// row chunk per lane -- 32 warps (64 registers); the plain search of FP8 rows,
// whose 8-lane rows leave registers to spare, 36 warps (56 registers),
// measured faster on the 128-d label workload than 32 or 40; wider rows, 1.
__host__ __device__ constexpr int graph_min_blocks(int CPL, int FMT, int POL) {
  return CPL != 1 ? 1 : (FMT == JAG_VEC_FP8 && POL == 0 ? 36 : 32) / graph_warps(POL);
}

// POL: 0 plain, 1 with the search policy, 2 with the policy and its trace.
template <int CAP, int P, int CPL, int FMT, int POL>
__global__ void __launch_bounds__(graph_warps(POL) * 32, graph_min_blocks(CPL, FMT, POL))
query_kernel(DevIndex ix, const float *queries, int d, const jag_filter *filters, const QueryPlan *plans,
             const uint8_t *lut_base, int64_t nq, int k, int ls, int hbits, int rr, int32_t *rr_ids,
             int32_t *out_ids, float *out_dist, int32_t *counters, unsigned long long *work,
             const __grid_constant__ jag_policy pol) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lcap = list_slots(ls);
  const size_t wbytes = warp_smem_bytes(lcap, hbits) + (POL == 2 ? kPolicyCtxBytes : 0);
  uint8_t *wb = smem + warp * wbytes;
  const WarpSmem S = carve_warp_smem(wb, lcap, hbits);
  const int64_t sample = ix.n < 4096 ? ix.n : 4096;
  for (;;) {
    unsigned long long qi = 0;
    if (lane == 0) qi = atomicAdd(work, 1ull);
    qi = __shfl_sync(kFull, qi, 0);
    if (qi >= (unsigned long long)nq) return;
    const QueryPlan pl = plans[qi];
    if (pl.route != kRouteGraph) continue;
    QChunks<CPL, FMT> q;
    load_point<P, CPL, FMT>(queries + (int64_t)qi * d, d, q);
    const jag_filter f = filters[qi];
    const QueryKey key{f.kind, f.payload, pl.lut_off >= 0 ? lut_base + pl.lut_off : nullptr};
    NoSink sink;
    SearchStats st;
    int cnt;
    if constexpr (POL == 1) {
      // the plain search loop up to hop h0, the decision outside it, then the
      // same loop again from where it stopped (one inlined copy of the loop,
      // no call inside it).  Only the beam and the hop limit of the current
      // phase stay live across the loop: the limit is h0 before the decision
      // and never h0 after it (a stop at h0 ends the search at the decision),
      // and the decision's inputs are read again when it is taken.  The
      // network's scratch is the candidate arrays cid, ck1, free between hops.
      SearchCursor cur{0, 0};
      int lsq = ls, lim = pol.mode != JAG_POLICY_PLAIN ? pol.h0 : 0x7FFFFFFF;
      if (pol.features && lane < JAG_MLP_FEATURES) pol.features[(int64_t)qi * JAG_MLP_FEATURES + lane] = 0.f;
      for (;;) {
        cnt = greedy_search<CAP, P, CPL, FMT, 0, true>(ix, key, q, lsq, hbits, S, sink, st, lim, &cur);
        if (lim != pol.h0 || st.hops < lim) break;
        __syncwarp();
        const QueryPlan pd = plans[qi];
        const int32_t kind = filters[qi].kind;
        const int64_t est = (kind == JAG_F_SUBSET || kind == JAG_F_BOOL) ? (int64_t)pd.est * ix.n / sample
                            : (kind == JAG_F_NONE ? ix.n : (int64_t)pd.est);
        const PolicyOut o = policy_decide(pol, S, reinterpret_cast<float *>(S.cid), cnt, k, est, kind, ls,
                                          pol.features ? pol.features + (int64_t)qi * JAG_MLP_FEATURES : nullptr,
                                          pol.forced ? pol.forced + (int64_t)qi * 2 : nullptr);
        __syncwarp();
        lsq = o.beam;
        if (cnt > lsq) cnt = lsq;
        if (o.stop > 0 && st.hops >= o.stop) break;
        lim = o.stop > 0 ? o.stop : 0x7FFFFFFF;
        cur.cnt = cnt;
      }
    } else if constexpr (POL == 2) {
      const int64_t est = (f.kind == JAG_F_SUBSET || f.kind == JAG_F_BOOL) ? (int64_t)pl.est * ix.n / sample
                          : (f.kind == JAG_F_NONE ? ix.n : (int64_t)pl.est);
      // the policy network's scratch: the candidate arrays cid, ck1 (free between hops)
      if (lane == 0)
        *policy_ctx(S) = PolicyCtx{&pol, est, f.kind, k, reinterpret_cast<float *>(S.cid),
                                   pol.features ? pol.features + (int64_t)qi * JAG_MLP_FEATURES : nullptr,
                                   pol.decisions ? pol.decisions + (int64_t)qi * 4 : nullptr,
                                   pol.forced ? pol.forced + (int64_t)qi * 2 : nullptr, 0};
      __syncwarp();
      cnt = greedy_search<CAP, P, CPL, FMT, POL>(ix, key, q, ls, hbits, S, sink, st);
    } else {
      cnt = greedy_search<CAP, P, CPL, FMT, 0>(ix, key, q, ls, hbits, S, sink, st);
    }
    if (FMT == JAG_VEC_F32) {
      write_answers(S, cnt, (int64_t)qi, k, out_ids, out_dist);
    } else {
      for (int j = lane; j < rr; j += 32) {
        int32_t id = -1;
        if (j < cnt && (S.bkey[j] >> 32) == 0) id = (int32_t)(S.bid[j] & ~kExpanded);
        rr_ids[(int64_t)qi * rr + j] = id;
      }
    }
    if (counters && lane == 0) {
      int32_t *c = counters + qi * 4;
      c[0] = st.hops; c[1] = st.seen; c[2] = st.dcs; c[3] = 0;
    }
    __syncwarp();
  }
}

template <int CAP, int P, int CPL, int FMT, int POL>
static cudaError_t launch_graph_one(const SearchLaunch &L) {
  const int lcap = list_slots(L.ls);
  constexpr int kGraphWarps = graph_warps(POL);
  auto kern = query_kernel<CAP, P, CPL, FMT, POL>;
  // The default visited set (2^10 slots) shrinks to 2^9 when that brings the
  // blocks per SM up to the number the kernel is compiled for; the set only
  // saves recomputation, answers do not depend on its size.
  int hbits = L.hbits;
  auto smem_of = [&](int hb) {
    return (size_t)kGraphWarps * (warp_smem_bytes(lcap, hb) + (POL == 2 ? kPolicyCtxBytes : 0));
  };
  int bps = blocks_per_sm(kern, smem_of(hbits), kGraphWarps);
  if (L.hbits_auto && hbits > 9 && bps < graph_min_blocks(CPL, FMT, POL)) {
    const int b9 = blocks_per_sm(kern, smem_of(9), kGraphWarps);
    if (b9 > bps) { hbits = 9; bps = b9; }
  }
  const size_t smem = smem_of(hbits);
  if (bps == 0) return cudaErrorInvalidConfiguration;
  const int64_t want = std::max<int64_t>((L.nq + kGraphWarps - 1) / kGraphWarps, 1);
  const int64_t grid = std::min<int64_t>((int64_t)bps * num_sms(), want);
  if (L.ev_begin) cudaEventRecord(L.ev_begin, L.stream);
  kern<<<(unsigned)grid, kGraphWarps * 32, smem, L.stream>>>(L.ix, L.queries, L.d, L.filters, L.plans, L.lut,
                                                             L.nq, L.k, L.ls, hbits, L.rr, L.rr_ids, L.out_ids,
                                                             L.out_dist, L.counters, L.work, L.policy);
  if (L.ev_end) cudaEventRecord(L.ev_end, L.stream);
  return cudaGetLastError();
}

template <int CAP, int FMT, int POL>
static cudaError_t launch_graph_cap(const SearchLaunch &L, int P, int CPL) {
#define JAG_GCASE(PP, CC) \
  if (P == PP && CPL == CC) return launch_graph_one<CAP, PP, CC, FMT, POL>(L);
  if constexpr (CAP == 512) {
    // the 512-entry list: plain search of rows of at most 32 chunks
    JAG_GCASE(8, 1)
    JAG_GCASE(16, 1)
    JAG_GCASE(32, 1)
    return cudaErrorInvalidValue;
  }
  JAG_GCASE(8, 1)
  JAG_GCASE(16, 1)
  JAG_GCASE(32, 1)
  JAG_GCASE(32, 2)
  JAG_GCASE(kGraphLanes, 32 / kGraphLanes)
  if constexpr (!POL) {
    JAG_GCASE(32, 4)
    if constexpr (FMT == JAG_VEC_F32) {
      JAG_GCASE(32, 8)
    }
  }
#undef JAG_GCASE
  return cudaErrorInvalidValue;
}

template <int FMT>
static cudaError_t launch_graph_fmt_plain(const SearchLaunch &L, int P, int CPL) {
  switch (list_capacity(L.ls)) {
    case 64: return launch_graph_cap<64, FMT, 0>(L, P, CPL);
    case 128: return launch_graph_cap<128, FMT, 0>(L, P, CPL);
    case 256: return launch_graph_cap<256, FMT, 0>(L, P, CPL);
    case 512: return launch_graph_cap<512, FMT, 0>(L, P, CPL);
    default: return cudaErrorInvalidValue;
  }
}

template <int FMT>
cudaError_t launch_graph_fmt(const SearchLaunch &L) {
  int P, CPL;
  const int nch = FMT == JAG_VEC_F32 ? L.ix.nchunks : L.ix.qchunks;
  if (!row_mapping(nch, &P, &CPL)) return cudaErrorInvalidValue;
  // rows of 17..32 chunks: kGraphLanes lanes per row, the first butterfly
  // levels folded into registers (fewer shuffles per row, more rows per load)
  if (nch > 16 && nch <= 32) { P = kGraphLanes; CPL = 32 / kGraphLanes; }
  if (L.has_policy) {
    // traces (decisions written) take the capacity-256 kernel for any beam
    if (L.policy.decisions) return launch_graph_cap<256, FMT, 2>(L, P, CPL);
    // the plain mode without features is the plain search
    if (L.policy.mode == JAG_POLICY_PLAIN && !L.policy.features) return launch_graph_fmt_plain<FMT>(L, P, CPL);
    if (list_capacity(L.ls) <= 128) return launch_graph_cap<128, FMT, 1>(L, P, CPL);
    return launch_graph_cap<256, FMT, 1>(L, P, CPL);
  }
  return launch_graph_fmt_plain<FMT>(L, P, CPL);
}

}  // namespace jag
