// GPU index build: Insert (Algorithm 3) and JointRobustPrune (Algorithm 4)
// over a deterministic batch schedule.
//
// Schedule (the paper inserts points one at a time; batch insertion with a
// frozen graph per batch is how parallel builders run Insert):
//   entry vertex s = the point nearest (fp64) to the fp64 centroid, lowest id
//   on a tie; insertion order s, then the other points by increasing id;
//   after s, each batch takes the next min(#inserted, max(1, n/50)) points.
//   Within a batch: (1) every point p runs GreedySearch with D_A(t) for each
//   of its thresholds t on the graph as it stood when the batch began and
//   keeps the expanded set V_t; (2) p's out-list = JointRobustPrune over the
//   union of its V_t; (3) back-edges v -> p are grouped by target v: v's list
//   gets the new sources in increasing id order, and a list that would
//   exceed R is pruned once over the old list plus the new sources.
// Thresholds: per point p, S = min(sample, n-1) points drawn uniformly (with
// replacement) from the others by SplitMix64 on counter (p << 20) | i; the
// threshold for percentile q is the sorted sample's element floor(q(S-1)/100)
// of dist_A(a_p, .) (implementation-details appendix).
// Pruning: for each threshold t in order, candidates ranked by
// (capped dist_A, distance, id); v joins the bucket if it was chosen for an
// earlier threshold, else if alpha^2 d(u,v) > d(p,v) (fp32 product) for every
// member u so far; a bucket stops at 0.9 R / |T| members; the out-list is the
// union of the buckets in the order first chosen.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <vector>

#include "launch.h"
#include "search_core.cuh"

namespace jag {

constexpr int kPruneWarps = 2;

__device__ __forceinline__ uint64_t sm64(uint64_t seed, uint64_t ctr) {
  uint64_t z = seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ int64_t order_id(int64_t k, int64_t entry) {
  if (k == 0) return entry;
  const int64_t j = k - 1;
  return j < entry ? j : j + 1;
}

// Warp bitonic sort of M (power of two) (key, id) pairs in shared memory.
__device__ void warp_sort_smem(uint64_t *key, uint32_t *id, int M) {
  const int lane = threadIdx.x & 31;
  for (int k = 2; k <= M; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < M; i += 32) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          const uint64_t a = key[i], b = key[l];
          const uint32_t ai = id[i], bi = id[l];
          const bool gt = key_less(b, bi, a, ai);
          if (gt == up) { key[i] = b; key[l] = a; id[i] = bi; id[l] = ai; }
        }
      }
      __syncwarp();
    }
  }
}

__device__ void warp_sort_u32(uint32_t *v, int M) {
  const int lane = threadIdx.x & 31;
  for (int k = 2; k <= M; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < M; i += 32) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          const uint32_t a = v[i], b = v[l];
          if ((a > b) == up) { v[i] = b; v[l] = a; }
        }
      }
      __syncwarp();
    }
  }
}

__host__ __device__ inline int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// ---------------------------------------------------------------------------
// thresholds and entry vertex
// ---------------------------------------------------------------------------

constexpr int kThrWarps = 8;
constexpr int kMaxSample = 1024;

struct Pct { int32_t v[4]; };

__global__ void __launch_bounds__(kThrWarps * 32)
thresholds_kernel(DevIndex ix, int S, uint64_t seed, int nT, Pct pct, uint32_t *thr) {
  __shared__ uint32_t buf[kThrWarps][kMaxSample];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t *b = buf[warp];
  const int64_t Ss = ix.n - 1 < S ? ix.n - 1 : S;
  const int M = next_pow2((int)(Ss > 0 ? Ss : 1));
  for (int64_t p = (int64_t)blockIdx.x * kThrWarps + warp; p < ix.n; p += (int64_t)gridDim.x * kThrWarps) {
    for (int i = lane; i < M; i += 32) {
      uint32_t v = 0xFFFFFFFFu;
      if (i < Ss) {
        const uint64_t r = sm64(seed, ((uint64_t)p << 20) | (uint64_t)i) % (uint64_t)(ix.n - 1);
        const int64_t o = (int64_t)r < p ? (int64_t)r : (int64_t)r + 1;
        v = attribute_distance(ix, p, o);
      }
      b[i] = v;
    }
    __syncwarp();
    warp_sort_u32(b, M);
    if (lane < nT) thr[p * nT + lane] = Ss > 0 ? b[(int64_t)pct.v[lane] * (Ss - 1) / 100] : 0u;
    __syncwarp();
  }
}

// Weight-JAG weights (implementation-details appendix): over the threshold
// sample of S points v, h = sigma / sigma_A with sigma the population standard
// deviation of dist(x_p, x_v) (canonical fp32 distances) and sigma_A that of
// dist_A(a_p, a_v) as a real number; sums in fp64, in sample order, by one
// lane (the order fixes the rounding); h = 0 if sigma_A = 0.  The weights
// of p are w_i = fp32(c_i h).
struct Mult { double v[8]; };
constexpr int kWgtWarps = 4;

template <int P, int CPL>
__global__ void __launch_bounds__(kWgtWarps * 32)
weights_kernel(DevIndex ix, int S, uint64_t seed, int nW, Mult mult, uint32_t *wout) {
  __shared__ float sa[kWgtWarps][kMaxSample], sd[kWgtWarps][kMaxSample];
  __shared__ uint32_t sid[kWgtWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t Ss = ix.n - 1 < S ? ix.n - 1 : S;
  for (int64_t p = (int64_t)blockIdx.x * kWgtWarps + warp; p < ix.n; p += (int64_t)gridDim.x * kWgtWarps) {
    QChunks<CPL, JAG_VEC_F32> q;
    load_point<P, CPL>(ix.x + p * ix.xs, (int)ix.xs, q);
    for (int64_t i0 = 0; i0 < Ss; i0 += 32) {
      const int nc = (int)min64(32, Ss - i0);
      if (lane < nc) {
        const int64_t i = i0 + lane;
        const uint64_t r = sm64(seed, ((uint64_t)p << 20) | (uint64_t)i) % (uint64_t)(ix.n - 1);
        const int64_t o = (int64_t)r < p ? (int64_t)r : (int64_t)r + 1;
        sid[warp][lane] = (uint32_t)o;
        const uint32_t da = attribute_distance(ix, p, o);
        sa[warp][i] = ix.dist_a == JAG_F_RANGE_F32 ? u2f(da) : __uint2float_rn(da);
      }
      __syncwarp();
      const float dist = candidate_distances<P, CPL, 4, JAG_VEC_F32, true>(ix, q, sid[warp], nc);
      if (lane < nc) sd[warp][i0 + lane] = dist;
      __syncwarp();
    }
    if (lane == 0) {
      double ma = 0.0, md = 0.0, va = 0.0, vd = 0.0;
      for (int64_t i = 0; i < Ss; ++i) { ma = __dadd_rn(ma, (double)sa[warp][i]); md = __dadd_rn(md, (double)sd[warp][i]); }
      if (Ss > 0) { ma = __ddiv_rn(ma, (double)Ss); md = __ddiv_rn(md, (double)Ss); }
      for (int64_t i = 0; i < Ss; ++i) {
        const double ta = __dsub_rn((double)sa[warp][i], ma), td = __dsub_rn((double)sd[warp][i], md);
        va = __dadd_rn(va, __dmul_rn(ta, ta));
        vd = __dadd_rn(vd, __dmul_rn(td, td));
      }
      if (Ss > 0) { va = __ddiv_rn(va, (double)Ss); vd = __ddiv_rn(vd, (double)Ss); }
      const double s_a = __dsqrt_rn(va), s_d = __dsqrt_rn(vd);
      const double h = s_a > 0.0 ? __ddiv_rn(s_d, s_a) : 0.0;
      for (int j = 0; j < nW; ++j) wout[p * nW + j] = f2u(__double2float_rn(__dmul_rn(mult.v[j], h)));
    }
    __syncwarp();
  }
}

// Column sums in index order (fp64), one thread per coordinate.
__global__ void centroid_kernel(DevIndex ix, double *c) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ix.d) return;
  double s = 0.0;
  int64_t i = 0;
  for (; i + 8 <= ix.n; i += 8) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = ix.x[(i + u) * ix.xs + j];
#pragma unroll
    for (int u = 0; u < 8; ++u) s = __dadd_rn(s, (double)v[u]);
  }
  for (; i < ix.n; ++i) s = __dadd_rn(s, (double)ix.x[i * ix.xs + j]);
  c[j] = __ddiv_rn(s, (double)ix.n);
}

__global__ void medoid_kernel(DevIndex ix, const double *c, unsigned long long *best, int pass) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ix.n) return;
  double s = 0.0;
  for (int j = 0; j < ix.d; ++j) {
    const double t = __dsub_rn((double)ix.x[i * ix.xs + j], c[j]);
    s = __dadd_rn(s, __dmul_rn(t, t));
  }
  const unsigned long long bits = (unsigned long long)__double_as_longlong(s);
  if (pass == 0) atomicMin(&best[0], bits);
  else if (bits == best[0]) atomicMin(&best[1], (unsigned long long)i);
}

// ---------------------------------------------------------------------------
// batch searches with D_A(t)
// ---------------------------------------------------------------------------

template <int CAP, int P, int CPL>
__global__ void __launch_bounds__(kSearchWarps * 32)
build_search_kernel(DevIndex ix, int64_t pos0, int64_t nb, int nT, const uint32_t *thr, int weighted, int lb,
                    int hbits, uint32_t *vis_ids, float *vis_d, int32_t *vis_n, int vcap, unsigned long long *work,
                    uint32_t *status) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const WarpSmem S = carve_warp_smem(smem + warp * warp_smem_bytes(CAP, hbits), CAP, hbits);
  const unsigned long long total = (unsigned long long)nb * nT;
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(work, 1ull);
    it = __shfl_sync(kFull, it, 0);
    if (it >= total) return;
    const int64_t bi = (int64_t)(it / nT);
    const int ti = (int)(it % nT);
    const int64_t p = order_id(pos0 + bi, ix.entry);
    QChunks<CPL, JAG_VEC_F32> q;
    load_point<P, CPL>(ix.x + p * ix.xs, (int)ix.xs, q);
    VisitSink sink{vis_ids + it * vcap, vis_d + it * vcap, vcap, 0};
    SearchStats st;
    if (weighted) {
      const WeightKey key{p, u2f(thr[p * nT + ti])};
      greedy_search<CAP, P, CPL, JAG_VEC_F32>(ix, key, q, lb, hbits, S, sink, st);
    } else {
      const BuildKey key{p, thr[p * nT + ti]};
      greedy_search<CAP, P, CPL, JAG_VEC_F32>(ix, key, q, lb, hbits, S, sink, st);
    }
    if (lane == 0) {
      vis_n[it] = sink.n;
      if (sink.n > vcap) atomicOr(status, kErrVisitedOverflow);
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// JointRobustPrune
// ---------------------------------------------------------------------------

// Candidate arrays of one prune: a slice of shared memory, or a per-warp
// region of global scratch when the candidate set is larger than the slice.
struct PruneSmem {
  uint32_t *cid;     // [cmax] candidate ids
  float *cdist;      // [cmax] d(p, candidate)
  uint64_t *skey;    // [cmax] sort keys
  uint32_t *sid;     // [cmax]
  uint32_t *bucket;  // [64] (always shared)
  uint32_t *chosen;  // [64]
  uint32_t *tmp;     // [64]
};

__host__ __device__ inline size_t cand_bytes(int cmax) { return (size_t)cmax * (4 + 4 + 8 + 4); }

__host__ __device__ inline size_t prune_smem_bytes(int cmax) { return cand_bytes(cmax) + 64 * 4 * 3; }

__device__ inline void carve_cands(uint8_t *base, int cmax, PruneSmem &s) {
  s.skey = reinterpret_cast<uint64_t *>(base);
  s.cid = reinterpret_cast<uint32_t *>(base + (size_t)cmax * 8);
  s.cdist = reinterpret_cast<float *>(s.cid + cmax);
  s.sid = reinterpret_cast<uint32_t *>(s.cdist + cmax);
}

__device__ inline PruneSmem carve_prune(uint8_t *base, int cmax) {
  PruneSmem s;
  carve_cands(base, cmax, s);
  s.bucket = s.sid + cmax;
  s.chosen = s.bucket + 64;
  s.tmp = s.chosen + 64;
  return s;
}

// The same small arrays, candidate arrays moved to global scratch.
__device__ inline PruneSmem spill_prune(const PruneSmem &sm, uint8_t *gbase, int cmax_g) {
  PruneSmem s = sm;
  carve_cands(gbase, cmax_g, s);
  return s;
}

__device__ __forceinline__ bool in_list(const uint32_t *list, int n, uint32_t v) {
  const int lane = threadIdx.x & 31;
  bool hit = false;
  for (int i = lane; i < n; i += 32) hit |= (list[i] == v);
  return __any_sync(kFull, hit);
}

// JointRobustPrune for base point p over candidates S.cid/S.cdist[0..nc).
// Writes the new out-list (-1 padded) to row.
//
// Weight-JAG (weighted != 0): T holds fp32 weights w and the ranking is by
// D_A^w(p, v) = fma(w, dist_A, dist(p, v)), then id.  The candidates are first
// put in id order, so that a candidate's index breaks ties like its id, and
// the ranking sorts indices; dist(p, v) for the alpha test comes from cdist.
template <int P, int CPL>
__device__ void joint_prune(const DevIndex &ix, int64_t p, const PruneSmem &S, int nc, int cmax,
                            const uint32_t *T, int nT, float alpha2, int weighted, int32_t *row) {
  const int lane = threadIdx.x & 31;
  const int R = ix.R;
  const int M = next_pow2(nc > 0 ? nc : 1);
  int nchosen = 0;
  if (weighted) {
    for (int i = lane; i < M; i += 32) {
      S.skey[i] = i < nc ? (uint64_t)S.cid[i] : kNoKey;
      S.sid[i] = i < nc ? f2u(S.cdist[i]) : kEmptySlot;
    }
    __syncwarp();
    warp_sort_smem(S.skey, S.sid, M);
    for (int i = lane; i < nc; i += 32) { S.cid[i] = (uint32_t)S.skey[i]; S.cdist[i] = u2f(S.sid[i]); }
    __syncwarp();
  }
  for (int ti = 0; ti < nT; ++ti) {
    const uint32_t t = T[ti];
    for (int i = lane; i < M; i += 32) {
      if (i < nc) {
        const uint32_t c = S.cid[i];
        if (weighted) {
          const uint32_t da = attribute_distance(ix, p, c);
          const float a = ix.dist_a == JAG_F_RANGE_F32 ? u2f(da) : __uint2float_rn(da);
          S.skey[i] = make_key(0u, __fmaf_rn(u2f(t), a, S.cdist[i]));
          S.sid[i] = (uint32_t)i;
        } else {
          S.skey[i] = make_key(capped_distance(ix.dist_a, attribute_distance(ix, p, c), t), S.cdist[i]);
          S.sid[i] = c;
        }
      } else {
        S.skey[i] = kNoKey;
        S.sid[i] = kEmptySlot;
      }
    }
    __syncwarp();
    warp_sort_smem(S.skey, S.sid, M);
    int nb = 0;
    for (int i = 0; i < nc; ++i) {
      const uint32_t v = weighted ? S.cid[S.sid[i]] : S.sid[i];
      const float dpv = weighted ? S.cdist[S.sid[i]] : u2f((uint32_t)S.skey[i]);
      bool keep = true;
      if (!in_list(S.chosen, nchosen, v) && nb > 0) {
        QChunks<CPL, JAG_VEC_F32> xv;
        load_point<P, CPL>(ix.x + (int64_t)v * ix.xs, (int)ix.xs, xv);
        for (int b0 = 0; b0 < nb && keep; b0 += 32) {
          const int m = min(32, nb - b0);
          const float duv = candidate_distances<P, CPL, 4, JAG_VEC_F32, true>(ix, xv, S.bucket + b0, m);
          const bool bad = lane < m && !(__fmul_rn(alpha2, duv) > dpv);
          if (__any_sync(kFull, bad)) keep = false;
        }
      }
      if (keep) {
        if (lane == 0) S.bucket[nb] = v;
        ++nb;
        __syncwarp();
      }
      if ((int64_t)nb * nT * 10 >= (int64_t)9 * R) break;
    }
    for (int j = 0; j < nb; ++j) {
      const uint32_t v = S.bucket[j];
      if (!in_list(S.chosen, nchosen, v)) {
        if (lane == 0) S.chosen[nchosen] = v;
        ++nchosen;
        __syncwarp();
      }
    }
  }
  const int m = nchosen < R ? nchosen : R;
  for (int r = lane; r < R; r += 32) row[r] = r < m ? (int32_t)S.chosen[r] : -1;
  __syncwarp();
}

// Union of a batch point's visited sets (deduplicated), then its new
// out-list; emits its back-edges.
template <int P, int CPL>
__global__ void __launch_bounds__(kPruneWarps * 32)
prune_insert_kernel(DevIndex ix, int32_t *graph, int64_t pos0, int64_t nb, int nT, const uint32_t *thr,
                    int weighted, float alpha2, const uint32_t *vis_ids, const float *vis_d, const int32_t *vis_n,
                    int vcap,
                    int cmax_s, int cmax_g, uint8_t *gscratch, int32_t *etgt, int32_t *esrc, uint32_t *status) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const PruneSmem Ss = carve_prune(smem + warp * prune_smem_bytes(cmax_s), cmax_s);
  const int64_t gw = (int64_t)blockIdx.x * kPruneWarps + warp;
  const PruneSmem Sg = spill_prune(Ss, gscratch + gw * cand_bytes(cmax_g), cmax_g);
  for (int64_t bi = gw; bi < nb; bi += (int64_t)gridDim.x * kPruneWarps) {
    const int64_t p = order_id(pos0 + bi, ix.entry);
    int total = 0;
    for (int ti = 0; ti < nT; ++ti) total += min(vis_n[bi * nT + ti], vcap);
    const PruneSmem &S = total <= cmax_s ? Ss : Sg;
    const int cmax = total <= cmax_s ? cmax_s : cmax_g;
    int nc = 0;
    for (int ti = 0; ti < nT; ++ti) {
      const int64_t it = bi * nT + ti;
      const int m = min(vis_n[it], vcap);
      for (int i = lane; i < m; i += 32) {
        // Weight-JAG lists hold D_A^w, not dist: sort by id only, recompute dist below
        S.skey[nc + i] = weighted ? (uint64_t)vis_ids[it * vcap + i] : make_key(0u, vis_d[it * vcap + i]);
        S.sid[nc + i] = vis_ids[it * vcap + i];
      }
      nc += m;
    }
    const int M = next_pow2(nc > 0 ? nc : 1);
    for (int i = nc + lane; i < M; i += 32) { S.skey[i] = kNoKey; S.sid[i] = kEmptySlot; }
    __syncwarp();
    warp_sort_smem(S.skey, S.sid, M);
    // drop repeats (equal id means equal distance: adjacent after the sort)
    int w = 0;
    for (int b = 0; b < nc; b += 32) {
      const int i = b + lane;
      uint64_t k = kNoKey;
      uint32_t id = kEmptySlot;
      bool keep = false;
      if (i < nc) {
        k = S.skey[i];
        id = S.sid[i];
        keep = (i == 0) || (S.sid[i - 1] != id);
      }
      const uint32_t m = __ballot_sync(kFull, keep);
      __syncwarp();
      if (keep) {
        const int pos = w + __popc(m & lanemask_lt());
        S.cid[pos] = id;
        S.cdist[pos] = u2f((uint32_t)k);
      }
      w += __popc(m);
    }
    __syncwarp();
    if (weighted) {
      QChunks<CPL, JAG_VEC_F32> xp;
      load_point<P, CPL>(ix.x + p * ix.xs, (int)ix.xs, xp);
      for (int b = 0; b < w; b += 32) {
        const int m = min(32, w - b);
        const float dv = candidate_distances<P, CPL, 4, JAG_VEC_F32, true>(ix, xp, S.cid + b, m);
        if (lane < m) S.cdist[b + lane] = dv;
      }
      __syncwarp();
    }
    int32_t *row = graph + p * ix.R;
    joint_prune<P, CPL>(ix, p, S, w, cmax, thr + p * nT, nT, alpha2, weighted, row);
    for (int r = lane; r < ix.R; r += 32) {
      const int32_t v = row[r];
      etgt[bi * ix.R + r] = v;
      esrc[bi * ix.R + r] = v >= 0 ? (int32_t)p : -1;
    }
    __syncwarp();
  }
}

// Back-edges: count per target, reserve, scatter, apply.
struct EdgeState {
  int32_t *tcount, *tfill;   // [n], zero between batches
  int64_t *toff;             // [n]
  int32_t *tlist;            // [nb*R]
  int32_t *srcbuf;           // [nb*R]
  unsigned long long *ctr;   // [0] targets, [1] cursor, [2] work
};

__global__ void edge_count_kernel(const int32_t *etgt, int64_t ne, EdgeState E) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const int32_t v = etgt[e];
  if (v < 0) return;
  if (atomicAdd(&E.tcount[v], 1) == 0) {
    const unsigned long long i = atomicAdd(&E.ctr[0], 1ull);
    E.tlist[i] = v;
  }
}

// Largest number of new back-edges of one target in the batch (ctr[3]).
__global__ void edge_max_kernel(int64_t cap, EdgeState E) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap || (unsigned long long)i >= E.ctr[0]) return;
  atomicMax(&E.ctr[3], (unsigned long long)E.tcount[E.tlist[i]]);
}

__global__ void edge_offset_kernel(int64_t cap, EdgeState E) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap || (unsigned long long)i >= E.ctr[0]) return;
  const int32_t v = E.tlist[i];
  E.toff[v] = (int64_t)atomicAdd(&E.ctr[1], (unsigned long long)E.tcount[v]);
}

__global__ void edge_scatter_kernel(const int32_t *etgt, const int32_t *esrc, int64_t ne, EdgeState E) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const int32_t v = etgt[e];
  if (v < 0) return;
  const int32_t slot = atomicAdd(&E.tfill[v], 1);
  E.srcbuf[E.toff[v] + slot] = esrc[e];
}

template <int P, int CPL>
__global__ void __launch_bounds__(kPruneWarps * 32)
edge_apply_kernel(DevIndex ix, int32_t *graph, int64_t cap_targets, int nT, const uint32_t *thr, int weighted,
                  float alpha2, int cmax_s, int cmax_g, uint8_t *gscratch, EdgeState E, uint32_t *status) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const PruneSmem Ss = carve_prune(smem + warp * prune_smem_bytes(cmax_s), cmax_s);
  const int64_t gw = (int64_t)blockIdx.x * kPruneWarps + warp;
  const PruneSmem Sg = spill_prune(Ss, gscratch + gw * cand_bytes(cmax_g), cmax_g);
  for (int64_t i = gw; i < cap_targets; i += (int64_t)gridDim.x * kPruneWarps) {
    if ((unsigned long long)i >= E.ctr[0]) return;
    const int32_t v = E.tlist[i];
    const int ns = E.tcount[v];
    const int32_t *src = E.srcbuf + E.toff[v];
    int32_t *row = graph + (int64_t)v * ix.R;
    int deg = 0;
    for (int r = lane; r < ix.R; r += 32) deg += row[r] >= 0 ? 1 : 0;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) deg += __shfl_xor_sync(kFull, deg, o);
    const PruneSmem &S = deg + ns <= cmax_s ? Ss : Sg;
    const int cmax = deg + ns <= cmax_s ? cmax_s : cmax_g;
    if (deg + ns > cmax_g) {
      if (lane == 0) atomicOr(status, kErrCandOverflow);
    } else if (deg + ns <= ix.R) {
      // append the new sources in increasing id order
      const int M = next_pow2(ns);
      for (int j = lane; j < M; j += 32) S.tmp[j] = j < ns ? (uint32_t)src[j] : 0xFFFFFFFFu;
      __syncwarp();
      warp_sort_u32(S.tmp, M);
      for (int j = lane; j < ns; j += 32) row[deg + j] = (int32_t)S.tmp[j];
    } else {
      const int nc = deg + ns;
      for (int j = lane; j < nc; j += 32) S.cid[j] = j < deg ? (uint32_t)row[j] : (uint32_t)src[j - deg];
      __syncwarp();
      QChunks<CPL, JAG_VEC_F32> xv;
      load_point<P, CPL>(ix.x + (int64_t)v * ix.xs, (int)ix.xs, xv);
      for (int b = 0; b < nc; b += 32) {
        const int m = min(32, nc - b);
        const float dv = candidate_distances<P, CPL, 4, JAG_VEC_F32, true>(ix, xv, S.cid + b, m);
        if (lane < m) S.cdist[b + lane] = dv;
      }
      __syncwarp();
      joint_prune<P, CPL>(ix, v, S, nc, cmax, thr + (int64_t)v * nT, nT, alpha2, weighted, row);
    }
    __syncwarp();
    if (lane == 0) { E.tcount[v] = 0; E.tfill[v] = 0; }
  }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------

static int dev_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

struct BuildScratch {
  uint32_t *vis_ids = nullptr;
  float *vis_d = nullptr;
  int32_t *vis_n = nullptr;
  int32_t *etgt = nullptr, *esrc = nullptr;
  EdgeState E{};
  unsigned long long *work = nullptr;
  uint32_t *status = nullptr;
  double *centroid = nullptr;
  unsigned long long *best = nullptr;
  uint8_t *gscratch = nullptr;   // per-warp candidate arrays of large prunes
  int64_t prune_blocks = 0;
  uint8_t *big = nullptr;        // per-warp arrays for a batch whose hub targets need more
  size_t big_bytes = 0;
  void *blocks[24] = {};
  int nblocks = 0;
};

static cudaError_t balloc(BuildScratch &s, void **p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes < 256 ? 256 : bytes);
  if (e == cudaSuccess) s.blocks[s.nblocks++] = *p;
  return e;
}

static void bfree(BuildScratch &s) {
  for (int i = 0; i < s.nblocks; ++i) cudaFree(s.blocks[i]);
  s.nblocks = 0;
  if (s.big) cudaFree(s.big);
  s.big = nullptr;
  s.big_bytes = 0;
}

// Budget of the per-warp candidate arrays of oversized back-edge prunes.
constexpr size_t kBigScratchBytes = size_t(1) << 30;

template <int CAP, int P, int CPL>
static cudaError_t launch_build_search(const BuildLaunch &B, int64_t pos0, int64_t nb, int hbits, BuildScratch &s,
                                       int vcap) {
  const size_t smem = (size_t)kSearchWarps * warp_smem_bytes(CAP, hbits);
  auto kern = build_search_kernel<CAP, P, CPL>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int bps = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kSearchWarps * 32, smem);
  if (bps <= 0) return cudaErrorInvalidConfiguration;
  const int64_t items = nb * B.nT;
  const int64_t grid = std::min<int64_t>((int64_t)bps * dev_sms(), (items + kSearchWarps - 1) / kSearchWarps);
  kern<<<(unsigned)grid, kSearchWarps * 32, smem, B.stream>>>(B.ix, pos0, nb, B.nT, B.thr, B.weighted, B.lb, hbits,
                                                             s.vis_ids, s.vis_d, s.vis_n, vcap, s.work, s.status);
  return cudaGetLastError();
}

template <int P, int CPL>
static cudaError_t launch_prunes(const BuildLaunch &B, int64_t pos0, int64_t nb, BuildScratch &s, int vcap,
                                 int cmax_s, int cmax_g) {
  const size_t smem = (size_t)kPruneWarps * prune_smem_bytes(cmax_s);
  auto pk = prune_insert_kernel<P, CPL>;
  cudaFuncSetAttribute(pk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int64_t pgrid = std::min<int64_t>((nb + kPruneWarps - 1) / kPruneWarps, s.prune_blocks);
  pk<<<(unsigned)std::max<int64_t>(pgrid, 1), kPruneWarps * 32, smem, B.stream>>>(
      B.ix, B.graph, pos0, nb, B.nT, B.thr, B.weighted, B.alpha2, s.vis_ids, s.vis_d, s.vis_n, vcap, cmax_s, cmax_g,
      s.gscratch, s.etgt, s.esrc, s.status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t ne = nb * B.ix.R;
  const unsigned eb = (unsigned)((ne + 255) / 256);
  edge_count_kernel<<<eb, 256, 0, B.stream>>>(s.etgt, ne, s.E);
  // A hub can receive more back-edges in one batch than the fixed per-warp
  // arrays hold.  Size this batch's arrays from its largest target: fewer
  // warps, each with room for a whole candidate set.
  edge_max_kernel<<<eb, 256, 0, B.stream>>>(ne, s.E);
  unsigned long long most = 0;
  if ((e = cudaMemcpyAsync(&most, s.E.ctr + 3, sizeof(most), cudaMemcpyDeviceToHost, B.stream)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(B.stream)) != cudaSuccess) return e;
  uint8_t *scratch = s.gscratch;
  int cmax = cmax_g;
  int64_t agrid = std::min<int64_t>((ne + kPruneWarps - 1) / kPruneWarps, s.prune_blocks);
  if ((int64_t)most + B.ix.R > cmax_g) {
    cmax = next_pow2((int)most + B.ix.R);
    const size_t per = cand_bytes(cmax);
    const int64_t warps = std::max<int64_t>(
        kPruneWarps, std::min<int64_t>(s.prune_blocks * kPruneWarps, (int64_t)(kBigScratchBytes / per)));
    agrid = std::max<int64_t>(1, std::min<int64_t>(agrid, warps / kPruneWarps));
    const size_t need = per * (size_t)agrid * kPruneWarps;
    if (s.big_bytes < need) {
      if (s.big) cudaFree(s.big);
      s.big = nullptr;
      s.big_bytes = 0;
      if ((e = cudaMalloc((void **)&s.big, need)) != cudaSuccess) return e;
      s.big_bytes = need;
    }
    scratch = s.big;
  }
  edge_offset_kernel<<<eb, 256, 0, B.stream>>>(ne, s.E);
  edge_scatter_kernel<<<eb, 256, 0, B.stream>>>(s.etgt, s.esrc, ne, s.E);
  auto ak = edge_apply_kernel<P, CPL>;
  cudaFuncSetAttribute(ak, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  ak<<<(unsigned)std::max<int64_t>(agrid, 1), kPruneWarps * 32, smem, B.stream>>>(
      B.ix, B.graph, ne, B.nT, B.thr, B.weighted, B.alpha2, cmax_s, cmax, scratch, s.E, s.status);
  return cudaGetLastError();
}

static cudaError_t launch_weights(const BuildLaunch &B, const Mult &mult, int64_t blocks) {
  int P, CPL;
  if (!row_mapping(B.ix.nchunks, &P, &CPL)) return cudaErrorInvalidValue;
#define JAG_WCASE(PP, CC)                                                                                      \
  if (P == PP && CPL == CC) {                                                                                  \
    weights_kernel<PP, CC><<<(unsigned)blocks, kWgtWarps * 32, 0, B.stream>>>(B.ix, B.sample, B.seed, B.nT,   \
                                                                             mult, B.thr);                     \
    return cudaGetLastError();                                                                                 \
  }
  JAG_WCASE(8, 1)
  JAG_WCASE(16, 1)
  JAG_WCASE(32, 1)
  JAG_WCASE(32, 2)
  JAG_WCASE(32, 4)
  JAG_WCASE(32, 8)
#undef JAG_WCASE
  return cudaErrorInvalidValue;
}

template <int CAP>
static cudaError_t dispatch_build(const BuildLaunch &B, int P, int CPL, int64_t pos0, int64_t nb, int hbits,
                                  BuildScratch &s, int vcap, int cmax_s, int cmax_g) {
  cudaError_t e = cudaErrorInvalidValue;
#define JAG_BCASE(PP, CC)                                                   \
  if (P == PP && CPL == CC) {                                               \
    e = launch_build_search<CAP, PP, CC>(B, pos0, nb, hbits, s, vcap);      \
    if (e == cudaSuccess) e = launch_prunes<PP, CC>(B, pos0, nb, s, vcap, cmax_s, cmax_g); \
    return e;                                                               \
  }
  JAG_BCASE(8, 1)
  JAG_BCASE(16, 1)
  JAG_BCASE(32, 1)
  JAG_BCASE(32, 2)
  JAG_BCASE(32, 4)
  JAG_BCASE(32, 8)
#undef JAG_BCASE
  return e;
}

int run_build(BuildLaunch &B, int32_t *entry_out, char *msg, size_t msg_len) {
  const int64_t n = B.ix.n;
  const int R = B.ix.R;
  int P, CPL;
  if (!row_mapping(B.ix.nchunks, &P, &CPL)) { snprintf(msg, msg_len, "dimension too large"); return JAG_EINVAL; }
  const int cap_list = list_capacity(B.lb);
  if (!cap_list) { snprintf(msg, msg_len, "l_b must be <= 256"); return JAG_EINVAL; }
  BuildScratch s;
  cudaError_t e = cudaSuccess;
  const int64_t bcap = std::max<int64_t>(1, n / 50);
  // visited lists: hop counts are ~l_b plus a few, but a search may expand
  // more; 16 l_b leaves a wide margin and an overflow is reported, not cut
  const int vcap = std::max(1024, 16 * B.lb);
  const int cmax_s = 1024;                                   // shared-memory slice
  const int cmax_g = std::max(8192, next_pow2(B.nT * vcap)); // global spill
  const int blocks_per_sm = (int)std::max<size_t>(1, (227 * 1024) / (kPruneWarps * prune_smem_bytes(cmax_s)));
  s.prune_blocks = (int64_t)blocks_per_sm * dev_sms();
  const int hbits = B.lb <= 64 ? 11 : (B.lb <= 128 ? 12 : 13);
#define JAG_TRY(x) do { e = (x); if (e != cudaSuccess) goto fail; } while (0)
  JAG_TRY(balloc(s, (void **)&s.vis_ids, sizeof(uint32_t) * (size_t)bcap * B.nT * vcap));
  JAG_TRY(balloc(s, (void **)&s.vis_d, sizeof(float) * (size_t)bcap * B.nT * vcap));
  JAG_TRY(balloc(s, (void **)&s.vis_n, sizeof(int32_t) * (size_t)bcap * B.nT));
  JAG_TRY(balloc(s, (void **)&s.etgt, sizeof(int32_t) * (size_t)bcap * R));
  JAG_TRY(balloc(s, (void **)&s.esrc, sizeof(int32_t) * (size_t)bcap * R));
  JAG_TRY(balloc(s, (void **)&s.E.tcount, sizeof(int32_t) * (size_t)n));
  JAG_TRY(balloc(s, (void **)&s.E.tfill, sizeof(int32_t) * (size_t)n));
  JAG_TRY(balloc(s, (void **)&s.E.toff, sizeof(int64_t) * (size_t)n));
  JAG_TRY(balloc(s, (void **)&s.E.tlist, sizeof(int32_t) * (size_t)bcap * R));
  JAG_TRY(balloc(s, (void **)&s.E.srcbuf, sizeof(int32_t) * (size_t)bcap * R));
  JAG_TRY(balloc(s, (void **)&s.E.ctr, 256));
  JAG_TRY(balloc(s, (void **)&s.work, 256));
  JAG_TRY(balloc(s, (void **)&s.status, 256));
  JAG_TRY(balloc(s, (void **)&s.centroid, sizeof(double) * (size_t)B.ix.d));
  JAG_TRY(balloc(s, (void **)&s.best, 256));
  JAG_TRY(balloc(s, (void **)&s.gscratch, cand_bytes(cmax_g) * (size_t)s.prune_blocks * kPruneWarps));
  JAG_TRY(cudaMemsetAsync(s.E.tcount, 0, sizeof(int32_t) * (size_t)n, B.stream));
  JAG_TRY(cudaMemsetAsync(s.E.tfill, 0, sizeof(int32_t) * (size_t)n, B.stream));
  JAG_TRY(cudaMemsetAsync(s.status, 0, 256, B.stream));
  JAG_TRY(cudaMemsetAsync(B.graph, 0xFF, sizeof(int32_t) * (size_t)n * R, B.stream));
  {
    Pct pct;
    for (int i = 0; i < 4; ++i) pct.v[i] = B.pct[i];
    const int64_t blocks = std::min<int64_t>((n + kThrWarps - 1) / kThrWarps, (int64_t)dev_sms() * 8);
    if (B.weighted) {
      Mult mult;
      for (int i = 0; i < 8; ++i) mult.v[i] = B.mult[i];
      const int64_t wb = std::min<int64_t>((n + kWgtWarps - 1) / kWgtWarps, (int64_t)dev_sms() * 16);
      JAG_TRY(launch_weights(B, mult, wb));
    } else {
      thresholds_kernel<<<(unsigned)blocks, kThrWarps * 32, 0, B.stream>>>(B.ix, B.sample, B.seed, B.nT, pct, B.thr);
    }
    JAG_TRY(cudaGetLastError());
    centroid_kernel<<<(B.ix.d + 127) / 128, 128, 0, B.stream>>>(B.ix, s.centroid);
    JAG_TRY(cudaMemsetAsync(s.best, 0xFF, 16, B.stream));
    medoid_kernel<<<(unsigned)((n + 255) / 256), 256, 0, B.stream>>>(B.ix, s.centroid, s.best, 0);
    medoid_kernel<<<(unsigned)((n + 255) / 256), 256, 0, B.stream>>>(B.ix, s.centroid, s.best, 1);
    JAG_TRY(cudaGetLastError());
    unsigned long long best[2];
    JAG_TRY(cudaMemcpyAsync(best, s.best, 16, cudaMemcpyDeviceToHost, B.stream));
    JAG_TRY(cudaStreamSynchronize(B.stream));
    B.ix.entry = (int32_t)best[1];
    *entry_out = B.ix.entry;
  }
  {
    int64_t pos = 1, inserted = 1;
    while (pos < n) {
      int64_t nb = std::min<int64_t>(inserted, bcap);
      nb = std::min<int64_t>(nb, n - pos);
      JAG_TRY(cudaMemsetAsync(s.work, 0, 256, B.stream));
      JAG_TRY(cudaMemsetAsync(s.E.ctr, 0, 256, B.stream));
      switch (cap_list) {
        case 64: e = dispatch_build<64>(B, P, CPL, pos, nb, hbits, s, vcap, cmax_s, cmax_g); break;
        case 128: e = dispatch_build<128>(B, P, CPL, pos, nb, hbits, s, vcap, cmax_s, cmax_g); break;
        default: e = dispatch_build<256>(B, P, CPL, pos, nb, hbits, s, vcap, cmax_s, cmax_g); break;
      }
      if (e != cudaSuccess) goto fail;
      pos += nb;
      inserted += nb;
    }
    uint32_t status = 0;
    JAG_TRY(cudaMemcpyAsync(&status, s.status, 4, cudaMemcpyDeviceToHost, B.stream));
    JAG_TRY(cudaStreamSynchronize(B.stream));
    bfree(s);
    if (status & kErrVisitedOverflow) {
      snprintf(msg, msg_len, "build search visited more than %d vertices", vcap);
      return JAG_EUNSUPPORTED;
    }
    if (status & kErrCandOverflow) {
      snprintf(msg, msg_len, "back-edge candidates exceeded %d", cmax_g);
      return JAG_EUNSUPPORTED;
    }
    return JAG_OK;
  }
fail:
  cudaStreamSynchronize(B.stream);
  bfree(s);
  snprintf(msg, msg_len, "CUDA error in build: %s", cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? JAG_ENOMEM : JAG_ECUDA;
#undef JAG_TRY
}

}  // namespace jag
