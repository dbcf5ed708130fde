// GreedySearch (Algorithm 1 of the paper) executed by one warp.
//
// One warp owns one search.  Its candidate list L (at most l_s entries,
// sorted by (first key, distance, id)) and a hashed visited set live in the
// warp's slice of shared memory; nothing else is kept per search.  Each hop:
//   select   the first unexpanded entry p of L (ballot over 32 entries);
//   fetch    p's out-list: one coalesced 4-byte load per lane (128 B at R=32);
//   dedupe   each lane tests/inserts its neighbour in the visited set
//            (shared-memory open addressing on full ids, atomicCAS);
//   filter   first key (dist_F or capped dist_A) from the neighbour's
//            attribute; a key above a full list's last entry is dropped
//            without touching its vector (exact: that entry's key only
//            decreases, so the neighbour could never be kept);
//   gather   survivors' rows as 16-byte chunks, P lanes per row, 32/P rows
//            per warp-wide load, several loads in flight;
//   reduce   squared L2 in the fixed order: chunk g -> lane g mod 32,
//            elements of a chunk in order by fma, then the butterfly
//            acc_l + acc_(l xor o) for o = 16..1 (groups of P < 32 lanes only
//            skip steps that would add exact zeros);
//   merge    each surviving neighbour's position in the merged list is its
//            rank in L (a fixed-step binary search on the keys, ties by id)
//            plus the number of smaller new keys; L is rebuilt from the back,
//            32 positions at a time, each lane fetching the entry that lands
//            on its position; the best l_s are kept and a neighbour already
//            in L (equal key and id) is dropped;
// until every entry of L is expanded.
//
// The visited set may forget (a new id replaces the first of its two probe
// slots when both hold other ids): that only costs recomputation, because an
// id still in L is caught by the merge (same key, same id) and an id that
// left L can never re-enter it.
#pragma once

#include "jag_internal.cuh"

namespace jag {

// Whether the graph search asks L2 for the rows of a hop's candidates past
// its first batch of loads before it starts the batches (the exact scans,
// re-ranks and the build always do: their batches hold up to 32 rows).  Requesting the
// out-list of the likely next vertex (the second unexpanded entry of L) was
// measured slower for every format.
__host__ __device__ constexpr bool prefetch_rows(int FMT) { return FMT != JAG_VEC_FP8; }
constexpr int kSearchWarps = 4;   // warps (searches) per CTA of the search kernels (the graph kernel: graph_warps)

// Shared-memory slice of one warp.
struct WarpSmem {
  uint64_t *bkey;   // [cap] keys of L
  uint32_t *bid;    // [cap] ids of L, bit 31 = expanded
  uint32_t *hash;   // [1 << hbits] visited set
  uint32_t *cid;    // [32] candidate ids of the current hop
  uint32_t *ck1;    // [32] their first keys
  uint32_t *rank;   // [32] scratch (anchors the policy context)
};

// Slots of a warp's list for beam ls: ls rounded up to a multiple of 32.
__host__ __device__ inline int list_slots(int ls) { return (ls + 31) & ~31; }

__host__ __device__ inline size_t warp_smem_bytes(int cap, int hbits) {
  return (size_t)cap * 12 + ((size_t)4 << hbits) + 32 * 4 * 3;
}

__device__ inline WarpSmem carve_warp_smem(uint8_t *base, int cap, int hbits) {
  WarpSmem s;
  s.bkey = reinterpret_cast<uint64_t *>(base);
  s.bid = reinterpret_cast<uint32_t *>(base + (size_t)cap * 8);
  s.hash = reinterpret_cast<uint32_t *>(base + (size_t)cap * 12);
  s.cid = s.hash + (1u << hbits);
  s.ck1 = s.cid + 32;
  s.rank = s.ck1 + 32;
  return s;
}

__device__ __forceinline__ int first_unexpanded(const uint32_t *bid, int cnt, int start) {
  const int lane = threadIdx.x & 31;
  for (int b = start; b < cnt; b += 32) {
    int j = b + lane;
    bool un = (j < cnt) && !(bid[j] & kExpanded);
    uint32_t m = __ballot_sync(kFull, un);
    if (m) return b + __ffs(m) - 1;
  }
  return -1;
}

// Visited-set probe (two slots, linear); returns true if id was not
// recorded.  The set forgets: when both slots hold other ids, id replaces the
// first, so the set keeps mostly recent ids (a slot, once filled, is never
// empty again, so an id stored in the second slot is still found there).  A
// forgotten id only costs a recomputed distance: the list drops a repeat, and
// a vertex that left a full list cannot re-enter it.
__device__ __forceinline__ bool visit_insert(uint32_t *tab, int hbits, uint32_t id) {
  const uint32_t mask = (1u << hbits) - 1;
  const uint32_t h = (id * 0x9E3779B1u) >> (32 - hbits);
  const uint32_t old = atomicCAS(&tab[h], kEmptySlot, id);
  bool fresh = old == kEmptySlot;
  if ((old != kEmptySlot) & (old != id)) {   // the first slot holds another id
    const uint32_t o2 = atomicCAS(&tab[(h + 1) & mask], kEmptySlot, id);
    fresh = o2 != id;
    if ((o2 != kEmptySlot) & (o2 != id)) atomicExch(&tab[h], id);
  }
  return fresh;
}

// Number of entries of the sorted list L[0..cnt) (cnt >= 1) whose 64-bit
// key is below k: a binary search on the keys alone (one shared-memory read
// a step), with a fixed number of steps and no branch, so that every lane
// runs the same instructions.  TOP is the first step: CAP, or CAP / 2 where
// the caller knows k precedes L's last entry when L holds CAP entries.  (A
// 4-way search, three probes a step, halves the chain of dependent reads but
// was measured slower: it issues more instructions.)
template <int TOP>
__device__ __forceinline__ int key_lower_bound(const uint64_t *bkey, int cnt, uint64_t k) {
  int pos = 0;
#pragma unroll
  for (int step = TOP; step >= 1; step >>= 1) {
    const int probe = pos + step;
    const int j = min(probe, cnt) - 1;
    pos = ((probe <= cnt) & (bkey[j] < k)) ? probe : pos;
  }
  return pos;
}

// Merge the lane-held candidates (any order; invalid = kNoKey, distinct ids)
// into L[0..cnt): keep the best ls, drop candidates already in L.  Returns
// the new count; r0 receives the smallest insertion position (cnt if none).
//
// A new key's position in the merged list is its rank in L plus the number
// of smaller new keys.  DEST (the long lists of the graph search): the list
// is rebuilt by destination, 32 positions at a time from the back -- a
// window's new-key positions are one OR-reduction of bits, so each lane
// finds the old entry that lands on its position (its index minus the new
// keys before it) and moves it; reads of a window stay at or below it and
// writes at or above it, so no entry is overwritten before it is read.
// Otherwise (the k-entry lists of the exact scans) an entry's shift is
// counted with one shuffle per new key: smaller code.
template <int CAP, bool DEST = true>
__device__ __forceinline__ int merge_candidates(uint64_t *bkey, uint32_t *bid, int cnt, int ls, uint64_t ck,
                                                uint32_t cv, int &r0) {
  const int lane = threadIdx.x & 31;
  bool valid = ck != kNoKey;
  r0 = cnt;
  if (!__any_sync(kFull, valid)) return cnt;
  // rank in L under (key, id): the entries with a smaller key, then those
  // with an equal key and a smaller id (equal keys are rare: one test).  The
  // graph search drops a key that follows a full list's last entry before
  // the merge, so its ranks stay below CAP.
  int rank = cnt == 0 ? 0 : key_lower_bound<DEST ? CAP / 2 : CAP>(bkey, cnt, ck);
  {
    int rr = min(rank, cnt - 1);
    bool tie = (rank < cnt) & (bkey[rr] == ck) & ((bid[rr] & ~kExpanded) < cv);
    if (__any_sync(kFull, tie)) {
      while (tie) {
        ++rank;
        rr = min(rank, cnt - 1);
        tie = (rank < cnt) & (bkey[rr] == ck) & ((bid[rr] & ~kExpanded) < cv);
      }
    }
    // a key equal to L's entry at its rank, with the same id, is a repeat
    const bool rep = (rank < cnt) & (bkey[rr] == ck) & ((bid[rr] & ~kExpanded) == cv);
    valid = valid & (rank < ls) & !rep;
  }
  const uint32_t vm = __ballot_sync(kFull, valid);
  r0 = cnt;
  if (vm == 0) return cnt;
  int crank = 0;   // new keys smaller than this one
  for (uint32_t m = vm; m; m &= m - 1) {
    const int src = __ffs(m) - 1;
    const uint64_t ok = __shfl_sync(kFull, ck, src);
    const uint32_t oi = __shfl_sync(kFull, cv, src);
    crank += key_less(ok, oi, ck, cv) ? 1 : 0;
  }
  r0 = (int)__reduce_min_sync(kFull, valid ? (unsigned)rank : 0xFFFFFFFFu);
  const int n2 = min(cnt + __popc(vm), ls);
  const int pos = rank + crank;   // distinct over the new keys
  if (DEST) {
    for (int f0 = r0 + ((n2 - 1 - r0) & ~31); f0 >= r0; f0 -= 32) {
      const int f = f0 + lane;
      const uint32_t inw = __reduce_or_sync(kFull, (valid && pos >= f0 && pos < f0 + 32) ? 1u << (pos - f0) : 0u);
      const int below = __popc(__ballot_sync(kFull, valid && pos < f0));
      const bool mv = f < n2 && !((inw >> lane) & 1u);
      uint64_t ek = 0;
      uint32_t ei = 0;
      if (mv) {
        const int j = f - below - __popc(inw & lanemask_lt());
        ek = bkey[j];
        ei = bid[j];
      }
      __syncwarp();
      if (mv) { bkey[f] = ek; bid[f] = ei; }
    }
  } else {
    // entry j moves right by the number of new keys ranked at or before j;
    // chunks from the back never overwrite an entry not yet read
    for (int t = (cnt - r0 + 31) / 32 - 1; t >= 0; --t) {
      const int j = r0 + 32 * t + lane;
      uint64_t ek = 0;
      uint32_t ei = 0;
      if (j < cnt) { ek = bkey[j]; ei = bid[j]; }
      int sh = 0;
      for (uint32_t m = vm; m; m &= m - 1) sh += (__shfl_sync(kFull, rank, __ffs(m) - 1) <= j) ? 1 : 0;
      __syncwarp();
      if (j < cnt && j + sh < ls) { bkey[j + sh] = ek; bid[j + sh] = ei; }
      __syncwarp();
    }
  }
  if (valid && pos < ls) { bkey[pos] = ck; bid[pos] = cv; }
  __syncwarp();
  return n2;
}

// The lane-held chunks of a search point: lane lig of a P-lane group holds
// chunks lig, lig + 32, ... (at most CPL of them), each as E/4 float4.
template <int CPL, int FMT>
struct QChunks {
  float4 v[CPL][RowFmt<FMT>::Q4];
};

// Start and length of stored row id in format FMT.
template <int FMT>
__device__ __forceinline__ const void *row_address(const DevIndex &ix, uint32_t id) {
  return FMT == JAG_VEC_F32 ? static_cast<const void *>(ix.x + (int64_t)id * ix.xs)
                            : static_cast<const void *>(ix.xq + (int64_t)id * ix.qbytes);
}
template <int FMT>
__device__ __forceinline__ int row_bytes(const DevIndex &ix) {
  return FMT == JAG_VEC_F32 ? ix.nchunks * 16 : ix.qbytes;
}

// Distances from the search point (lane-held chunks q) to the nc rows whose
// ids are cid[0..nc), rows stored in format FMT; lane c < nc returns the
// distance of candidate c.
//
// Lane mapping: a row is held by a group of P lanes; lane lig holds chunks
// lig + j*P (j < CPL).  Chunk g belongs to canonical accumulator g mod 32, so
// a lane with P < 32 keeps F = 32/P of the canonical accumulators (chunk j in
// accumulator j mod F, in chunk order) and performs the butterfly levels
// 16..P in registers before the shuffle levels P/2..1: the same additions in
// the same order as the 32-lane canonical reduction (levels that would add
// exact zeros are skipped).
template <int P, int CPL, int ROWS = 4, int FMT = JAG_VEC_F32, bool PREF = false>
__device__ __forceinline__ float candidate_distances(const DevIndex &ix, const QChunks<CPL, FMT> &q,
                                                     const uint32_t *cid, int nc) {
  constexpr int VPW = 32 / P;                        // rows per warp-wide load
  constexpr int U = VPW >= ROWS ? 1 : ROWS / VPW;    // loads in flight per lane (ROWS rows per warp)
  constexpr int F = 32 / P;                          // canonical accumulators per lane
  constexpr int NA = CPL < F ? CPL : F;              // of which can be non-zero
  const int lane = threadIdx.x & 31;
  const int grp = lane / P, lig = lane % P;
  const int nch = FMT == JAG_VEC_F32 ? ix.nchunks : ix.qchunks;
  // rows past the first batch are requested from L2 at once (one lane per
  // row), so that their loads below do not each wait a memory latency
  if (PREF && nc > VPW * U && lane < nc - VPW * U)
    prefetch_l2(row_address<FMT>(ix, cid[VPW * U + lane]), row_bytes<FMT>(ix));
  float mine = 0.f;
  for (int base = 0; base < nc; base += VPW * U) {
    uint4 xv[U][CPL];
    float sc[U];
    // straight-line over the batch's U loads: a row past nc is not read (its
    // chunks are zero) and its sum is never handed out
#pragma unroll
    for (int s = 0; s < U; ++s) {
      const int c = base + s * VPW + grp;
      const bool ok = c < nc;
      const uint32_t id = ok ? cid[c] : 0u;
      const uint8_t *row = FMT == JAG_VEC_F32 ? reinterpret_cast<const uint8_t *>(ix.x + (int64_t)id * ix.xs)
                                              : ix.xq + (int64_t)id * ix.qbytes;
      sc[s] = 1.f;
      if (FMT == JAG_VEC_FP8) sc[s] = ok ? __ldg(ix.qscale + id) : 1.f;
#pragma unroll
      for (int j = 0; j < CPL; ++j) {
        const int ch = lig + j * P;
        xv[s][j] = (ok && ch < nch) ? ld_chunk_u4(row + ch * 16) : make_uint4(0, 0, 0, 0);
      }
    }
    float acc[U];
#pragma unroll
    for (int s = 0; s < U; ++s) {
      float a[NA];
#pragma unroll
      for (int i = 0; i < NA; ++i) a[i] = 0.f;
#pragma unroll
      for (int j = 0; j < CPL; ++j) a[j % F] = chunk_acc<FMT>(a[j % F], q.v[j], xv[s][j], sc[s]);
#pragma unroll
      for (int h = F / 2; h >= 1; h >>= 1) {
#pragma unroll
        for (int i = 0; i < h; ++i)
          if (i + h < NA) a[i] = __fadd_rn(a[i], a[i + h]);
      }
      acc[s] = a[0];
    }
    // candidate base + s*VPW + g is row s of group g
    const float tot = group_reduce_spread<P, U>(acc);
    const int rel = lane - base;
    const bool mine_here = rel >= 0 && rel < VPW * U;
    const float v = __shfl_sync(kFull, tot, mine_here ? spread_source<P, U>(rel / VPW, rel % VPW) : 0);
    if (mine_here) mine = v;
  }
  return mine;
}

// Lane chunks of a search point given as a contiguous fp32 row of d values
// (not necessarily 16-byte aligned); elements past d are zero.  Lane lig of a
// P-lane group holds chunks lig + j*P (the mapping of candidate_distances).
template <int P, int CPL, int FMT = JAG_VEC_F32>
__device__ __forceinline__ void load_point(const float *row, int d, QChunks<CPL, FMT> &q) {
  constexpr int E = RowFmt<FMT>::E;
  const int lig = (threadIdx.x & 31) % P;
#pragma unroll
  for (int j = 0; j < CPL; ++j) {
    const int e0 = (lig + j * P) * E;
#pragma unroll
    for (int i = 0; i < RowFmt<FMT>::Q4; ++i) {
      const int e = e0 + 4 * i;
      q.v[j][i].x = e + 0 < d ? row[e + 0] : 0.f;
      q.v[j][i].y = e + 1 < d ? row[e + 1] : 0.f;
      q.v[j][i].z = e + 2 < d ? row[e + 2] : 0.f;
      q.v[j][i].w = e + 3 < d ? row[e + 3] : 0.f;
    }
  }
}

// First-key policies.  A policy with kEdgeAttr reads the neighbour's
// attribute from the edge table in the same wave as the neighbour id.
// A key policy gives, for candidate u, a 32-bit word (operator()), and the
// 64-bit list key from that word and u's vector distance (key()).  With
// kScalar the key is one number (no first component), so a full list cannot
// reject a candidate before its distance is known.
struct QueryKey {   // dist_F of the query's filter (Sec. 3.1)
  static constexpr bool kEdgeAttr = true;
  static constexpr bool kScalar = false;
  __device__ __forceinline__ uint64_t key(uint32_t w, float dist) const { return make_key(w, dist); }
  int32_t kind;
  uint64_t payload;
  const uint8_t *lut;
  __device__ __forceinline__ uint32_t operator()(const DevIndex &ix, int64_t u) const {
    return filter_distance(ix, u, kind, payload, lut);
  }
  __device__ __forceinline__ uint64_t edge_word(const DevIndex &ix, int64_t e) const {
    return edge_attr(ix, e, kind);
  }
  __device__ __forceinline__ uint32_t from_word(uint64_t raw) const {
    return filter_distance_raw(kind, payload, lut, raw);
  }
};

struct BuildKey {   // capped dist_A from base point p with threshold t (Sec. 3.2)
  static constexpr bool kEdgeAttr = false;   // the graph changes while it is built
  static constexpr bool kScalar = false;
  __device__ __forceinline__ uint64_t key(uint32_t w, float dist) const { return make_key(w, dist); }
  int64_t p;
  uint32_t t;
  __device__ __forceinline__ uint32_t operator()(const DevIndex &ix, int64_t u) const {
    return capped_distance(ix.dist_a, attribute_distance(ix, p, u), t);
  }
  __device__ __forceinline__ uint64_t edge_word(const DevIndex &, int64_t) const { return 0; }
  __device__ __forceinline__ uint32_t from_word(uint64_t) const { return 0; }
};

// Weight-JAG's build comparator D_A^w(p, u) = w dist_A(a_p, a_u) + dist(x_p,
// x_u) (the weighted variant of Sec. 3), one fp32 fma; the word carries
// dist_A as an fp32 value.
struct WeightKey {
  static constexpr bool kEdgeAttr = false;
  static constexpr bool kScalar = true;
  int64_t p;
  float w;
  __device__ __forceinline__ uint32_t operator()(const DevIndex &ix, int64_t u) const {
    const uint32_t da = attribute_distance(ix, p, u);
    return f2u(ix.dist_a == JAG_F_RANGE_F32 ? u2f(da) : __uint2float_rn(da));
  }
  __device__ __forceinline__ uint64_t key(uint32_t w_bits, float dist) const {
    return make_key(0u, __fmaf_rn(w, u2f(w_bits), dist));
  }
  __device__ __forceinline__ uint64_t edge_word(const DevIndex &, int64_t) const { return 0; }
  __device__ __forceinline__ uint32_t from_word(uint64_t) const { return 0; }
};

struct NoSink {
  __device__ __forceinline__ void visit(int, uint32_t, uint64_t) {}
};

// Records the expanded vertices (the set V of Algorithm 1) with their
// distances from the search point.
struct VisitSink {
  uint32_t *ids;
  float *dist;
  int cap;
  int n;
  __device__ __forceinline__ void visit(int lane, uint32_t id, uint64_t key) {
    if (lane == 0 && n < cap) { ids[n] = id; dist[n] = u2f((uint32_t)key); }
    ++n;
  }
};

struct SearchStats {
  int hops, seen, dcs;
};

// ---------------------------------------------------------------------------
// learned beam width and stop hop
// ---------------------------------------------------------------------------

// Monotone stand-in for log2 from the float encoding: (bits >> 16)/128 - 127.
__device__ __forceinline__ float flog_bits(float x) {
  return __fsub_rn(__fmul_rn((float)(f2u(x) >> 16), 0.0078125f), 127.f);
}

__device__ __forceinline__ float bf16_value(uint16_t h) { return u2f((uint32_t)h << 16); }

// Outcome of the policy at the decision hop.
struct PolicyOut {
  int beam, stop, learned;
};

// Features of the list L[0..cnt) after the decision hop and the policy's
// beam / stop (every lane returns the same).  hbuf: 64 floats of the warp.
// Inlined: with the lean search loop the policy kernels fit their register
// budget without a call.
__device__ __forceinline__ static PolicyOut policy_decide(const jag_policy &pol, const WarpSmem &S, float *hbuf,
                                                          int cnt, int k, int64_t est, int32_t kind, int fixed,
                                                          float *feat_out, const int32_t *forced_q) {
  const int lane = threadIdx.x & 31;
  // passing prefix and first unexpanded entry
  int np = cnt;
  for (int b = 0; b < cnt; b += 32) {
    const int j = b + lane;
    const uint32_t m = __ballot_sync(kFull, j < cnt && (S.bkey[j] >> 32) != 0);
    if (m) { np = b + __ffs(m) - 1; break; }
  }
  int fu = first_unexpanded(S.bid, cnt, 0);
  if (fu < 0) fu = cnt;
  const uint32_t e = est > 0x7FFFFFFE ? 0x7FFFFFFFu : (uint32_t)est + 1u;
  const int kk = np < k ? np : k;
  float f[JAG_MLP_FEATURES];
  f[0] = __fmul_rn((float)(32 - __clz(e)), 0.05f);
#pragma unroll
  for (int i = 0; i < 5; ++i) f[1 + i] = (kind == i + 1) ? 1.f : 0.f;
  f[6] = __fdiv_rn((float)np, (float)cnt);
  f[7] = __fmul_rn(flog_bits(u2f((uint32_t)S.bkey[0])), 0.125f);
  f[8] = __fmul_rn(flog_bits(u2f((uint32_t)S.bkey[np > 0 ? kk - 1 : cnt - 1])), 0.125f);
  f[9] = __fdiv_rn((float)kk, (float)k);
  f[10] = __fdiv_rn((float)fu, (float)cnt);
  f[11] = __fmul_rn(flog_bits(u2f((uint32_t)S.bkey[cnt - 1])), 0.125f);
  if (feat_out) {
#pragma unroll
    for (int i = 0; i < JAG_MLP_FEATURES; ++i)
      if (lane == i) feat_out[i] = f[i];
  }
  PolicyOut o;
  if (pol.mode == JAG_POLICY_FORCED) {
    const int fb = forced_q[0], fs = forced_q[1];
    o.beam = fb > 0 ? (fb < k ? k : fb > fixed ? fixed : fb) : fixed;
    o.stop = fs > 0 ? (fs < pol.h0 ? pol.h0 : fs) : 0;
    o.learned = fb > 0 ? 1 : 0;
    return o;
  }
  // network: lanes hold neurons lane and lane + 32 of each hidden layer
  const uint16_t *w1 = pol.w_bf16, *w2 = w1 + JAG_MLP_HIDDEN * JAG_MLP_FEATURES, *w3 = w2 + JAG_MLP_HIDDEN * JAG_MLP_HIDDEN;
  const float *b1 = pol.b_f32, *b2 = b1 + JAG_MLP_HIDDEN, *b3 = b2 + JAG_MLP_HIDDEN;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int n = lane + 32 * h;
    float acc = b1[n];
#pragma unroll
    for (int i = 0; i < JAG_MLP_FEATURES; ++i) acc = __fmaf_rn(bf16_value(w1[n * JAG_MLP_FEATURES + i]), f[i], acc);
    hbuf[n] = acc > 0.f ? acc : 0.f;
  }
  __syncwarp();
  // the second layer is held in registers until every lane has read the
  // first, then takes its place (64 floats of scratch in all)
  float h2[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int n = lane + 32 * h;
    float acc = b2[n];
    for (int i = 0; i < JAG_MLP_HIDDEN; ++i) acc = __fmaf_rn(bf16_value(w2[n * JAG_MLP_HIDDEN + i]), hbuf[i], acc);
    h2[h] = acc > 0.f ? acc : 0.f;
  }
  __syncwarp();
  hbuf[lane] = h2[0];
  hbuf[lane + 32] = h2[1];
  __syncwarp();
  const int nl = pol.n_ladder;
  float out = -INFINITY;
  if (lane <= nl) {
    float acc = b3[lane];
    for (int i = 0; i < JAG_MLP_HIDDEN; ++i) acc = __fmaf_rn(bf16_value(w3[lane * JAG_MLP_HIDDEN + i]), hbuf[i], acc);
    out = acc;
  }
  __syncwarp();
  // largest beam output (lowest class on a tie), then the runner-up
  float v = lane < nl ? out : -INFINITY;
  int c = lane;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const float ov = __shfl_xor_sync(kFull, v, off);
    const int oc = __shfl_xor_sync(kFull, c, off);
    if (ov > v || (ov == v && oc < c)) { v = ov; c = oc; }
  }
  float v2 = (lane < nl && lane != c) ? out : -INFINITY;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v2 = fmaxf(v2, __shfl_xor_sync(kFull, v2, off));
  const float margin = __fsub_rn(v, v2);
  const float sv = __shfl_sync(kFull, out, nl);
  if (!(margin >= pol.tau)) {
    o.beam = fixed; o.stop = 0; o.learned = 0;
    return o;
  }
  const float r = rintf(__fmul_rn(sv, pol.stop_scale));
  int st;
  if (!(pol.stop_scale > 0.f)) st = 0;
  else if (!(r == r) || r >= 65535.f) st = 65535;
  else if (r <= (float)pol.h0) st = pol.h0;
  else st = (int)r;
  o.beam = pol.ladder[c] < fixed ? pol.ladder[c] : fixed;
  o.stop = st; o.learned = 1;
  return o;
}

// Per-search policy context of greedy_search.  It lives in the warp's shared
// memory, kPolicyCtxBytes right after its search arrays (policy_ctx), so that
// the search loop keeps no register for it.
struct PolicyCtx {
  const jag_policy *pol;   // nullptr: plain search
  int64_t est;
  int32_t kind;
  int32_t k;
  float *hbuf;             // 64 floats of the warp (its free candidate scratch)
  float *feat_out;         // [12] or nullptr
  int32_t *dec_out;        // [4] or nullptr
  const int32_t *forced_q; // [2] or nullptr
  int32_t lim;             // hop limit of the current phase (set by greedy_search)
};
constexpr size_t kPolicyCtxBytes = 64;
static_assert(sizeof(PolicyCtx) <= kPolicyCtxBytes, "policy context slot");

__device__ __forceinline__ PolicyCtx *policy_ctx(const WarpSmem &S) {
  return reinterpret_cast<PolicyCtx *>(S.rank + 32);
}

// Where a search stands between two calls of greedy_search: the count of L
// and the first position that may hold an unexpanded entry.
struct SearchCursor {
  int cnt, start;
};

// Algorithm 1 for one search by the calling warp.  On return S.bkey/S.bid
// hold the final list L (count returned).
// POL: 0 plain search; 1 with the policy's decision at hop h0 taken inside
// the loop; 2 as 1, and the trace of the search (decisions and the last hop
// that changed the first k entries) written to dec_out; for 1 and 2 the
// caller fills policy_ctx(S) first.  The kernels use 2 for traced searches
// only; an untraced policy search runs POL 0 with RES and takes its decision
// between two calls (query_kernel, serve_query).
// RES: the search stops before a hop once st.hops >= max_hops, and ends by
// storing its cursor in *cur; if cur->cnt > 0 on entry it resumes instead of
// starting (L, the visited set and st are then as the stopped search left
// them).  Without RES both arguments are ignored.
template <int CAP, int P, int CPL, int FMT, int POL = 0, bool RES = false, class KeyFn, class Sink>
__device__ int greedy_search(const DevIndex &ix, const KeyFn &key1, const QChunks<CPL, FMT> &q, int ls,
                             int hbits, const WarpSmem &S, Sink &sink, SearchStats &st,
                             int max_hops = 0x7FFFFFFF, SearchCursor *cur = nullptr) {
  // policy state: the hop limit of the current phase, kept in shared memory
  // -- the decision hop h0, then the stop hop (>= h0; a stop at h0 ends the
  // search right after the decision, so a limit equal to h0 is always the
  // decision's) -- and, for a trace, the last hop that changed the first k
  // entries
  const int lane = threadIdx.x & 31;
  int last_change = 0;
  const int kq = POL == 2 ? policy_ctx(S)->k : 0;
  if (POL && lane == 0) {
    PolicyCtx *pc = policy_ctx(S);
    pc->lim = pc->pol->mode != JAG_POLICY_PLAIN ? pc->pol->h0 : 0x7FFFFFFF;
    if (pc->dec_out) { pc->dec_out[0] = ls; pc->dec_out[1] = 0; pc->dec_out[2] = 0; pc->dec_out[3] = 0; }
  }
  const bool resume = RES && cur->cnt > 0;
  int cnt = 1, start = 0;
  if (resume) {
    cnt = cur->cnt;
    start = cur->start;
  } else {
    const uint32_t hsize = 1u << hbits;
    for (uint32_t i = lane; i < hsize; i += 32) S.hash[i] = kEmptySlot;
    __syncwarp();
    const int32_t s = ix.entry;
    if (lane == 0) { S.cid[0] = (uint32_t)s; S.hash[((uint32_t)s * 0x9E3779B1u) >> (32 - hbits)] = (uint32_t)s; }
    __syncwarp();
    const float d0 = candidate_distances<P, CPL, 4, FMT>(ix, q, S.cid, 1);
    const uint32_t k0 = key1(ix, s);
    const float d0b = __shfl_sync(kFull, d0, 0);
    if (lane == 0) { S.bkey[0] = key1.key(k0, d0b); S.bid[0] = (uint32_t)s; }
    __syncwarp();
    st.hops = 0; st.seen = 0; st.dcs = 1;
  }
  if (POL) {
    float *fo = policy_ctx(S)->feat_out;
    if (fo && lane < JAG_MLP_FEATURES) fo[lane] = 0.f;
  }
  for (;;) {
    // the decision, after hop h0
    if (POL && st.hops >= policy_ctx(S)->lim) {
      const PolicyCtx *pc = policy_ctx(S);
      if (pc->lim != pc->pol->h0) break;
      const PolicyOut o = policy_decide(*pc->pol, S, pc->hbuf, cnt, pc->k, pc->est, pc->kind, ls, pc->feat_out,
                                        pc->forced_q);
      const int lim = o.stop > 0 ? o.stop : 0x7FFFFFFF;
      __syncwarp();
      if (lane == 0) {
        PolicyCtx *pw = policy_ctx(S);
        if (pw->dec_out) { pw->dec_out[0] = o.beam; pw->dec_out[1] = o.stop; pw->dec_out[3] = o.learned; }
        pw->lim = lim;
      }
      __syncwarp();
      ls = o.beam;
      if (cnt > ls) cnt = ls;
      if (st.hops >= lim) break;
    }
    if (RES && st.hops >= max_hops) break;
    const int sel = first_unexpanded(S.bid, cnt, start);
    if (sel < 0) break;
    const uint32_t pid = S.bid[sel];
    const uint64_t pkey = S.bkey[sel];
    __syncwarp();
    if (lane == 0) S.bid[sel] = pid | kExpanded;
    sink.visit(lane, pid, pkey);
    st.hops += 1;
    const int64_t e0 = (int64_t)pid * ix.R;
    int rmin = cnt;
    for (int rb = 0; rb < ix.R; rb += 32) {
      // the out-edge and its target's attribute word: the attribute is read
      // whether or not the slot holds an edge, so both loads leave at once
      const bool slot = rb + lane < ix.R;
      const int u = slot ? __ldg(ix.graph + e0 + rb + lane) : -1;
      uint64_t aw = 0;
      if (KeyFn::kEdgeAttr && slot) aw = key1.edge_word(ix, e0 + rb + lane);
      const bool full = (cnt == ls);
      const uint64_t tkey = full ? S.bkey[ls - 1] : kNoKey;
      const uint32_t tid = full ? (S.bid[ls - 1] & ~kExpanded) : kEmptySlot;
      // first key, and early rejection, before the visited set: a rejected
      // neighbour is rejected again at any later meeting, so only neighbours
      // whose distance is computed need to be remembered
      uint32_t k1 = 0;
      bool cand = u >= 0;
      if (KeyFn::kEdgeAttr) {
        k1 = key1.from_word(aw);   // every lane (aw is 0 past the out-list): no branch
      } else if (cand) {
        k1 = key1(ix, u);
      }
      cand = cand & (KeyFn::kScalar | !(full & (k1 > (uint32_t)(tkey >> 32))));
      bool keep = false;
      if (cand) keep = visit_insert(S.hash, hbits, (uint32_t)u);
      const uint32_t km = __ballot_sync(kFull, keep);
      const int nc = __popc(km);
      st.seen += nc;
      if (keep) {
        const int r = __popc(km & lanemask_lt());
        S.cid[r] = (uint32_t)u;
        S.ck1[r] = k1;
      }
      __syncwarp();
      if (nc == 0) continue;
      st.dcs += nc;
      const float dist = candidate_distances<P, CPL, 4, FMT, prefetch_rows(FMT)>(ix, q, S.cid, nc);
      // lanes past nc read stale slots of the 32-entry arrays and drop them
      uint64_t ck = key1.key(S.ck1[lane], dist);
      uint32_t cv = S.cid[lane];
      const bool drop = (lane >= nc) | (full & !key_less(ck, cv, tkey, tid));
      ck = drop ? kNoKey : ck;
      cv = drop ? kEmptySlot : cv;
      int r0;
      cnt = merge_candidates<CAP>(S.bkey, S.bid, cnt, ls, ck, cv, r0);
      rmin = r0 < rmin ? r0 : rmin;
      if (POL == 2 && r0 < kq) last_change = st.hops;
    }
    start = (sel + 1) < rmin ? (sel + 1) : rmin;
  }
  if (POL == 2 && lane == 0 && policy_ctx(S)->dec_out) policy_ctx(S)->dec_out[2] = last_change;
  if (RES) { cur->cnt = cnt; cur->start = start; }
  return cnt;
}

__device__ __forceinline__ void write_answers(const WarpSmem &S, int cnt, int64_t qi, int k, int32_t *out_ids,
                                              float *out_dist) {
  const int lane = threadIdx.x & 31;
  for (int j = lane; j < k; j += 32) {
    int32_t id = -1;
    float dd = __int_as_float(0x7F800000);
    if (j < cnt) {
      const uint64_t kk = S.bkey[j];
      if ((kk >> 32) == 0) { id = (int32_t)(S.bid[j] & ~kExpanded); dd = u2f((uint32_t)kk); }
    }
    out_ids[qi * k + j] = id;
    out_dist[qi * k + j] = dd;
  }
}

}  // namespace jag
