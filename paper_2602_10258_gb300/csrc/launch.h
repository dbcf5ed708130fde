// Host-side launch interface between the C ABI layer and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "jag_internal.cuh"

namespace jag {

// Queries of one work item of the tensor-core exact scan at most (the MMA's N).
constexpr int kTcItemQueries = 64;

// Scratch of the tensor-core exact scan (scan_tc.cu): approximate distances
// [nq][cap] and |q|^2 [nq]; per work unit (2 T0 tiles of the two sorted
// columns, T0 = ceil(n / 128), then one list unit per query) the count, fill
// and first entry of its query list, and its first work item; the lists
// (tq); the unit of every work item; block sums of the unit scan.
struct TcScratch {
  float *approx, *qnorm;
  int32_t *tcnt, *tfill, *toff, *tq, *item_unit;
  int64_t *ioff, *bsum;
};

// Grouping of identical list-routed filters (a hash table of `slots`
// entries): per query its slot, per slot its leader, and the leaders.
struct ListGroups {
  uint64_t *hkey;
  int32_t *hlead, *lslot, *leaders;
  size_t slots;
};

// One jag_search call, resolved to device pointers.
struct SearchLaunch {
  DevIndex ix;
  const float *queries;
  int32_t d;
  const jag_filter *filters;
  const uint8_t *aux;
  int64_t aux_bytes;
  int64_t nq;
  int32_t k, ls, hbits;
  int32_t hbits_auto;      // hbits is the default: the graph launch may lower it
  int64_t s0, cap;
  int32_t scan_all;
  int32_t *out_ids;
  float *out_dist;
  int32_t *counters;
  // scratch
  QueryPlan *plans;
  uint8_t *lut;
  int32_t *lists;          // [nq][cap] passing ids gathered by list-routed leaders
  ListGroups lgroup;       // identical list-routed filters share their leader's list
  int32_t *list_counts;    // [nq]
  unsigned long long *work;  // [4] work counters
  uint32_t *status;
  uint64_t *part_key;      // partial top-k lists [nq][ntiles][k]
  uint32_t *part_id;
  uint64_t *scan_items;    // [nq * ntiles] (query, tile) work items of the exact scan
  int32_t ntiles;
  int64_t tile;
  jag_policy policy;       // learned / forced beam and stop hop (has_policy)
  int32_t has_policy;
  int32_t rr;              // re-ranked candidates per query (BF16 / FP8 rows)
  int32_t *rr_ids;         // [nq][rr]
  cudaEvent_t ev_begin, ev_end;
  cudaStream_t stream;
  int32_t fork_scan;       // run the exact scan on a side stream, concurrently
  TcScratch tc;            // tensor-core scan scratch; tc.approx == nullptr: the fp32 scan kernels
};

// Graph-search launch for rows stored in format FMT (search_<fmt>.cu).
template <int FMT>
cudaError_t launch_graph_fmt(const SearchLaunch &L);

// Scratch of one search call: byte offsets of its regions (256-aligned) in
// one buffer, and the total.  A region is sized only when the call can use
// it: mask lists when the scan route is on and the index has a mask column,
// partial lists and scan work items when any query can be scanned, re-rank
// ids for BF16 / FP8 rows.  jag_search, jag_search_host and
// jag_search_noalloc all lay out their scratch with this one function.
// With tc, the scan route runs on the tensor cores (scan_tc.cu) and its
// regions replace the fp32 scan's partial lists and work items.
struct SearchScratch {
  size_t plans, lut, lists, lhkey, lhlead, lslot, leaders, lslots, list_counts, work, status, part_key, part_id,
      scan_items, rr_ids;
  size_t approx, qnorm, tcnt, tfill, toff, tq, item_unit, ioff, bsum;
  size_t total;
  int32_t rr, ntiles, tc;
  int64_t tile;
};
SearchScratch search_scratch_layout(const DevIndex &ix, int64_t nq, int64_t aux_bytes, int64_t cap, int32_t k,
                                    int32_t ls, int scan_all, int64_t s0, int tc);
// Points the scratch pointers of L into base by the layout s.
void bind_scratch(SearchLaunch &L, const SearchScratch &s, uint8_t *base);
// Default log2 size of the visited set (1024 slots, 4 KB): a larger set costs
// occupancy, a smaller one recomputation.
inline int default_hash_bits() { return 10; }
// Resolves, on the current device, the device address of the fixed scratch
// area of jag_search_noalloc (noalloc.cu); jag_build calls it so that the
// area is in place before any search.
cudaError_t noalloc_prepare(int device);
// Candidates re-ranked in fp32 per query with BF16 / FP8 rows: min(4k, ls).
inline int32_t rerank_count(int32_t k, int32_t ls) { return 4 * k < ls ? 4 * k : ls; }
// Partial top-k lists: the brute-force scan cuts the points into tiles of
// 65536, the scan route cuts each passing set (at most max(s0, cap) ids) into
// tiles of 1024.
void scan_tiling(int64_t n, int scan_all, int64_t s0, int64_t cap, int32_t *ntiles, int64_t *tile);

cudaError_t run_search(const SearchLaunch &L);

// The tensor-core exact scan of the scan-routed queries (scan_tc.cu).
cudaError_t launch_scan_tc(const SearchLaunch &L);
// Slots of a grouping hash table for nq queries: a power of two >= 2 nq.
size_t tc_slots(int64_t nq);
// Tiles of 128 positions of a sorted column of n points.
int64_t tc_column_tiles(int64_t n);
// |x|^2 of every row into xn and their maximum into *xmax_host (dmax: one
// device word of scratch); synchronous on stream.
cudaError_t row_norms(const DevIndex &ix, float *xn, unsigned int *dmax, float *xmax_host, cudaStream_t stream);

// Smallest supported list capacity >= ls (64, 128, 256 or 512); 0 if ls > 512.
int list_capacity(int ls);
// Lanes per row P and chunks per lane for a row of nchunks 16-byte chunks.
bool row_mapping(int nchunks, int *P, int *CPL);

// BF16 / FP8 rows of an index from its fp32 rows (quant.cu).
cudaError_t quantize_rows(const DevIndex &ix, int fmt, uint8_t *xq, float *qscale, cudaStream_t stream);

// Accessors of the C ABI layer for other translation units.
bool index_view(const jag_index *idx, DevIndex *ix, int *device);
jag_status check_search(const jag_index *idx, const jag_search_args *a);
jag_status set_error(jag_status s, const char *msg);

// Fill the edge attribute tables of a finished graph (any pointer may be NULL).
cudaError_t build_edge_attrs(const DevIndex &ix, int32_t *ea_i32, float *ea_f32, uint64_t *ea_mask,
                             cudaStream_t stream);

// GPU index build (Algorithms 3 and 4); see build.cu.
struct BuildLaunch {
  DevIndex ix;              // graph pointer is writable
  int32_t *graph;
  uint32_t *thr;            // [n][nT]
  int32_t nT;
  int32_t pct[4];
  int32_t sample;
  uint64_t seed;
  int32_t lb;
  float alpha2;
  int32_t weighted;         // Weight-JAG: thr holds fp32 weights mult[i] * h_p
  double mult[8];
  cudaStream_t stream;
};
// Returns 0 on success, else a jag_status code; msg receives a description.
int run_build(BuildLaunch &B, int32_t *entry_out, char *msg, size_t msg_len);

}  // namespace jag
