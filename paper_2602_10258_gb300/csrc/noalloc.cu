// jag_search_noalloc: the search of jag_search, run entirely in a fixed
// scratch area that the library reserves when it is loaded, so the call
// never asks the CUDA runtime for memory.
//
// Who needs this: code that must search without allocating device memory.
// cudaMalloc can wait for work already queued on the device, which a
// latency-bound serving thread cannot afford; some processes hand all device
// memory to their own allocator up front, so a raw cudaMalloc would fail; and
// some deployments forbid dynamic allocation after start-up.  jag_search
// allocates its per-stream scratch on first use and grows it for larger
// batches; this entry point uses a file-scope device array instead.
//
// The array (kNoAllocScratchBytes) is part of the library's device image:
// every GPU on which the library is loaded holds it until the process exits.
// All calls, on every stream, share it and it keeps the previous call's
// contents; calls whose device work overlaps therefore race.
#include <cstdio>
#include <mutex>

#include "launch.h"
#include "search_core.cuh"

namespace jag {

constexpr size_t kNoAllocScratchBytes = 16u << 20;   // 16 MiB per device

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
uint8_t *g_scratch_ptr[kMaxDevices] = {};

size_t a256(size_t v) { return (v + 255) & ~size_t(255); }

// Device address of the scratch array on the current device.  On the host
// the array's name is only a stand-in, so the address comes from the
// runtime, once per device, with that device current.
cudaError_t scratch_address(int device, uint8_t **out) {
  std::lock_guard<std::mutex> g(g_setup_mu);
  if (!g_scratch_ptr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = static_cast<uint8_t *>(p);
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

}  // namespace
}  // namespace jag

extern "C" JAG_API jag_status jag_search_noalloc(jag_index *idx, const jag_search_args *a) {
  using namespace jag;
  jag_status st = check_search(idx, a);
  if (st != JAG_OK) return st;
  DevIndex ix;
  int device = 0;
  index_view(idx, &ix, &device);
  if (device < 0 || device >= kMaxDevices) return set_error(JAG_EUNSUPPORTED, "device ordinal too large");
  const int64_t nq = a->nq;
  const int64_t s0 = a->s0 < 0 ? 2048 : a->s0;
  const int64_t cap = a->scan_cap <= 0 ? 8192 : a->scan_cap;
  const int scan_all = (a->flags & JAG_SEARCH_SCAN_ALL) ? 1 : 0;
  // scratch layout: only the regions this call can touch
  int64_t tile;
  int32_t ntiles;
  scan_tiling(ix.n, scan_all, s0, cap, &ntiles, &tile);
  const bool lists = !scan_all && s0 > 0 && ix.a_mask != nullptr;
  size_t off = 0;
  const size_t o_plans = off; off += a256(sizeof(QueryPlan) * (size_t)(nq > 0 ? nq : 1));
  const size_t o_lut = off; off += a256((size_t)(a->aux_bytes > 0 ? a->aux_bytes : 1) * 8);
  const size_t o_lists = off; off += lists ? a256((size_t)nq * (size_t)cap * 4) : 256;
  const size_t o_counts = off; off += a256(4 * (size_t)(nq > 0 ? nq : 1));
  const size_t o_work = off; off += 256;
  const size_t o_status = off; off += 256;
  const size_t parts = (scan_all || s0 > 0) ? (size_t)nq * (size_t)ntiles * (size_t)a->k : 1;
  const size_t o_pkey = off; off += a256(parts * 8);
  const size_t o_pid = off; off += a256(parts * 4);
  off += (!scan_all && s0 > 0) ? a256(parts * 8) : 0;   // scan work items follow the partial lists
  const int32_t rr = ix.fmt != JAG_VEC_F32 ? rerank_count(a->k, a->beam) : 0;
  const size_t o_rr = off; off += a256((size_t)(nq > 0 ? nq : 1) * (size_t)(rr > 0 ? rr : 1) * 4);
  if (off > kNoAllocScratchBytes) {
    char msg[256];
    snprintf(msg, sizeof(msg),
             "jag_search_noalloc needs %zu bytes of scratch, more than its fixed %zu; use fewer queries per "
             "call, a smaller scan_cap or filter_aux, s0 = 0, or jag_search",
             off, kNoAllocScratchBytes);
    return set_error(JAG_EINVAL, msg);
  }
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return set_error(JAG_ECUDA, "cudaSetDevice failed");
  uint8_t *base = nullptr;
  cudaError_t e = scratch_address(device, &base);
  if (e != cudaSuccess) {
    cudaSetDevice(prev);
    return set_error(JAG_ECUDA, "cudaGetSymbolAddress of the no-allocation scratch failed");
  }
  cudaStream_t stream = (cudaStream_t)a->stream;
  SearchLaunch L{};
  L.ix = ix;
  L.queries = a->queries;
  L.d = ix.d;
  L.filters = a->filters;
  L.aux = a->filter_aux;
  L.aux_bytes = a->aux_bytes;
  L.nq = nq;
  L.k = a->k; L.ls = a->beam;
  L.hbits = a->hash_bits ? a->hash_bits : 10;
  L.hbits_auto = a->hash_bits == 0;
  L.s0 = s0; L.cap = cap; L.scan_all = scan_all;
  L.out_ids = a->out_ids; L.out_dist = a->out_dist; L.counters = a->counters;
  L.plans = (QueryPlan *)(base + o_plans);
  L.lut = base + o_lut;
  L.lists = (int32_t *)(base + o_lists);
  L.list_counts = (int32_t *)(base + o_counts);
  L.work = (unsigned long long *)(base + o_work);
  L.status = (uint32_t *)(base + o_status);
  L.part_key = (uint64_t *)(base + o_pkey);
  L.part_id = (uint32_t *)(base + o_pid);
  L.ntiles = ntiles; L.tile = tile;
  L.rr = rr;
  L.rr_ids = (int32_t *)(base + o_rr);
  if (a->policy) { L.policy = *a->policy; L.has_policy = 1; }
  L.ev_begin = (cudaEvent_t)a->ev_graph_begin;
  L.ev_end = (cudaEvent_t)a->ev_graph_end;
  L.stream = stream;
  // the status word must start at zero (the work counters are cleared by the launch sequence)
  e = cudaMemsetAsync(L.status, 0, 4, stream);
  if (e == cudaSuccess) e = run_search(L);
  cudaSetDevice(prev);
  if (e != cudaSuccess) return set_error(JAG_ECUDA, cudaGetErrorString(e));
  return JAG_OK;
}
