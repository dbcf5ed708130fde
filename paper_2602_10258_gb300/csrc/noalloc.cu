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
// With CUDA's lazy module loading the array is placed on a device when its
// address is first looked up; jag_build does that on the index's device, so
// the area is in place before the first search.  All calls, on every stream,
// share it and it keeps the previous call's contents; calls whose device
// work overlaps therefore race.
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

// Device address of the scratch array on the current device, which must be
// `device`.  On the host the array's name is only a stand-in, so the address
// comes from the runtime, once per device, with that device current.  The
// lookup also loads the array on that device if it is not loaded yet.
cudaError_t scratch_address(int device, uint8_t **out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
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

cudaError_t noalloc_prepare(int device) {
  uint8_t *p = nullptr;
  return scratch_address(device, &p);
}

}  // namespace jag

extern "C" JAG_API jag_status jag_search_noalloc(jag_index *idx, const jag_search_args *a) {
  using namespace jag;
  jag_status st = check_search(idx, a);
  if (st != JAG_OK) return st;
  DevIndex ix;
  int device = 0;
  index_view(idx, &ix, &device);
  if (device < 0 || device >= kMaxDevices) return set_error(JAG_EUNSUPPORTED, "device ordinal too large");
  const int64_t s0 = a->s0 < 0 ? 2048 : a->s0;
  const int64_t cap = a->scan_cap <= 0 ? 8192 : a->scan_cap;
  const int scan_all = (a->flags & JAG_SEARCH_SCAN_ALL) ? 1 : 0;
  // the layout jag_search uses, in the fixed area
  // (with the fp32 scan kernels, whose scratch is far smaller than the
  // tensor-core scan's nq * scan_cap approximations; the answers are the same)
  const SearchScratch lay = search_scratch_layout(ix, a->nq, a->aux_bytes, cap, a->k, a->beam, scan_all, s0, 0);
  if (lay.total > kNoAllocScratchBytes) {
    char msg[256];
    snprintf(msg, sizeof(msg),
             "jag_search_noalloc needs %zu bytes of scratch, more than its fixed %zu; use fewer queries per "
             "call, a smaller scan_cap or filter_aux, s0 = 0, or jag_search",
             lay.total, kNoAllocScratchBytes);
    return set_error(JAG_EINVAL, msg);
  }
  if (a->nq == 0) return JAG_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return set_error(JAG_ECUDA, "cudaSetDevice failed");
  uint8_t *base = nullptr;
  cudaError_t e = scratch_address(device, &base);
  if (e != cudaSuccess) {
    cudaSetDevice(prev);
    return set_error(JAG_ECUDA, "cudaGetSymbolAddress of the no-allocation scratch failed");
  }
  SearchLaunch L{};
  L.ix = ix;
  L.queries = a->queries;
  L.d = ix.d;
  L.filters = a->filters;
  L.aux = a->filter_aux;
  L.aux_bytes = a->aux_bytes;
  L.nq = a->nq;
  L.k = a->k; L.ls = a->beam;
  L.hbits = a->hash_bits ? a->hash_bits : default_hash_bits();
  L.hbits_auto = a->hash_bits == 0;
  L.s0 = s0; L.cap = cap; L.scan_all = scan_all;
  L.out_ids = a->out_ids; L.out_dist = a->out_dist; L.counters = a->counters;
  bind_scratch(L, lay, base);
  if (a->policy) { L.policy = *a->policy; L.has_policy = 1; }
  L.ev_begin = (cudaEvent_t)a->ev_graph_begin;
  L.ev_end = (cudaEvent_t)a->ev_graph_end;
  L.stream = (cudaStream_t)a->stream;
  // the status word must start at zero (the work counters are cleared by the launch sequence)
  e = cudaMemsetAsync(L.status, 0, 4, L.stream);
  if (e == cudaSuccess) e = run_search(L);
  cudaSetDevice(prev);
  if (e != cudaSuccess) return set_error(JAG_ECUDA, cudaGetErrorString(e));
  return JAG_OK;
}
