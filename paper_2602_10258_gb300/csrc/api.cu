// C ABI of the library (include/jag.h): argument checks, device memory of an
// index, per-stream scratch, and the launch sequences of search and build.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include "jag.h"
#include "launch.h"
#include "search_core.cuh"

namespace {

thread_local std::string g_err;

jag_status fail(jag_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

jag_status cuda_fail(cudaError_t e, const char *what) {
  return fail(e == cudaErrorMemoryAllocation ? JAG_ENOMEM : JAG_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

struct Buffer {
  void *ptr = nullptr;
  size_t bytes = 0;
};

// Device scratch owned by the library, one per stream.
struct Workspace {
  std::mutex mu;
  Buffer buf;
};

// Device staging for jag_search_host.
struct HostStage {
  std::mutex mu;
  Buffer q, f, aux, ids, dist, cnt;
  cudaStream_t stream = nullptr;
};

cudaError_t ensure(Buffer &b, size_t bytes, cudaStream_t stream) {
  if (b.bytes >= bytes && b.ptr) return cudaSuccess;
  if (b.ptr) {
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return e;
    cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
  }
  size_t want = std::max<size_t>(bytes, 4096);
  cudaError_t e = cudaMalloc(&b.ptr, want);
  if (e != cudaSuccess) { b.ptr = nullptr; return e; }
  b.bytes = want;
  return cudaSuccess;
}

}  // namespace

struct jag_index {
  int device = 0;
  jag::DevIndex ix{};
  int64_t n = 0, d = 0;
  int32_t R = 0, storage = JAG_VEC_F32, nT = 0, dist_a = 0, weighted = 0;
  std::vector<void *> allocs;
  size_t device_bytes = 0;
  double build_seconds = 0.0;
  float *x = nullptr;
  int32_t *graph = nullptr;
  uint32_t *thr = nullptr;
  std::mutex mu;
  std::unordered_map<cudaStream_t, Workspace *> ws;
  HostStage host;

  ~jag_index() {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    for (auto &kv : ws) {
      if (kv.second->buf.ptr) cudaFree(kv.second->buf.ptr);
      delete kv.second;
    }
    for (Buffer *b : {&host.q, &host.f, &host.aux, &host.ids, &host.dist, &host.cnt})
      if (b->ptr) cudaFree(b->ptr);
    if (host.stream) cudaStreamDestroy(host.stream);
    for (void *p : allocs) cudaFree(p);
    cudaSetDevice(prev);
  }

  cudaError_t alloc(void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 256);
    if (e == cudaSuccess) { allocs.push_back(*p); device_bytes += bytes; }
    return e;
  }

  Workspace *workspace(cudaStream_t s) {
    std::lock_guard<std::mutex> g(mu);
    auto it = ws.find(s);
    if (it != ws.end()) return it->second;
    Workspace *w = new Workspace();
    ws.emplace(s, w);
    return w;
  }
};

namespace {

struct DeviceGuard {
  int prev = 0;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
  }
  ~DeviceGuard() { cudaSetDevice(prev); }
};

template <class T>
bool all_finite(const T *v, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite((double)v[i])) return false;
  return true;
}

template <class V>
void sorted_column(const V *vals, int64_t n, std::vector<V> &sv, std::vector<int32_t> &si) {
  std::vector<std::pair<V, int32_t>> tmp((size_t)n);
  for (int64_t i = 0; i < n; ++i) tmp[(size_t)i] = {vals[i], (int32_t)i};
  std::sort(tmp.begin(), tmp.end());
  sv.resize((size_t)n);
  si.resize((size_t)n);
  for (int64_t i = 0; i < n; ++i) { sv[(size_t)i] = tmp[(size_t)i].first; si[(size_t)i] = tmp[(size_t)i].second; }
}

constexpr size_t kSmemLimit = 227 * 1024;

jag_status check_search_args(const jag_index *idx, const jag_search_args *a) {
  if (!idx) return fail(JAG_EINVAL, "index is NULL");
  if (!a) return fail(JAG_EINVAL, "args is NULL");
  if (a->nq < 0) return fail(JAG_EINVAL, "nq < 0");
  if (a->nq > 0 && (!a->queries || !a->filters || !a->out_ids || !a->out_dist))
    return fail(JAG_EINVAL, "NULL query, filter or output pointer");
  if (a->beam < 1 || a->beam > 512) return fail(JAG_EINVAL, "beam must be in [1, 512]");
  if (a->k < 1 || a->k > a->beam || a->k > 256) return fail(JAG_EINVAL, "k must be in [1, min(beam, 256)]");
  if (a->policy && a->beam > 256) return fail(JAG_EINVAL, "a search with a policy takes beams of at most 256");
  if (a->aux_bytes < 0 || (a->aux_bytes > 0 && !a->filter_aux)) return fail(JAG_EINVAL, "bad filter_aux");
  if (a->nq > (int64_t)1 << 31) return fail(JAG_EINVAL, "nq too large");
  if (a->policy) {
    const jag_policy *p = a->policy;
    if (p->mode < JAG_POLICY_PLAIN || p->mode > JAG_POLICY_FORCED) return fail(JAG_EINVAL, "bad policy mode");
    if (p->mode != JAG_POLICY_PLAIN && p->h0 < 1) return fail(JAG_EINVAL, "policy h0 must be >= 1");
    if (p->mode == JAG_POLICY_LEARNED) {
      if (!p->w_bf16 || !p->b_f32) return fail(JAG_EINVAL, "policy weights are NULL");
      if (p->n_ladder < 1 || p->n_ladder > 16) return fail(JAG_EINVAL, "n_ladder must be in [1, 16]");
      for (int i = 0; i < p->n_ladder; ++i)
        if (p->ladder[i] < a->k || p->ladder[i] > 256) return fail(JAG_EINVAL, "ladder beams must be in [k, 256]");
    }
    if (p->mode == JAG_POLICY_FORCED && !p->forced) return fail(JAG_EINVAL, "forced policy needs `forced`");
  }
  int hb = a->hash_bits ? a->hash_bits : jag::default_hash_bits();
  if (hb < 5 || hb > 16) return fail(JAG_EINVAL, "hash_bits must be in [5, 16]");
  if ((size_t)jag::kSearchWarps * jag::warp_smem_bytes(jag::list_slots(a->beam), hb) > kSmemLimit)
    return fail(JAG_EINVAL, "hash_bits too large for the beam");
  return JAG_OK;
}

}  // namespace

namespace jag {

// Read access for other translation units of the library: the device-side
// view of an index and its device ordinal.
bool index_view(const jag_index *idx, DevIndex *ix, int *device) {
  if (!idx) return false;
  *ix = idx->ix;
  *device = idx->device;
  return true;
}

// The argument checks of jag_search, with the thread's error message set.
jag_status check_search(const jag_index *idx, const jag_search_args *a) {
  g_err.clear();
  return check_search_args(idx, a);
}

jag_status set_error(jag_status s, const char *msg) { return fail(s, "%s", msg); }

}  // namespace jag

extern "C" {

const char *jag_last_error(void) { return g_err.c_str(); }

const char *jag_version(void) { return "jag-gb300 0.1 (sm_103a)"; }

jag_status jag_build(const jag_build_params *p, jag_index **out) {
  g_err.clear();
  if (!p || !out) return fail(JAG_EINVAL, "NULL params or out");
  *out = nullptr;
  if (p->n < 1 || p->n >= ((int64_t)1 << 31) - 1) return fail(JAG_EINVAL, "n out of range");
  if (p->d < 1 || p->d > 1024) return fail(JAG_EINVAL, "d must be in [1, 1024]");
  if (!p->x) return fail(JAG_EINVAL, "x is NULL");
  if (p->R < 1 || p->R > 64) return fail(JAG_EINVAL, "R must be in [1, 64]");
  if (p->storage != JAG_VEC_F32 && p->storage != JAG_VEC_BF16 && p->storage != JAG_VEC_FP8)
    return fail(JAG_EINVAL, "bad storage format");
  const bool prebuilt = p->graph != nullptr;
  if (!prebuilt) {
    if (p->l_b < 1 || p->l_b > 256) return fail(JAG_EINVAL, "l_b must be in [1, 256]");
    if (!(p->alpha >= 1.0f) || !std::isfinite(p->alpha)) return fail(JAG_EINVAL, "alpha must be finite and >= 1");
    if (p->n_weights < 0 || p->n_weights > 8) return fail(JAG_EINVAL, "n_weights must be in [0, 8]");
    if (p->n_weights > 0) {
      for (int i = 0; i < p->n_weights; ++i)
        if (!(p->weight_mult[i] >= 0.0) || !std::isfinite(p->weight_mult[i]))
          return fail(JAG_EINVAL, "weight_mult must be finite and >= 0");
    } else {
      if (p->n_thresholds < 1 || p->n_thresholds > 4) return fail(JAG_EINVAL, "n_thresholds must be in [1, 4]");
      for (int i = 0; i < p->n_thresholds; ++i)
        if (p->threshold_pct[i] < 0 || p->threshold_pct[i] > 100)
          return fail(JAG_EINVAL, "threshold_pct out of [0,100]");
    }
    if (p->sample_size < 1 || p->sample_size > 1024) return fail(JAG_EINVAL, "sample_size must be in [1, 1024]");
    switch (p->dist_a) {
      case JAG_F_LABEL: case JAG_F_RANGE_I32:
        if (!p->attr_i32) return fail(JAG_EINVAL, "dist_a needs attr_i32");
        break;
      case JAG_F_RANGE_F32:
        if (!p->attr_f32) return fail(JAG_EINVAL, "dist_a needs attr_f32");
        break;
      case JAG_F_SUBSET: case JAG_F_BOOL:
        if (!p->attr_mask) return fail(JAG_EINVAL, "dist_a needs attr_mask");
        break;
      default: return fail(JAG_EINVAL, "bad dist_a");
    }
  } else if (p->entry < 0 || p->entry >= p->n) {
    return fail(JAG_EINVAL, "entry out of range");
  }
  const int64_t n = p->n, d = p->d;
  if (!all_finite(p->x, (size_t)(n * d))) return fail(JAG_EINVAL, "non-finite base vector element");
  if (p->attr_f32 && !all_finite(p->attr_f32, (size_t)n)) return fail(JAG_EINVAL, "non-finite float attribute");
  if (prebuilt) {
    for (int64_t i = 0; i < n * p->R; ++i)
      if (p->graph[i] < -1 || p->graph[i] >= n) return fail(JAG_EINVAL, "graph id out of range");
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) return fail(JAG_ECUDA, "no CUDA device");
  if (p->device < 0 || p->device >= ndev) return fail(JAG_EINVAL, "device ordinal out of range");
  DeviceGuard dg(p->device);
  if (!dg.ok) return fail(JAG_ECUDA, "cudaSetDevice failed");

  auto *I = new jag_index();
  I->device = p->device;
  I->n = n; I->d = d; I->R = p->R; I->storage = p->storage;
  I->dist_a = p->dist_a;
  cudaError_t e;
  const int64_t xs = (d + 3) / 4 * 4;
  jag::DevIndex &ix = I->ix;
  ix.n = n; ix.d = (int32_t)d; ix.xs = xs; ix.nchunks = (int32_t)(xs / 4); ix.R = p->R; ix.dist_a = p->dist_a;
  auto bail = [&](jag_status s) { delete I; return s; };
#define API_TRY(x, what) do { e = (x); if (e != cudaSuccess) { jag_status s_ = cuda_fail(e, what); return bail(s_); } } while (0)
  API_TRY(I->alloc((void **)&I->x, sizeof(float) * (size_t)(n * xs)), "allocate vectors");
  API_TRY(cudaMemset(I->x, 0, sizeof(float) * (size_t)(n * xs)), "clear vectors");
  API_TRY(cudaMemcpy2D(I->x, sizeof(float) * xs, p->x, sizeof(float) * d, sizeof(float) * d, (size_t)n,
                       cudaMemcpyHostToDevice), "copy vectors");
  ix.x = I->x;
  {
    float *xn;
    unsigned int *dmax;
    API_TRY(I->alloc((void **)&xn, sizeof(float) * (size_t)n), "allocate row norms");
    API_TRY(I->alloc((void **)&dmax, sizeof(unsigned int)), "allocate row norms");
    API_TRY(jag::row_norms(ix, xn, dmax, &ix.xnorm_max, 0), "row norms");
    ix.xnorm = xn;
  }
  ix.fmt = p->storage;
  if (p->storage != JAG_VEC_F32) {
    const int64_t eb = p->storage == JAG_VEC_BF16 ? 2 : 1;
    ix.qbytes = (int32_t)((d * eb + 15) / 16 * 16);
    ix.qchunks = ix.qbytes / 16;
    uint8_t *xq;
    float *qs;
    API_TRY(I->alloc((void **)&xq, (size_t)(n * ix.qbytes)), "allocate stored rows");
    API_TRY(I->alloc((void **)&qs, sizeof(float) * (size_t)n), "allocate row scales");
    API_TRY(jag::quantize_rows(ix, p->storage, xq, qs, 0), "quantize rows");
    ix.xq = xq;
    ix.qscale = qs;
  }
  if (p->attr_i32) {
    int32_t *a, *sv, *si;
    API_TRY(I->alloc((void **)&a, 4 * (size_t)n), "allocate attr_i32");
    API_TRY(cudaMemcpy(a, p->attr_i32, 4 * (size_t)n, cudaMemcpyHostToDevice), "copy attr_i32");
    std::vector<int32_t> v, id;
    sorted_column(p->attr_i32, n, v, id);
    API_TRY(I->alloc((void **)&sv, 4 * (size_t)n), "allocate sorted column");
    API_TRY(I->alloc((void **)&si, 4 * (size_t)n), "allocate sorted column");
    API_TRY(cudaMemcpy(sv, v.data(), 4 * (size_t)n, cudaMemcpyHostToDevice), "copy sorted column");
    API_TRY(cudaMemcpy(si, id.data(), 4 * (size_t)n, cudaMemcpyHostToDevice), "copy sorted column");
    ix.a_i32 = a; ix.si32_val = sv; ix.si32_id = si;
  }
  if (p->attr_f32) {
    float *a, *sv;
    int32_t *si;
    API_TRY(I->alloc((void **)&a, 4 * (size_t)n), "allocate attr_f32");
    API_TRY(cudaMemcpy(a, p->attr_f32, 4 * (size_t)n, cudaMemcpyHostToDevice), "copy attr_f32");
    std::vector<float> v;
    std::vector<int32_t> id;
    sorted_column(p->attr_f32, n, v, id);
    API_TRY(I->alloc((void **)&sv, 4 * (size_t)n), "allocate sorted column");
    API_TRY(I->alloc((void **)&si, 4 * (size_t)n), "allocate sorted column");
    API_TRY(cudaMemcpy(sv, v.data(), 4 * (size_t)n, cudaMemcpyHostToDevice), "copy sorted column");
    API_TRY(cudaMemcpy(si, id.data(), 4 * (size_t)n, cudaMemcpyHostToDevice), "copy sorted column");
    ix.a_f32 = a; ix.sf32_val = sv; ix.sf32_id = si;
  }
  if (p->attr_mask) {
    uint64_t *a;
    API_TRY(I->alloc((void **)&a, 8 * (size_t)n), "allocate attr_mask");
    API_TRY(cudaMemcpy(a, p->attr_mask, 8 * (size_t)n, cudaMemcpyHostToDevice), "copy attr_mask");
    ix.a_mask = a;
    // posting lists per bit (CSR), for the exact scan of subset filters
    std::vector<int64_t> off(65, 0);
    for (int64_t i = 0; i < n; ++i)
      for (uint64_t v = p->attr_mask[i]; v; v &= v - 1) off[__builtin_ctzll(v) + 1] += 1;
    for (int j = 0; j < 64; ++j) off[j + 1] += off[j];
    std::vector<int32_t> ids((size_t)std::max<int64_t>(off[64], 1));
    std::vector<int64_t> fill(off.begin(), off.end() - 1);
    for (int64_t i = 0; i < n; ++i)
      for (uint64_t v = p->attr_mask[i]; v; v &= v - 1) ids[(size_t)fill[__builtin_ctzll(v)]++] = (int32_t)i;
    int64_t *doff;
    int32_t *dids;
    API_TRY(I->alloc((void **)&doff, sizeof(int64_t) * 65), "allocate posting lists");
    API_TRY(I->alloc((void **)&dids, sizeof(int32_t) * ids.size()), "allocate posting lists");
    API_TRY(cudaMemcpy(doff, off.data(), sizeof(int64_t) * 65, cudaMemcpyHostToDevice), "copy posting lists");
    API_TRY(cudaMemcpy(dids, ids.data(), sizeof(int32_t) * ids.size(), cudaMemcpyHostToDevice), "copy posting lists");
    ix.bit_off = doff;
    ix.bit_ids = dids;
  }
  API_TRY(I->alloc((void **)&I->graph, sizeof(int32_t) * (size_t)(n * p->R)), "allocate graph");
  ix.graph = I->graph;
  if (prebuilt) {
    API_TRY(cudaMemcpy(I->graph, p->graph, sizeof(int32_t) * (size_t)(n * p->R), cudaMemcpyHostToDevice),
            "copy graph");
    ix.entry = (int32_t)p->entry;
  } else {
    I->weighted = p->n_weights > 0 ? 1 : 0;
    I->nT = I->weighted ? p->n_weights : p->n_thresholds;
    API_TRY(I->alloc((void **)&I->thr, sizeof(uint32_t) * (size_t)(n * I->nT)), "allocate thresholds");
    jag::BuildLaunch B{};
    B.ix = ix;
    B.graph = I->graph;
    B.thr = I->thr;
    B.nT = I->nT;
    B.weighted = I->weighted;
    for (int i = 0; i < 8; ++i) B.mult[i] = i < p->n_weights ? p->weight_mult[i] : 0.0;
    for (int i = 0; i < 4; ++i) B.pct[i] = !I->weighted && i < I->nT ? p->threshold_pct[i] : 0;
    B.sample = p->sample_size;
    B.seed = p->seed;
    B.lb = p->l_b;
    B.alpha2 = (float)((double)p->alpha * (double)p->alpha);
    cudaStream_t st;
    API_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "create stream");
    B.stream = st;
    char msg[256] = {0};
    int32_t entry = 0;
    auto t0 = std::chrono::steady_clock::now();
    int rc = jag::run_build(B, &entry, msg, sizeof(msg));
    auto t1 = std::chrono::steady_clock::now();
    cudaStreamDestroy(st);
    if (rc != JAG_OK) { jag_status s_ = fail((jag_status)rc, "%s", msg); return bail(s_); }
    ix.entry = entry;
    I->build_seconds = std::chrono::duration<double>(t1 - t0).count();
  }
  {
    int32_t *ea_i32 = nullptr;
    float *ea_f32 = nullptr;
    uint64_t *ea_mask = nullptr;
    const size_t ne = (size_t)(n * p->R);
    if (ix.a_i32) API_TRY(I->alloc((void **)&ea_i32, 4 * ne), "allocate edge attributes");
    if (ix.a_f32) API_TRY(I->alloc((void **)&ea_f32, 4 * ne), "allocate edge attributes");
    if (ix.a_mask) API_TRY(I->alloc((void **)&ea_mask, 8 * ne), "allocate edge attributes");
    API_TRY(jag::build_edge_attrs(ix, ea_i32, ea_f32, ea_mask, 0), "edge attributes");
    ix.ea_i32 = ea_i32; ix.ea_f32 = ea_f32; ix.ea_mask = ea_mask;
  }
  API_TRY(cudaDeviceSynchronize(), "finish upload");
#undef API_TRY
  // Put the fixed scratch area of jag_search_noalloc in place on this device
  // now, while the caller still expects allocations (with lazy module loading
  // the area would otherwise be loaded by the first no-allocation search).
  // A failure here is not the build's: that search reports it.
  if (jag::noalloc_prepare(p->device) != cudaSuccess) cudaGetLastError();
  *out = I;
  return JAG_OK;
}

void jag_free(jag_index *idx) { delete idx; }

jag_status jag_get_info(const jag_index *idx, jag_info *out) {
  if (!idx || !out) return fail(JAG_EINVAL, "NULL argument");
  out->n = idx->n; out->d = idx->d; out->R = idx->R; out->storage = idx->storage;
  out->entry = idx->ix.entry; out->device_bytes = (int64_t)idx->device_bytes;
  out->build_seconds = idx->build_seconds; out->n_thresholds = idx->nT; out->dist_a = idx->dist_a;
  out->weighted = idx->weighted; out->reserved = 0;
  return JAG_OK;
}

jag_status jag_get_graph(const jag_index *idx, int32_t *host_out) {
  if (!idx || !host_out) return fail(JAG_EINVAL, "NULL argument");
  DeviceGuard dg(idx->device);
  cudaError_t e = cudaMemcpy(host_out, idx->graph, sizeof(int32_t) * (size_t)(idx->n * idx->R), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? JAG_OK : cuda_fail(e, "copy graph");
}

jag_status jag_get_thresholds(const jag_index *idx, uint32_t *host_out) {
  if (!idx || !host_out) return fail(JAG_EINVAL, "NULL argument");
  if (!idx->thr) return fail(JAG_EINVAL, "index graph was uploaded, not built");
  DeviceGuard dg(idx->device);
  cudaError_t e = cudaMemcpy(host_out, idx->thr, sizeof(uint32_t) * (size_t)(idx->n * idx->nT), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? JAG_OK : cuda_fail(e, "copy thresholds");
}

jag_status jag_get_stored_rows(const jag_index *idx, uint8_t *rows_out, float *scales_out, int32_t *row_bytes_out) {
  if (!idx) return fail(JAG_EINVAL, "NULL index");
  if (idx->ix.fmt == JAG_VEC_F32) return fail(JAG_EINVAL, "index stores fp32 rows");
  if (row_bytes_out) *row_bytes_out = idx->ix.qbytes;
  DeviceGuard dg(idx->device);
  cudaError_t e = cudaSuccess;
  if (rows_out) e = cudaMemcpy(rows_out, idx->ix.xq, (size_t)(idx->n * idx->ix.qbytes), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && scales_out)
    e = cudaMemcpy(scales_out, idx->ix.qscale, sizeof(float) * (size_t)idx->n, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? JAG_OK : cuda_fail(e, "copy stored rows");
}

static jag_status search_on(jag_index *idx, const jag_search_args *a, cudaStream_t stream) {
  const int hb = a->hash_bits ? a->hash_bits : jag::default_hash_bits();
  const int64_t s0 = a->s0 < 0 ? 2048 : a->s0;
  const int64_t cap = a->scan_cap <= 0 ? 8192 : a->scan_cap;
  const int scan_all = (a->flags & JAG_SEARCH_SCAN_ALL) ? 1 : 0;
  const jag::SearchScratch L0 = jag::search_scratch_layout(idx->ix, a->nq, a->aux_bytes, cap, a->k, a->beam, scan_all, s0, 1);
  Workspace *w = idx->workspace(stream);
  std::lock_guard<std::mutex> g(w->mu);
  cudaError_t e = ensure(w->buf, L0.total, stream);
  if (e != cudaSuccess) return cuda_fail(e, "allocate search scratch");
  jag::SearchLaunch L{};
  L.ix = idx->ix;
  L.queries = a->queries;
  L.d = (int32_t)idx->d;
  L.filters = a->filters;
  L.aux = a->filter_aux;
  L.aux_bytes = a->aux_bytes;
  L.nq = a->nq;
  L.k = a->k; L.ls = a->beam; L.hbits = hb; L.hbits_auto = a->hash_bits == 0;
  L.s0 = s0; L.cap = cap; L.scan_all = scan_all;
  L.out_ids = a->out_ids; L.out_dist = a->out_dist; L.counters = a->counters;
  jag::bind_scratch(L, L0, (uint8_t *)w->buf.ptr);
  if (a->policy) { L.policy = *a->policy; L.has_policy = 1; }
  L.fork_scan = 1;
  L.ev_begin = (cudaEvent_t)a->ev_graph_begin;
  L.ev_end = (cudaEvent_t)a->ev_graph_end;
  L.stream = stream;
  e = cudaMemsetAsync(L.status, 0, 4, stream);
  if (e == cudaSuccess) e = jag::run_search(L);
  if (e != cudaSuccess) return cuda_fail(e, "search launch");
  return JAG_OK;
}

jag_status jag_search(jag_index *idx, const jag_search_args *a) {
  g_err.clear();
  jag_status s = check_search_args(idx, a);
  if (s != JAG_OK) return s;
  DeviceGuard dg(idx->device);
  if (!dg.ok) return fail(JAG_ECUDA, "cudaSetDevice failed");
  return search_on(idx, a, (cudaStream_t)a->stream);
}

jag_status jag_query(jag_index *idx, const float *queries, const jag_filter *filters, const uint8_t *filter_aux,
                     int64_t aux_bytes, int64_t nq, int32_t k, int32_t beam, int32_t *out_ids, float *out_dist,
                     void *stream) {
  jag_search_args a{};
  a.queries = queries;
  a.filters = filters;
  a.filter_aux = filter_aux;
  a.aux_bytes = aux_bytes;
  a.nq = nq;
  a.k = k;
  a.beam = beam;
  a.out_ids = out_ids;
  a.out_dist = out_dist;
  a.stream = stream;
  a.s0 = -1;
  return jag_search(idx, &a);
}

jag_status jag_search_host(jag_index *idx, const jag_search_args *a) {
  g_err.clear();
  jag_status s = check_search_args(idx, a);
  if (s != JAG_OK) return s;
  DeviceGuard dg(idx->device);
  if (!dg.ok) return fail(JAG_ECUDA, "cudaSetDevice failed");
  HostStage &H = idx->host;
  std::lock_guard<std::mutex> g(H.mu);
  cudaError_t e = cudaSuccess;
  cudaStream_t st = (cudaStream_t)a->stream;
  if (!st) {
    if (!H.stream && (e = cudaStreamCreateWithFlags(&H.stream, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(e, "create stream");
    st = H.stream;
  }
  const size_t qb = sizeof(float) * (size_t)(a->nq * idx->d), fb = sizeof(jag_filter) * (size_t)a->nq;
  const size_t ob = sizeof(int32_t) * (size_t)(a->nq * a->k), db = sizeof(float) * (size_t)(a->nq * a->k);
  const size_t cb = a->counters ? sizeof(int32_t) * 4 * (size_t)a->nq : 0;
  if ((e = ensure(H.q, qb, st)) || (e = ensure(H.f, fb, st)) || (e = ensure(H.aux, (size_t)a->aux_bytes, st)) ||
      (e = ensure(H.ids, ob, st)) || (e = ensure(H.dist, db, st)) || (e = ensure(H.cnt, cb, st)))
    return cuda_fail(e, "allocate staging");
  if (a->nq > 0) {
    if ((e = cudaMemcpyAsync(H.q.ptr, a->queries, qb, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(H.f.ptr, a->filters, fb, cudaMemcpyHostToDevice, st)))
      return cuda_fail(e, "copy inputs");
  }
  if (a->aux_bytes > 0 && (e = cudaMemcpyAsync(H.aux.ptr, a->filter_aux, (size_t)a->aux_bytes, cudaMemcpyHostToDevice, st)))
    return cuda_fail(e, "copy filter aux");
  jag_search_args d = *a;
  d.queries = (const float *)H.q.ptr;
  d.filters = (const jag_filter *)H.f.ptr;
  d.filter_aux = a->aux_bytes > 0 ? (const uint8_t *)H.aux.ptr : nullptr;
  d.out_ids = (int32_t *)H.ids.ptr;
  d.out_dist = (float *)H.dist.ptr;
  d.counters = a->counters ? (int32_t *)H.cnt.ptr : nullptr;
  d.stream = st;
  s = search_on(idx, &d, st);
  if (s != JAG_OK) return s;
  if (a->nq > 0) {
    if ((e = cudaMemcpyAsync(a->out_ids, H.ids.ptr, ob, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaMemcpyAsync(a->out_dist, H.dist.ptr, db, cudaMemcpyDeviceToHost, st)))
      return cuda_fail(e, "copy outputs");
    if (cb && (e = cudaMemcpyAsync(a->counters, H.cnt.ptr, cb, cudaMemcpyDeviceToHost, st)))
      return cuda_fail(e, "copy counters");
  }
  uint32_t status = 0;
  Workspace *w = idx->workspace(st);
  if (w->buf.ptr) {
    const jag::SearchScratch L0 = jag::search_scratch_layout(idx->ix, a->nq, a->aux_bytes,
                                                             a->scan_cap <= 0 ? 8192 : a->scan_cap, a->k, a->beam,
                                                             (a->flags & JAG_SEARCH_SCAN_ALL) ? 1 : 0,
                                                             a->s0 < 0 ? 2048 : a->s0, 1);
    if ((e = cudaMemcpyAsync(&status, (uint8_t *)w->buf.ptr + L0.status, 4, cudaMemcpyDeviceToHost, st)))
      return cuda_fail(e, "read status");
  }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "search");
  if (status & jag::kErrTcTimeout) return fail(JAG_ETIMEOUT, "the exact scan's tensor-core wait timed out");
  if (status & jag::kErrBadFilter) return fail(JAG_EINVAL, "invalid filter record(s): their answers are padded");
  return JAG_OK;
}

}  // extern "C"
