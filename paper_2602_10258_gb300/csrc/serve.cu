// Host side of the serve loop: admission (ring slots, host arena, device
// table budget), publication of requests to the device loop through mapped
// host memory, collection of answers, relaunch of the loop after an idle
// exit, and an open-loop replay driver for latency measurements.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "launch.h"
#include "serve_core.cuh"

namespace jag {
namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int64_t align16(int64_t v) { return (v + 15) & ~int64_t(15); }
int64_t align8(int64_t v) { return (v + 7) & ~int64_t(7); }

// Byte ring over [0, cap): allocations are handed out in order, released in
// any order; the space of the oldest live allocation bounds the free space.
// An allocation that does not fit before the end wraps to 0 and also holds
// the unused end, which it gives back when released.
class RingAlloc {
 public:
  void init(int64_t cap) { cap_ = cap; head_ = 0; spans_.clear(); }

  // Offset, -1 if there is no room now, -2 if len can never fit.
  int64_t alloc(int64_t len, uint64_t owner) {
    if (len > cap_) return -2;
    if (len == 0) return 0;
    if (spans_.empty()) {
      head_ = len;
      spans_.push_back({owner, 0, len, false});
      return 0;
    }
    const int64_t tail = spans_.front().start;
    if (head_ > tail) {
      if (cap_ - head_ >= len) return take(head_, len, owner);
      if (tail >= len) {
        if (cap_ > head_) spans_.push_back({owner, head_, cap_ - head_, false});
        head_ = 0;
        return take(0, len, owner);
      }
      return -1;
    }
    if (head_ < tail && tail - head_ >= len) return take(head_, len, owner);
    return -1;
  }

  void release(uint64_t owner) {
    for (auto &s : spans_)
      if (s.owner == owner) s.freed = true;
    while (!spans_.empty() && spans_.front().freed) spans_.pop_front();
    if (spans_.empty()) head_ = 0;
  }

 private:
  struct Span {
    uint64_t owner;
    int64_t start, len;
    bool freed;
  };
  int64_t take(int64_t off, int64_t len, uint64_t owner) {
    spans_.push_back({owner, off, len, false});
    head_ = off + len;
    return off;
  }
  int64_t cap_ = 0, head_ = 0;
  std::deque<Span> spans_;
};

}  // namespace
}  // namespace jag

using namespace jag;

struct jag_server {
  jag_index *idx = nullptr;
  int device = 0, fmt = JAG_VEC_F32, ctas = 0, grid = 0;
  int64_t d = 0;
  int32_t k = 0, slots = 0;
  int64_t qcap = 0, arena_bytes = 0, lut_bytes = 0;
  ServeArgs args{};
  cudaStream_t stream = nullptr, aux_stream = nullptr;
  // mapped host memory (host pointers)
  ServeCtl *ctl = nullptr;
  ServeReq *ring = nullptr;
  ServeDone *done = nullptr;
  uint32_t *qmap = nullptr;
  uint8_t *arena = nullptr;
  void *host_block = nullptr;
  // device memory
  void *dev_block = nullptr;
  uint8_t *lut = nullptr;
  // bookkeeping
  RingAlloc arena_alloc, lut_alloc;
  std::vector<int32_t> free_slots;
  struct Req {
    int32_t slot, nq;
    int64_t ids_off, dist_off;
    double submit;
    uint64_t qbase;
  };
  std::unordered_map<uint64_t, Req> reqs;
  // first query index of every uncollected request (the query map's live
  // window starts at the smallest)
  std::map<uint64_t, uint64_t> open_base;
  uint64_t next_ticket = 1, published = 0;
  int64_t held_queries = 0, launches = 0;
  bool launched = false;
  std::mutex mu;
};

namespace {

// Launch the device loop unless it is running (call with mu held).
jag_status ensure_running(jag_server *s) {
  if (s->launched) {
    const cudaError_t q = cudaStreamQuery(s->stream);
    if (q == cudaErrorNotReady) return JAG_OK;
    if (q != cudaSuccess) return set_error(JAG_ECUDA, cudaGetErrorString(q));
  }
  cudaError_t e;
  if (s->fmt == JAG_VEC_F32) e = launch_serve_fmt<JAG_VEC_F32>(s->args, s->ctas, s->stream, &s->grid);
  else if (s->fmt == JAG_VEC_BF16) e = launch_serve_fmt<JAG_VEC_BF16>(s->args, s->ctas, s->stream, &s->grid);
  else e = launch_serve_fmt<JAG_VEC_FP8>(s->args, s->ctas, s->stream, &s->grid);
  if (e != cudaSuccess) return set_error(JAG_ECUDA, cudaGetErrorString(e));
  s->launched = true;
  ++s->launches;
  return JAG_OK;
}

// Repacked size of the boolean tables of a request's filters.
int64_t packed_aux_bytes(const jag_filter *f, int32_t nq, const uint8_t *aux, int64_t aux_bytes) {
  int64_t b = 0;
  for (int32_t i = 0; i < nq; ++i) {
    if (f[i].kind != JAG_F_BOOL) continue;
    const int m = __builtin_popcountll(f[i].payload);
    if (m > 16 || !aux || f[i].aux_off < 0) continue;
    const int64_t tb = std::max<int64_t>(1, ((int64_t)1 << m) / 8);
    if (f[i].aux_off + tb > aux_bytes) continue;
    b += align8(tb);
  }
  return b;
}

enum Admit { kAdmitted, kNoRoom, kNever };

// Try to admit one request (mu held).  On success fills *ticket.
Admit try_admit(jag_server *s, const float *queries, const jag_filter *filters, const uint8_t *aux,
                int64_t aux_bytes, int32_t nq, uint64_t *ticket, double submit) {
  const int64_t auxc = packed_aux_bytes(filters, nq, aux, aux_bytes);
  const int64_t qb = align16((int64_t)nq * s->d * 4), fb = align16((int64_t)nq * 16), ab = align16(auxc);
  const int64_t ob = align16((int64_t)nq * s->k * 4);
  const int64_t total = qb + fb + ab + 2 * ob;
  if (nq > s->qcap || total > s->arena_bytes || auxc * 8 > s->lut_bytes) return kNever;
  // the query map is a ring over query indices: a new request's entries must
  // not reach those of the oldest request still open, which may be claimed
  // by a warp that has not read them yet
  const uint64_t oldest = s->open_base.empty() ? s->published : s->open_base.begin()->first;
  if (s->free_slots.empty() || s->held_queries + nq > s->qcap || s->published + nq - oldest > (uint64_t)s->qcap)
    return kNoRoom;
  const uint64_t t = s->next_ticket;
  const int64_t off = s->arena_alloc.alloc(total, t);
  if (off < 0) return off == -2 ? kNever : kNoRoom;
  const int64_t loff = s->lut_alloc.alloc(auxc * 8, t);
  if (loff < 0) {
    s->arena_alloc.release(t);
    return loff == -2 ? kNever : kNoRoom;
  }
  ++s->next_ticket;
  const int32_t slot = s->free_slots.back();
  s->free_slots.pop_back();
  uint8_t *base = s->arena + off;
  std::memcpy(base, queries, (size_t)nq * s->d * 4);
  jag_filter *fo = reinterpret_cast<jag_filter *>(base + qb);
  uint8_t *ao = base + qb + fb;
  int64_t apos = 0;
  for (int32_t i = 0; i < nq; ++i) {
    fo[i] = filters[i];
    if (filters[i].kind != JAG_F_BOOL) continue;
    const int m = __builtin_popcountll(filters[i].payload);
    const int64_t tb = m <= 16 ? std::max<int64_t>(1, ((int64_t)1 << m) / 8) : 0;
    if (m > 16 || !aux || filters[i].aux_off < 0 || filters[i].aux_off + tb > aux_bytes) {
      fo[i].aux_off = -1;   // rejected on the device: answers padded, status bit set
      continue;
    }
    std::memcpy(ao + apos, aux + filters[i].aux_off, (size_t)tb);
    fo[i].aux_off = (int32_t)apos;
    apos += align8(tb);
  }
  ServeReq r{};
  r.ticket = t;
  r.qbase = (int64_t)s->published;
  r.nq = nq;
  r.q_off = off;
  r.f_off = off + qb;
  r.aux_off = off + qb + fb;
  r.aux_bytes = auxc;
  r.ids_off = off + qb + fb + ab;
  r.dist_off = r.ids_off + ob;
  r.lut_off = loff;
  s->ring[slot] = r;
  for (int32_t i = 0; i < nq; ++i) s->qmap[(s->published + i) % (uint64_t)s->qcap] = (uint32_t)slot;
  s->held_queries += nq;
  s->reqs[t] = {slot, nq, r.ids_off, r.dist_off, submit, s->published};
  s->open_base[s->published] = t;
  s->published += nq;
  __atomic_store_n(&s->ctl->published, (unsigned long long)s->published, __ATOMIC_RELEASE);
  *ticket = t;
  return kAdmitted;
}

bool is_done(const jag_server *s, int32_t slot, uint64_t ticket) {
  return __atomic_load_n(&s->done[slot].ticket, __ATOMIC_ACQUIRE) == ticket;
}

// Copy out the answers of a completed request and release its space (mu held).
void collect(jag_server *s, uint64_t ticket, int32_t *ids, float *dist, jag_serve_timing *tm, double seen) {
  const jag_server::Req r = s->reqs[ticket];
  const size_t ob = (size_t)r.nq * s->k;
  if (ids) std::memcpy(ids, s->arena + r.ids_off, ob * 4);
  if (dist) std::memcpy(dist, s->arena + r.dist_off, ob * 4);
  if (tm) {
    const ServeDone &dn = s->done[r.slot];
    tm->submit_s = r.submit;
    tm->done_s = seen;
    tm->device_s = (double)(dn.t_end - dn.t_first) * 1e-9;
    tm->status = dn.status;
    tm->reserved = 0;
  }
  s->arena_alloc.release(ticket);
  s->lut_alloc.release(ticket);
  s->free_slots.push_back(r.slot);
  s->held_queries -= r.nq;
  s->open_base.erase(r.qbase);
  s->reqs.erase(ticket);
}

}  // namespace

extern "C" {

JAG_API jag_status jag_serve_start(jag_index *idx, const jag_serve_params *p, jag_server **out) {
  if (!idx || !p || !out) return set_error(JAG_EINVAL, "NULL index, params or out");
  *out = nullptr;
  jag_search_args a{};
  a.k = p->k;
  a.beam = p->beam;
  a.hash_bits = p->hash_bits;
  a.policy = p->policy;
  if (jag_status st = check_search(idx, &a)) return st;
  if (p->beam > 256) return set_error(JAG_EINVAL, "the serve loop takes beams of at most 256");
  if (p->policy && (p->policy->mode == JAG_POLICY_FORCED || p->policy->forced || p->policy->features ||
                    p->policy->decisions))
    return set_error(JAG_EINVAL, "serving takes a LEARNED or PLAIN policy without per-query buffers");
  if (p->max_requests < 0 || p->max_requests > 65536) return set_error(JAG_EINVAL, "max_requests must be in [0, 65536]");
  if (p->max_queries < 0 || p->arena_bytes < 0 || p->lut_bytes < 0 || p->ctas < 0 || !(p->idle_exit_s >= 0.0))
    return set_error(JAG_EINVAL, "negative size or time");
  DevIndex ix;
  int device;
  index_view(idx, &ix, &device);
  if (ix.nchunks > 64) return set_error(JAG_EUNSUPPORTED, "serving supports rows of at most 1 KiB (d <= 256)");
  const int hb = p->hash_bits ? p->hash_bits : 10;
  if (ix.fmt != JAG_VEC_F32 && hb < 8) return set_error(JAG_EINVAL, "BF16 / FP8 serving needs hash_bits >= 8");
  jag_server *s = new jag_server();
  s->idx = idx;
  s->device = device;
  s->fmt = ix.fmt;
  s->d = ix.d;
  s->k = p->k;
  s->slots = p->max_requests ? p->max_requests : 1024;
  s->qcap = p->max_queries ? p->max_queries : 65536;
  s->arena_bytes = p->arena_bytes ? p->arena_bytes
                                  : s->qcap * (align16(s->d * 4) + 16 + 64 + 2 * align16((int64_t)s->k * 4)) +
                                        (int64_t)s->slots * 80;
  s->lut_bytes = p->lut_bytes ? p->lut_bytes : ((int64_t)16 << 20);
  s->ctas = p->ctas;
  auto fail_free = [&](jag_status st, const char *msg) {
    if (s->host_block) cudaFreeHost(s->host_block);
    if (s->dev_block) cudaFree(s->dev_block);
    if (s->lut) cudaFree(s->lut);
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->aux_stream) cudaStreamDestroy(s->aux_stream);
    delete s;
    return set_error(st, msg);
  };
  if (cudaSetDevice(device) != cudaSuccess) return fail_free(JAG_ECUDA, "cudaSetDevice failed");
  // mapped host block: control words, ring, completion records, query map, arena
  const size_t o_ring = 256, o_done = o_ring + align16(sizeof(ServeReq) * s->slots);
  const size_t o_qmap = o_done + align16(sizeof(ServeDone) * s->slots);
  const size_t o_arena = (o_qmap + 4 * (size_t)s->qcap + 255) & ~size_t(255);
  const size_t hbytes = o_arena + (size_t)s->arena_bytes;
  if (cudaHostAlloc(&s->host_block, hbytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
    s->host_block = nullptr;
    return fail_free(JAG_ENOMEM, "cannot allocate the pinned serving arena");
  }
  std::memset(s->host_block, 0, o_arena);
  uint8_t *hb8 = static_cast<uint8_t *>(s->host_block), *db8 = nullptr;
  if (cudaHostGetDevicePointer((void **)&db8, s->host_block, 0) != cudaSuccess)
    return fail_free(JAG_ECUDA, "cannot map the serving arena");
  s->ctl = reinterpret_cast<ServeCtl *>(hb8);
  s->ring = reinterpret_cast<ServeReq *>(hb8 + o_ring);
  s->done = reinterpret_cast<ServeDone *>(hb8 + o_done);
  s->qmap = reinterpret_cast<uint32_t *>(hb8 + o_qmap);
  s->arena = hb8 + o_arena;
  // device block: loop state, per-slot counters, status, first-claim times
  const size_t d_cnt = 256, d_status = d_cnt + align16(4 * (size_t)s->slots);
  const size_t d_first = d_status + align16(4 * (size_t)s->slots);
  const size_t dbytes = d_first + 8 * (size_t)s->slots;
  if (cudaMalloc(&s->dev_block, dbytes) != cudaSuccess) {
    s->dev_block = nullptr;
    return fail_free(JAG_ENOMEM, "cannot allocate the serving state");
  }
  if (cudaMalloc((void **)&s->lut, (size_t)std::max<int64_t>(s->lut_bytes, 256)) != cudaSuccess) {
    s->lut = nullptr;
    return fail_free(JAG_ENOMEM, "cannot allocate the boolean table budget");
  }
  if (cudaMemset(s->dev_block, 0, dbytes) != cudaSuccess) return fail_free(JAG_ECUDA, "cudaMemset failed");
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->aux_stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail_free(JAG_ECUDA, "cannot create the serving streams");
  uint8_t *dv = static_cast<uint8_t *>(s->dev_block);
  ServeArgs &g = s->args;
  g.ix = ix;
  g.d = (int)ix.d;
  g.k = p->k;
  g.ls = p->beam;
  g.hbits = hb;
  g.s0 = p->s0 < 0 ? 2048 : p->s0;
  g.cap = p->scan_cap <= 0 ? 8192 : p->scan_cap;
  g.ctl = reinterpret_cast<const ServeCtl *>(db8);
  g.ring = reinterpret_cast<const ServeReq *>(db8 + o_ring);
  g.done = reinterpret_cast<ServeDone *>(db8 + o_done);
  g.qmap = reinterpret_cast<const uint32_t *>(db8 + o_qmap);
  g.qcap = s->qcap;
  g.arena = db8 + o_arena;
  g.lut = s->lut;
  g.dev = reinterpret_cast<ServeDev *>(dv);
  g.done_cnt = reinterpret_cast<int32_t *>(dv + d_cnt);
  g.req_status = reinterpret_cast<uint32_t *>(dv + d_status);
  g.t_first = reinterpret_cast<unsigned long long *>(dv + d_first);
  g.nslots = s->slots;
  g.idle_ns = (unsigned long long)((p->idle_exit_s > 0.0 ? p->idle_exit_s : 1.0) * 1e9);
  g.has_policy = p->policy && p->policy->mode == JAG_POLICY_LEARNED ? 1 : 0;
  if (g.has_policy) g.pol = *p->policy;
  s->arena_alloc.init(s->arena_bytes);
  s->lut_alloc.init(s->lut_bytes);
  for (int32_t i = s->slots - 1; i >= 0; --i) s->free_slots.push_back(i);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (jag_status st = ensure_running(s)) {
      const std::string msg = jag_last_error();
      return fail_free(st, msg.c_str());
    }
  }
  *out = s;
  return JAG_OK;
}

JAG_API jag_status jag_serve_submit(jag_server *s, const float *queries, const jag_filter *filters,
                                    const uint8_t *aux, int64_t aux_bytes, int32_t nq, double timeout_s,
                                    uint64_t *ticket) {
  if (!s || !queries || !filters || !ticket || nq < 1 || aux_bytes < 0 || !(timeout_s >= 0.0))
    return set_error(JAG_EINVAL, "bad serve_submit arguments");
  const double t0 = now_s();
  for (;;) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      const Admit r = try_admit(s, queries, filters, aux, aux_bytes, nq, ticket, t0);
      if (r == kNever) return set_error(JAG_EINVAL, "request can never fit the serving budgets");
      if (r == kAdmitted) {
        cudaSetDevice(s->device);
        return ensure_running(s);
      }
    }
    if (now_s() - t0 >= timeout_s) return set_error(JAG_ETIMEOUT, "no room for the request in time");
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

JAG_API jag_status jag_serve_wait(jag_server *s, uint64_t ticket, int32_t *ids, float *dist, jag_serve_timing *t,
                                  double timeout_s) {
  if (!s || !(timeout_s >= 0.0)) return set_error(JAG_EINVAL, "bad serve_wait arguments");
  int32_t slot;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(JAG_EINVAL, "unknown ticket");
    slot = it->second.slot;
  }
  const double t0 = now_s();
  double last_check = t0;
  for (;;) {
    if (is_done(s, slot, ticket)) {
      const double seen = now_s();
      std::lock_guard<std::mutex> lk(s->mu);
      collect(s, ticket, ids, dist, t, seen);
      return JAG_OK;
    }
    const double now = now_s();
    if (now - t0 >= timeout_s) return set_error(JAG_ETIMEOUT, "request not complete in time");
    if (now - last_check > 1e-3) {   // the loop may have exited idle just before this request arrived
      std::lock_guard<std::mutex> lk(s->mu);
      cudaSetDevice(s->device);
      if (jag_status st = ensure_running(s)) return st;
      last_check = now;
    }
    std::this_thread::yield();
  }
}

JAG_API jag_status jag_serve_info(const jag_server *s, int64_t *launches, int64_t *queries_done) {
  if (!s) return set_error(JAG_EINVAL, "server is NULL");
  jag_server *m = const_cast<jag_server *>(s);
  std::lock_guard<std::mutex> lk(m->mu);
  if (launches) *launches = m->launches;
  if (queries_done) {
    unsigned long long v = 0;
    cudaSetDevice(m->device);
    cudaError_t e = cudaMemcpyAsync(&v, &m->args.dev->queries_done, sizeof(v), cudaMemcpyDeviceToHost, m->aux_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->aux_stream);
    if (e != cudaSuccess) return set_error(JAG_ECUDA, cudaGetErrorString(e));
    *queries_done = (int64_t)v;
  }
  return JAG_OK;
}

JAG_API jag_status jag_serve_stop(jag_server *s) {
  if (!s) return JAG_OK;
  cudaSetDevice(s->device);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    bool pending = false;
    for (auto &kv : s->reqs)
      if (!is_done(s, kv.second.slot, kv.first)) pending = true;
    if (pending) ensure_running(s);
    __atomic_store_n(&s->ctl->stop, 1u, __ATOMIC_RELEASE);
  }
  const double t0 = now_s();
  for (;;) {
    const cudaError_t q = cudaStreamQuery(s->stream);
    if (q != cudaErrorNotReady) break;
    if (now_s() - t0 > 60.0) return set_error(JAG_ETIMEOUT, "serve loop did not finish within 60 s");
    std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
  cudaFreeHost(s->host_block);
  cudaFree(s->dev_block);
  cudaFree(s->lut);
  cudaStreamDestroy(s->stream);
  cudaStreamDestroy(s->aux_stream);
  delete s;
  return JAG_OK;
}

JAG_API jag_status jag_serve_replay(jag_server *s, int64_t n_req, const double *arrival_s, const int32_t *sizes,
                                    const int64_t *first, const float *queries, const jag_filter *filters,
                                    const uint8_t *aux, int64_t aux_bytes, int32_t *ids, float *dist,
                                    double *latency_s, double *device_s, double timeout_s) {
  if (!s || n_req < 0 || (n_req > 0 && (!arrival_s || !sizes || !first || !queries || !filters)) ||
      !(timeout_s > 0.0))
    return set_error(JAG_EINVAL, "bad serve_replay arguments");
  for (int64_t r = 0; r < n_req; ++r)
    if (sizes[r] < 1 || first[r] < 0 || (r > 0 && arrival_s[r] < arrival_s[r - 1]))
      return set_error(JAG_EINVAL, "bad request sizes, rows or arrival order");
  cudaSetDevice(s->device);
  struct Open {
    int64_t r;
    uint64_t ticket;
    int32_t slot;
  };
  std::deque<Open> open;
  const double start = now_s();
  double last_check = start;
  int64_t next = 0, finished = 0;
  while (finished < n_req) {
    const double now = now_s();
    if (now - start > timeout_s) return set_error(JAG_ETIMEOUT, "replay did not finish in time");
    bool progress = false;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      // arrivals that are due, in order, while there is room (the loop is
      // checked once for the whole group)
      bool admitted = false;
      while (next < n_req && now >= start + arrival_s[next]) {
        uint64_t t;
        const int64_t row = first[next];
        const Admit a = try_admit(s, queries + row * s->d, filters + row, aux, aux_bytes, sizes[next], &t,
                                  start + arrival_s[next]);
        if (a == kNever) return set_error(JAG_EINVAL, "a request can never fit the serving budgets");
        if (a == kNoRoom) break;
        open.push_back({next, t, s->reqs[t].slot});
        ++next;
        progress = admitted = true;
      }
      if (admitted)
        if (jag_status st = ensure_running(s)) return st;
      // completions, in any order
      for (auto it = open.begin(); it != open.end();) {
        if (!is_done(s, it->slot, it->ticket)) { ++it; continue; }
        const double seen = now_s();
        const int64_t row = first[it->r];
        jag_serve_timing tm;
        collect(s, it->ticket, ids ? ids + row * s->k : nullptr, dist ? dist + row * s->k : nullptr, &tm, seen);
        if (latency_s) latency_s[it->r] = seen - (start + arrival_s[it->r]);
        if (device_s) device_s[it->r] = tm.device_s;
        ++finished;
        progress = true;
        it = open.erase(it);
      }
      if (!open.empty() && now - last_check > 1e-3) {
        if (jag_status st = ensure_running(s)) return st;
        last_check = now;
      }
    }
    if (!progress) std::this_thread::yield();
  }
  return JAG_OK;
}

}  // extern "C"
