// Continuous-batching server for quantised (int16) block-DCT planes.
//
// Requests (1-4 int16 coefficient planes, a dequantisation and a
// requantisation table per plane, one mask) arrive from any thread.  One worker thread:
//   * retires finished batches (CUDA event per batch): copies results to the
//     caller's buffers, frees their share of the HBM budget, records latency;
//   * admits waiting requests, in arrival order, while a batch slot is free
//     and their device memory fits in the HBM budget (first-fit arena);
//   * builds or reuses each request's operator: an LRU cache keyed by
//     (mask, anchor, boundary, n), FP64 build on its own stream, an event
//     marks it ready; operators used by an in-flight batch are never evicted;
//   * launches the batch on the slot's stream: one upload of the batch's
//     descriptors, quantisation tables and zeroed status word; for requests
//     whose planes are mapped page-locked memory, ONE host-direct grouped
//     kernel that reads and writes those planes over the host link itself
//     (no copies, no device memory); for the others, host -> HBM copies
//     (straight from page-locked buffers, else through pinned staging), ONE
//     persistent grouped kernel over their planes and HBM -> host copies.
//     Both kernels dequantise, filter and requantise in one pass.
// Several slots are in flight at once on separate streams, so requests that
// arrive while a batch runs are admitted as soon as a slot and memory free
// up, and their copies and kernels overlap the running batch on the device.
// Per-block arithmetic does not depend on the batch, so a request's result is
// the same alone or in any mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "apply_group.cuh"

namespace dctf {
namespace {

constexpr int kMaxPlanes = 4;
constexpr size_t kAlign = 256;
constexpr int kQBytes = 128;        // one quantisation table
// CTAs of a host-direct batch.  The host link bounds it; on the serving
// stream 64 CTAs sustained the most (42.4k req/s; 16: 37.6k, 32: 40.4k,
// 152: 42.3k with a longer tail), leaving SMs to the other batches in flight.
constexpr int kDirectCtas = 64;

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

size_t round_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator of byte ranges of one arena.
class Arena {
 public:
  void init(size_t size) {
    free_.clear();
    free_[0] = size;
    used_ = 0;
  }
  bool alloc(size_t bytes, size_t *off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0;
};

struct OpKey {
  std::vector<double> w;
  int mh, mw, ar, ac, boundary;
  bool operator==(const OpKey &o) const {
    return mh == o.mh && mw == o.mw && ar == o.ar && ac == o.ac && boundary == o.boundary &&
           w == o.w;
  }
  uint64_t hash() const {   // FNV-1a over the key's bytes
    uint64_t h = 1469598103934665603ull;
    auto mix = [&h](const void *p, size_t n) {
      const unsigned char *c = static_cast<const unsigned char *>(p);
      for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ull; }
    };
    mix(w.data(), w.size() * sizeof(double));
    const int v[5] = {mh, mw, ar, ac, boundary};
    mix(v, sizeof v);
    return h;
  }
};

struct OpEntry {
  OpKey key;
  dctf_operator *op = nullptr;
  cudaEvent_t ready = nullptr;
  int refs = 0;
  std::list<OpEntry *>::iterator lru;
};

struct Req {
  uint64_t ticket = 0;
  int nplanes = 0;
  const int16_t *in[kMaxPlanes] = {};
  int16_t *out[kMaxPlanes] = {};
  int64_t nblocks[kMaxPlanes] = {};
  uint16_t q[kMaxPlanes][64] = {};      // dequantisation table per plane
  uint16_t qout[kMaxPlanes][64] = {};   // requantisation table per plane
  OpKey key;
  double t_submit = 0, t_done = 0;
  // arena layout: [inputs][outputs], each plane 256-aligned (host-direct
  // requests take no device memory: bytes = 0)
  size_t off = 0, bytes = 0, in_bytes = 0, out_start = 0;
  size_t in_off[kMaxPlanes] = {}, out_off[kMaxPlanes] = {};
  const void *din[kMaxPlanes] = {};   // host-direct: device addresses of the planes
  void *dout[kMaxPlanes] = {};
  OpEntry *op = nullptr;
  dctf_status status = DCTF_OK;
  bool done = false;
  bool in_pinned = false;    // caller buffers already page-locked: copied by DMA directly
  bool out_pinned = false;
  bool direct = false;       // every plane mapped page-locked: the kernel does the I/O
  bool waited = false;       // did not fit the HBM budget at the head of the queue
};

// Page-locked (or registered) host memory can be the source / target of an
// asynchronous copy directly; anything else goes through the pinned staging.
bool is_pinned(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

// Host-direct eligibility: every plane's input and output 16-byte aligned
// and mapped, and no two of the request's buffers overlapping unless a plane
// is filtered in place (in == out).  Fills the device addresses.
bool direct_planes(Req *r) {
  for (int p = 0; p < r->nplanes; ++p) {
    const size_t len = (size_t)r->nblocks[p] * 128;
    if ((reinterpret_cast<uintptr_t>(r->in[p]) | reinterpret_cast<uintptr_t>(r->out[p])) & 15)
      return false;
    r->din[p] = mapped_host(r->in[p], len);
    r->dout[p] = mapped_host(r->out[p], len);
    if (r->din[p] == nullptr || r->dout[p] == nullptr) return false;
  }
  auto overlap = [](const void *a, size_t la, const void *b, size_t lb) {
    const char *x = static_cast<const char *>(a), *y = static_cast<const char *>(b);
    return x < y + lb && y < x + la;
  };
  for (int p = 0; p < r->nplanes; ++p) {
    const size_t lp = (size_t)r->nblocks[p] * 128;
    if (r->in[p] != r->out[p] && overlap(r->in[p], lp, r->out[p], lp)) return false;
    for (int q = p + 1; q < r->nplanes; ++q) {
      const size_t lq = (size_t)r->nblocks[q] * 128;
      if (overlap(r->in[p], lp, r->in[q], lq) || overlap(r->in[p], lp, r->out[q], lq) ||
          overlap(r->out[p], lp, r->in[q], lq) || overlap(r->out[p], lp, r->out[q], lq))
        return false;
    }
  }
  return true;
}

// Per-batch upload buffer (pinned on the host, mirrored on the device):
// [GroupItem x nitems][(q_in, q_out) tables x nitems][status word], packed
// per batch.
struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  GroupItem *h_items = nullptr;   // pinned
  GroupItem *d_items = nullptr;
  uint32_t *h_err = nullptr;      // pinned copy of the status word
  int cap = 0;
  bool busy = false;
  std::vector<Req *> reqs;
};

}  // namespace
}  // namespace dctf

struct dctf_server {
  dctf_server_cfg cfg;
  int device = 0;
  int sms = 0;
  char *d_arena = nullptr;
  char *h_arena = nullptr;
  dctf::Arena arena;
  std::vector<dctf::Slot> slots;
  std::unordered_multimap<uint64_t, dctf::OpEntry *> cache;
  std::list<dctf::OpEntry *> lru;       // front = most recent
  cudaStream_t build_stream = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<dctf::Req *> pending;
  std::unordered_map<uint64_t, dctf::Req *> live;
  uint64_t next_ticket = 1;
  std::thread worker;
  bool stop = false;
  // statistics (under mu)
  std::vector<double> lat_ms;
  uint64_t completed = 0, failed = 0, batches = 0, blocks = 0, hits = 0, misses = 0, builds = 0;
  uint64_t direct = 0, budget_waits = 0;
  size_t hbm_peak = 0;
  double t_first_submit = 0, t_last_done = 0;
  int max_batch_seen = 0;
};

namespace dctf {
namespace {

// Operator for a request: cached, else built on the build stream.
dctf_status get_op(dctf_server *s, Req *r) {
  const uint64_t h = r->key.hash();
  auto range = s->cache.equal_range(h);
  for (auto it = range.first; it != range.second; ++it) {
    if (it->second->key == r->key) {
      OpEntry *e = it->second;
      s->lru.splice(s->lru.begin(), s->lru, e->lru);
      ++e->refs;
      r->op = e;
      ++s->hits;
      return DCTF_OK;
    }
  }
  ++s->misses;
  // evict least recently used entries that no in-flight batch holds
  while ((int)s->cache.size() >= s->cfg.op_cache_capacity) {
    OpEntry *victim = nullptr;
    for (auto it = s->lru.rbegin(); it != s->lru.rend(); ++it)
      if ((*it)->refs == 0) { victim = *it; break; }
    if (victim == nullptr) break;
    auto rg = s->cache.equal_range(victim->key.hash());
    for (auto it = rg.first; it != rg.second; ++it)
      if (it->second == victim) { s->cache.erase(it); break; }
    s->lru.erase(victim->lru);
    if (victim->ready) cudaEventDestroy(victim->ready);
    dctf_release_operator(victim->op);
    delete victim;
  }
  ++s->builds;
  if (s->cfg.inject_build_failure_every > 0 &&
      s->builds % (uint64_t)s->cfg.inject_build_failure_every == 0)
    return set_error(DCTF_ECUDA, "injected operator build failure");
  OpEntry *e = new OpEntry();
  e->key = r->key;
  const int anchor[2] = {r->key.ar, r->key.ac};
  dctf_status st = dctf_build_operator(r->key.w.data(), r->key.mh, r->key.mw, anchor, 8,
                                       (dctf_boundary)r->key.boundary, s->build_stream, &e->op);
  if (st == DCTF_OK && cudaEventCreateWithFlags(&e->ready, cudaEventDisableTiming) != cudaSuccess)
    st = set_error(DCTF_ECUDA, "event create");
  if (st == DCTF_OK && cudaEventRecord(e->ready, s->build_stream) != cudaSuccess)
    st = set_error(DCTF_ECUDA, "event record");
  if (st != DCTF_OK) {
    if (e->op) dctf_release_operator(e->op);
    if (e->ready) cudaEventDestroy(e->ready);
    delete e;
    return st;
  }
  s->cache.emplace(h, e);
  s->lru.push_front(e);
  e->lru = s->lru.begin();
  e->refs = 1;
  r->op = e;
  return DCTF_OK;
}

void finish(dctf_server *s, Req *r, dctf_status st) {
  r->status = st;
  r->t_done = now_ms();
  r->done = true;
  if (st == DCTF_OK) {
    s->lat_ms.push_back(r->t_done - r->t_submit);
    ++s->completed;
    if (r->direct) ++s->direct;
    for (int p = 0; p < r->nplanes; ++p) s->blocks += r->nblocks[p];
  } else {
    ++s->failed;
  }
  s->t_last_done = r->t_done;
}

// Copy results out of finished slots and release their resources.
void retire(dctf_server *s) {
  for (Slot &sl : s->slots) {
    if (!sl.busy || cudaEventQuery(sl.done) != cudaSuccess) continue;
    const dctf_status kst =
        *sl.h_err == 0 ? DCTF_OK : set_error(DCTF_ETIMEOUT, "device wait timed out");
    for (Req *r : sl.reqs) {
      if (r->status == DCTF_OK && !r->out_pinned) {
        for (int p = 0; p < r->nplanes; ++p)
          memcpy(r->out[p], s->h_arena + r->out_off[p], (size_t)r->nblocks[p] * 128);
      }
      if (r->op) --r->op->refs;
      std::lock_guard<std::mutex> lk(s->mu);
      if (r->bytes > 0) s->arena.release(r->off, r->bytes);
      finish(s, r, r->status != DCTF_OK ? r->status : kst);
    }
    sl.reqs.clear();
    sl.busy = false;
    s->cv_done.notify_all();
  }
}

dctf_status launch_batch(dctf_server *s, Slot &sl, std::vector<Req *> &batch) {
  // descriptors: host-direct planes first, then staged planes; each group's
  // half_begin counts from its own start
  int nitems = 0, ndirect = 0;
  for (Req *r : batch) {
    r->status = get_op(s, r);
    if (r->status == DCTF_OK && r->direct) ndirect += r->nplanes;
    if (r->status == DCTF_OK) nitems += r->nplanes;
  }
  char *hb = reinterpret_cast<char *>(sl.h_items), *db = reinterpret_cast<char *>(sl.d_items);
  const size_t q0 = (size_t)nitems * sizeof(GroupItem);
  const size_t err_off = q0 + (size_t)nitems * 2 * kQBytes;
  uint32_t *d_err = reinterpret_cast<uint32_t *>(db + err_off);
  int id = 0, is = ndirect;
  int64_t hd = 0, hs = 0;
  cudaError_t e = cudaSuccess;
  for (Req *r : batch) {
    if (r->status != DCTF_OK) continue;
    if (!r->direct) {
      if (r->in_pinned) {
        for (int p = 0; p < r->nplanes && e == cudaSuccess; ++p)
          e = cudaMemcpyAsync(s->d_arena + r->in_off[p], r->in[p], (size_t)r->nblocks[p] * 128,
                              cudaMemcpyHostToDevice, sl.stream);
      } else {
        for (int p = 0; p < r->nplanes; ++p)
          memcpy(s->h_arena + r->in_off[p], r->in[p], (size_t)r->nblocks[p] * 128);
        e = cudaMemcpyAsync(s->d_arena + r->off, s->h_arena + r->off, r->in_bytes,
                            cudaMemcpyHostToDevice, sl.stream);
      }
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sl.stream, r->op->ready, 0);
    if (e != cudaSuccess) return cuda_error(e, "batch input copy");
    for (int p = 0; p < r->nplanes; ++p) {
      const int i = r->direct ? id++ : is++;
      GroupItem &gi = sl.h_items[i];
      memcpy(hb + q0 + (size_t)(2 * i) * kQBytes, r->q[p], kQBytes);
      memcpy(hb + q0 + (size_t)(2 * i + 1) * kQBytes, r->qout[p], kQBytes);
      const uint16_t *dq = reinterpret_cast<const uint16_t *>(db + q0 + (size_t)(2 * i) * kQBytes);
      const uint16_t *dqo = dq + 64;
      if (r->direct) {
        e = fill_group_item_host(&gi, r->op->op, r->din[p], r->dout[p], r->nblocks[p], dq, dqo);
        gi.half_begin = hd;
        hd += (r->nblocks[p] + 63) / 64;
      } else {
        e = fill_group_item(&gi, r->op->op, s->d_arena + r->in_off[p], s->d_arena + r->out_off[p],
                            r->nblocks[p], true, dq, dqo);
        gi.half_begin = hs;
        hs += (r->nblocks[p] + 63) / 64;
      }
      if (e != cudaSuccess) return cuda_error(e, "batch descriptor");
    }
  }
  *sl.h_err = 0;
  if (nitems > 0) {
    *reinterpret_cast<uint32_t *>(hb + err_off) = 0;
    e = cudaMemcpyAsync(db, hb, err_off + sizeof(uint32_t), cudaMemcpyHostToDevice, sl.stream);
    if (e == cudaSuccess && ndirect > 0)
      e = launch_apply_group_host(sl.d_items, ndirect, hd, kDirectCtas, d_err, sl.stream);
    if (e == cudaSuccess && nitems > ndirect)
      e = launch_apply_group(sl.d_items + ndirect, nullptr, nitems - ndirect, hs, true, s->sms, 2,
                             d_err, sl.stream);
    for (Req *r : batch) {
      if (e != cudaSuccess || r->status != DCTF_OK || r->direct) continue;
      if (r->out_pinned) {
        for (int p = 0; p < r->nplanes && e == cudaSuccess; ++p)
          e = cudaMemcpyAsync(r->out[p], s->d_arena + r->out_off[p], (size_t)r->nblocks[p] * 128,
                              cudaMemcpyDeviceToHost, sl.stream);
      } else {
        e = cudaMemcpyAsync(s->h_arena + r->out_start, s->d_arena + r->out_start,
                            r->bytes - (r->out_start - r->off), cudaMemcpyDeviceToHost, sl.stream);
      }
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(sl.h_err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, sl.stream);
    if (e != cudaSuccess) return cuda_error(e, "batch launch");
  }
  if (cudaEventRecord(sl.done, sl.stream) != cudaSuccess)
    return set_error(DCTF_ECUDA, "batch event");
  sl.reqs = batch;
  sl.busy = true;
  std::lock_guard<std::mutex> lk(s->mu);
  ++s->batches;
  s->max_batch_seen = std::max(s->max_batch_seen, (int)batch.size());
  return DCTF_OK;
}

void worker_loop(dctf_server *s) {
  cudaSetDevice(s->device);
  for (;;) {
    retire(s);
    Slot *free_slot = nullptr;
    bool any_busy = false;
    for (Slot &sl : s->slots) {
      if (sl.busy) any_busy = true;
      else if (!free_slot) free_slot = &sl;
    }
    std::vector<Req *> batch;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop && s->pending.empty() && !any_busy) break;
      if (free_slot) {
        // A batch holds its arena bytes until all of it has retired, so one
        // batch may take at most a quarter of the budget (a request larger
        // than that goes alone): several batches are then in flight, and one
        // batch's copies back overlap the next one's copies in and kernel.
        const size_t cap_bytes = s->cfg.hbm_budget_bytes / 4;
        int planes = 0;
        size_t batch_bytes = 0;
        while (!s->pending.empty() && (int)batch.size() < s->cfg.max_batch_requests) {
          Req *r = s->pending.front();
          if (planes + r->nplanes > free_slot->cap) break;
          if (!batch.empty() && r->bytes > 0 && batch_bytes + r->bytes > cap_bytes) break;
          if (r->bytes > 0 && !s->arena.alloc(r->bytes, &r->off)) {   // wait for memory
            if (!r->waited) { r->waited = true; ++s->budget_waits; }
            break;
          }
          s->hbm_peak = std::max(s->hbm_peak, s->arena.used());
          batch_bytes += r->bytes;
          s->pending.pop_front();
          planes += r->nplanes;
          batch.push_back(r);
        }
      }
      if (batch.empty()) {
        // nothing to admit: wait for a submit, or poll the running batches
        if (any_busy)
          s->cv_work.wait_for(lk, std::chrono::microseconds(20));
        else
          s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        continue;
      }
    }
    for (Req *r : batch) {   // arena offsets are known now
      if (r->direct) continue;
      size_t o = r->off;
      for (int p = 0; p < r->nplanes; ++p) { r->in_off[p] = o; o += round_up(r->nblocks[p] * 128); }
      r->in_bytes = o - r->off;
      r->out_start = o;
      for (int p = 0; p < r->nplanes; ++p) { r->out_off[p] = o; o += round_up(r->nblocks[p] * 128); }
    }
    dctf_status st = launch_batch(s, *free_slot, batch);
    if (st != DCTF_OK) {
      // a launch error: fail the batch's requests, keep serving
      cudaStreamSynchronize(free_slot->stream);
      for (Req *r : batch) {
        if (r->op) { --r->op->refs; r->op = nullptr; }
        if (r->status == DCTF_OK) r->status = st;
      }
      free_slot->busy = true;   // retire() finishes them
      free_slot->reqs = batch;
      *free_slot->h_err = 0;
      cudaEventRecord(free_slot->done, free_slot->stream);
    }
  }
}

size_t request_bytes(const dctf_request *rq) {
  size_t b = 0;
  for (int p = 0; p < rq->nplanes; ++p) b += 2 * round_up(rq->nblocks[p] * 128);
  return b;
}

}  // namespace
}  // namespace dctf

using namespace dctf;

extern "C" {

dctf_status dctf_server_create(const dctf_server_cfg *cfg, dctf_server **out) {
  if (out == nullptr || cfg == nullptr) return set_error(DCTF_EINVAL, "NULL argument");
  *out = nullptr;
  if (cfg->hbm_budget_bytes < (1 << 20) || cfg->max_inflight < 1 || cfg->max_inflight > 8 ||
      cfg->max_batch_requests < 1 || cfg->op_cache_capacity < 1)
    return set_error(DCTF_EINVAL, "bad server configuration");
  dctf_server *s = new (std::nothrow) dctf_server();
  if (s == nullptr) return set_error(DCTF_ENOMEM, "host allocation failed");
  s->cfg = *cfg;
  cudaError_t e = cudaGetDevice(&s->device);
  s->sms = sm_count(s->device);
  const size_t budget = round_up(cfg->hbm_budget_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_arena, budget);
  if (e == cudaSuccess) e = cudaHostAlloc(&s->h_arena, budget, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->build_stream, cudaStreamNonBlocking);
  s->arena.init(budget);
  const int cap = std::max(1, cfg->max_batch_requests) * kMaxPlanes;
  s->slots.resize(cfg->max_inflight);
  for (Slot &sl : s->slots) {
    if (e != cudaSuccess) break;
    sl.cap = cap;
    e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    const size_t ub = (size_t)cap * (sizeof(GroupItem) + 2 * kQBytes) + 256;
    if (e == cudaSuccess) e = cudaHostAlloc(&sl.h_items, ub, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(&sl.h_err, 64, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc(&sl.d_items, ub);
  }
  if (e != cudaSuccess) {
    dctf_server_destroy(s);
    return cuda_error(e, "server set-up");
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return DCTF_OK;
}

dctf_status dctf_server_submit(dctf_server *s, const dctf_request *rq, uint64_t *ticket) {
  if (s == nullptr || rq == nullptr || ticket == nullptr)
    return set_error(DCTF_EINVAL, "NULL argument");
  if (rq->nplanes < 1 || rq->nplanes > kMaxPlanes)
    return set_error(DCTF_EINVAL, "nplanes must be 1..4");
  for (int p = 0; p < rq->nplanes; ++p) {
    if (rq->in[p] == nullptr || rq->out[p] == nullptr || rq->q[p] == nullptr ||
        rq->nblocks[p] <= 0 || rq->nblocks[p] > ((int64_t)1 << 30))
      return set_error(DCTF_EINVAL, "plane %d: bad buffers or nblocks", p);
  }
  if (rq->mask == nullptr || rq->mh < 1 || rq->mw < 1 || rq->mh > 8 || rq->mw > 8 ||
      rq->anchor[0] < 0 || rq->anchor[0] >= rq->mh || rq->anchor[1] < 0 ||
      rq->anchor[1] >= rq->mw || (rq->boundary != DCTF_ZERO && rq->boundary != DCTF_REPLICATE))
    return set_error(DCTF_EINVAL, "bad mask, anchor or boundary");
  Req *r = new (std::nothrow) Req();
  if (r == nullptr) return set_error(DCTF_ENOMEM, "host allocation failed");
  r->nplanes = rq->nplanes;
  for (int p = 0; p < rq->nplanes; ++p) {
    r->in[p] = rq->in[p];
    r->out[p] = rq->out[p];
    r->nblocks[p] = rq->nblocks[p];
    memcpy(r->q[p], rq->q[p], 128);
    memcpy(r->qout[p], rq->q_out[p] != nullptr ? rq->q_out[p] : rq->q[p], 128);
  }
  r->key.w.assign(rq->mask, rq->mask + rq->mh * rq->mw);
  r->key.mh = rq->mh; r->key.mw = rq->mw;
  r->key.ar = rq->anchor[0]; r->key.ac = rq->anchor[1];
  r->key.boundary = rq->boundary;
  r->direct = !s->cfg.staged_only && direct_planes(r);
  r->bytes = r->direct ? 0 : request_bytes(rq);
  if (r->bytes > s->cfg.hbm_budget_bytes) {
    const size_t b = r->bytes;
    delete r;
    return set_error(DCTF_EBUDGET, "request needs %zu bytes of HBM, budget is %zu", b,
                     (size_t)s->cfg.hbm_budget_bytes);
  }
  r->in_pinned = r->out_pinned = true;
  for (int p = 0; p < rq->nplanes && !r->direct; ++p) {
    r->in_pinned = r->in_pinned && is_pinned(rq->in[p]);
    r->out_pinned = r->out_pinned && is_pinned(rq->out[p]);
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) { delete r; return set_error(DCTF_EINVAL, "server is stopping"); }
    r->ticket = s->next_ticket++;
    r->t_submit = now_ms();
    if (s->t_first_submit == 0) s->t_first_submit = r->t_submit;
    s->live[r->ticket] = r;
    s->pending.push_back(r);
  }
  s->cv_work.notify_one();
  *ticket = r->ticket;
  return DCTF_OK;
}

dctf_status dctf_server_wait(dctf_server *s, uint64_t ticket, int timeout_ms) {
  if (s == nullptr) return set_error(DCTF_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->live.find(ticket);
  if (it == s->live.end()) return set_error(DCTF_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
  Req *r = it->second;
  const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                      [r] { return r->done; });
  if (!ok) return set_error(DCTF_ETIMEOUT, "request %llu not finished after %d ms",
                            (unsigned long long)ticket, timeout_ms);
  const dctf_status st = r->status;
  s->live.erase(it);
  delete r;
  if (st != DCTF_OK) return set_error(st, "request %llu failed", (unsigned long long)ticket);
  return DCTF_OK;
}

dctf_status dctf_server_stats(dctf_server *s, dctf_stats *out) {
  if (s == nullptr || out == nullptr) return set_error(DCTF_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  memset(out, 0, sizeof *out);
  std::vector<double> v = s->lat_ms;
  std::sort(v.begin(), v.end());
  if (!v.empty()) {
    out->p50_ms = v[(v.size() - 1) / 2];
    out->p99_ms = v[(size_t)((v.size() - 1) * 0.99)];
    out->max_ms = v.back();
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_ms = sum / v.size();
  }
  out->completed = s->completed;
  out->failed = s->failed;
  out->batches = s->batches;
  out->blocks = s->blocks;
  out->cache_hits = s->hits;
  out->cache_misses = s->misses;
  out->max_batch_requests_seen = s->max_batch_seen;
  out->wall_s = s->t_last_done > s->t_first_submit ? (s->t_last_done - s->t_first_submit) / 1e3 : 0;
  out->hbm_in_use = s->arena.used();
  out->direct_requests = s->direct;
  out->budget_waits = s->budget_waits;
  out->hbm_peak = s->hbm_peak;
  return DCTF_OK;
}

dctf_status dctf_server_reset_stats(dctf_server *s) {
  if (s == nullptr) return set_error(DCTF_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  s->lat_ms.clear();
  s->completed = s->failed = s->batches = s->blocks = s->hits = s->misses = 0;
  s->direct = s->budget_waits = 0;
  s->hbm_peak = s->arena.used();
  s->t_first_submit = s->t_last_done = 0;
  s->max_batch_seen = 0;
  return DCTF_OK;
}

void dctf_server_destroy(dctf_server *s) {
  if (s == nullptr) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto &kv : s->live) delete kv.second;
  for (OpEntry *e : s->lru) {
    if (e->ready) cudaEventDestroy(e->ready);
    dctf_release_operator(e->op);
    delete e;
  }
  for (Slot &sl : s->slots) {
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.h_items) cudaFreeHost(sl.h_items);
    if (sl.h_err) cudaFreeHost(sl.h_err);
    if (sl.d_items) cudaFree(sl.d_items);
  }
  if (s->build_stream) cudaStreamDestroy(s->build_stream);
  if (s->d_arena) cudaFree(s->d_arena);
  if (s->h_arena) cudaFreeHost(s->h_arena);
  delete s;
}

}  // extern "C"
