// server.cu — the served form: a request loop over resident time series. The paper's setting
// is in-situ compression of simulation output as it is produced (§I), one variable after
// another, timestep after timestep (§IV.D). Here a server owns one device arena supplied by
// the caller and keeps, for every series, the last reconstruction (the prev of its next
// compression, Eq. 4 uses R_{i-1}), the reconstruction before it and the latest blob resident
// in HBM; clients submit compress requests (the next timestep, from pinned host memory) and
// decompress requests (all or part of the latest timestep) from any thread and poll
// completions.
//
// Scheduling: requests of one series run one at a time in submission order (a compression
// changes the series' state). Across series the oldest runnable request is started whenever a
// slot (one CUDA stream) is free and its transient buffers fit in the arena (admission by free
// HBM, first-fit, 256-byte granules). A younger request may start ahead of an older one that
// does not fit only if the older one still fits afterwards, so large requests are not starved.
// A worker thread issues the copies and kernels and polls CUDA events; nothing blocks a client.
// With dry_run set no CUDA call is made: every stage of a request takes dry_run_us, which
// exercises the scheduling logic on a host without a GPU.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "launch.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr size_t kGranule = 256;
constexpr size_t kNone = ~(size_t)0;
constexpr int kMaxSlots = 64;

size_t granules(size_t b) { return (std::max<size_t>(b, 1) + kGranule - 1) / kGranule * kGranule; }

// Allocator over [0, size) with coalescing of freed ranges. Transient buffers are placed
// first-fit from the bottom, long-lived ones (a series' resident buffers) from the top, so that
// the free space between them stays in one piece.
class Arena {
 public:
  explicit Arena(size_t size) : size_(size / kGranule * kGranule) {
    if (size_) free_[0] = size_;
  }
  size_t alloc(size_t bytes, bool high = false) {
    const size_t off = place(free_, granules(bytes), high);
    if (off != kNone) {
      used_ += granules(bytes);
      peak_ = std::max(peak_, used_);
    }
    return off;
  }
  void release(size_t off, size_t bytes) {
    bytes = granules(bytes);
    used_ -= bytes;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + bytes == next->first) {
      bytes += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }
  // Would all of `sizes` (in this order, low or high placement) be placed right now?
  bool fits(const std::vector<size_t>& sizes, bool high = false) const {
    std::map<size_t, size_t> f = free_;
    for (size_t b : sizes)
      if (place(f, granules(b), high) == kNone) return false;
    return true;
  }
  size_t size() const { return size_; }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }

 private:
  static size_t place(std::map<size_t, size_t>& f, size_t b, bool high) {
    if (high) {
      for (auto it = f.rbegin(); it != f.rend(); ++it) {
        if (it->second < b) continue;
        it->second -= b;
        const size_t off = it->first + it->second;
        if (it->second == 0) f.erase(std::next(it).base());
        return off;
      }
      return kNone;
    }
    for (auto it = f.begin(); it != f.end(); ++it) {
      if (it->second < b) continue;
      const size_t off = it->first, len = it->second;
      f.erase(it);
      if (len > b) f[off + b] = len - b;
      return off;
    }
    return kNone;
  }

  std::map<size_t, size_t> free_;
  size_t size_, used_ = 0, peak_ = 0;
};

struct Series {
  bool live = false;    // reference timestep stored
  bool busy = false;    // a request of this series is running
  int dtype = 0;
  int64_t n = 0;
  size_t recon = kNone, base = kNone, blob = kNone;   // arena offsets
  size_t blob_cap = 0;
  bool has_blob = false;
};

struct Req {
  uint64_t id = 0;
  numarck_request r{};
  double t_submit = 0, t_start = 0;
  std::vector<size_t> need;      // transient buffers (bytes)
  std::vector<size_t> offs;      // their arena offsets once admitted
  bool reference = false;        // first compression of a series: store the timestep only
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  unsigned char* hdr = nullptr;  // pinned copy of the blob header
  bool busy = false;
  int stage = 0;
  Req req;
  int status = NUMARCK_OK;
  uint64_t out_bytes = 0;
  double deadline = 0;           // dry run
};

}  // namespace

struct numarck_server {
  numarck_server_config cfg{};
  int device = 0;
  Clock::time_point t0;
  Arena arena{0};
  unsigned char* base = nullptr;
  std::vector<Series> series;
  std::vector<Slot> slots;
  std::mutex mu;                            // incoming, done, stop, statistics
  std::condition_variable cv_work, cv_done;
  std::deque<Req> incoming;                 // submitted, not yet seen by the worker
  std::deque<Req> waiting;                  // seen, not started (submission order)
  std::deque<numarck_completion> done;
  std::thread worker;
  bool stop = false;
  uint64_t next_id = 1;
  // statistics
  uint64_t started = 0, completed = 0, deferred_memory = 0;
  int max_inflight = 0, inflight = 0;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
  void run();
  bool admit();
  bool poll();
  void start(Slot& sl, Req&& rq);
  void finish(Slot& sl);
  void fail(Req& rq, int status);
};

namespace {

size_t elem_bytes(int dtype) { return dtype == NUMARCK_F64 ? 8 : 4; }

numarck_params series_params(const numarck_params& p) {
  numarck_params q = p;
  q.B = NUMARCK_MAX_B;   // blob capacity and workspace cover every index length
  return q;
}

}  // namespace

void numarck_server::fail(Req& rq, int status) {
  numarck_completion c{};
  c.id = rq.id;
  c.status = status;
  c.kind = rq.r.kind;
  c.series = rq.r.series;
  c.t_submit = rq.t_submit;
  c.t_start = c.t_end = now();
  std::lock_guard<std::mutex> lk(mu);
  done.push_back(c);
  ++completed;
  cv_done.notify_all();
}

// Starts every request that can run now; true if one was started.
bool numarck_server::admit() {
  bool any = false;
  std::vector<char> blocked(series.size(), 0);
  bool have_head = false;                        // the oldest runnable request that did not fit
  std::vector<size_t> head_need;
  uint64_t head_id = 0;
  for (auto it = waiting.begin(); it != waiting.end();) {
    Req& rq = *it;
    Series& s = series[rq.r.series];
    if (s.busy || blocked[rq.r.series]) {          // keep per-series order
      blocked[rq.r.series] = 1;
      ++it;
      continue;
    }
    int free_slot = -1;
    for (int i = 0; i < (int)slots.size(); ++i)
      if (!slots[i].busy) { free_slot = i; break; }
    if (free_slot < 0) break;
    // a series keeps the length and type of its first timestep
    const bool reference = rq.r.kind == NUMARCK_REQ_COMPRESS && !s.live;
    if (!reference && (!s.live || rq.r.n != s.n || rq.r.params.dtype != s.dtype)) {
      Req bad = std::move(rq);
      it = waiting.erase(it);
      fail(bad, NUMARCK_ERR_INVALID_ARG);
      any = true;
      continue;
    }
    // the buffers this request needs (a series' resident buffers at its first compression)
    rq.reference = reference;
    rq.need.clear();
    const size_t L = elem_bytes(rq.r.params.dtype);
    if (rq.r.kind == NUMARCK_REQ_COMPRESS) {
      if (rq.reference) {
        const numarck_params q = series_params(rq.r.params);
        rq.need = {(size_t)rq.r.n * L, (size_t)rq.r.n * L, numarck_compress_bound(rq.r.n, &q)};
      } else {
        rq.need = {(size_t)rq.r.n * L, numarck_workspace_bytes(rq.r.n, &rq.r.params)};
      }
    } else {
      rq.need = {(size_t)std::max<int64_t>(rq.r.count, 1) * L};
    }
    size_t total = 0;
    for (size_t b : rq.need) total += granules(b);
    if (total > arena.size()) {                    // can never fit
      Req bad = std::move(rq);
      it = waiting.erase(it);
      fail(bad, NUMARCK_ERR_CAPACITY);
      any = true;
      continue;
    }
    std::vector<size_t> with_head = rq.need;
    with_head.insert(with_head.end(), head_need.begin(), head_need.end());
    const bool fit = rq.reference ? arena.fits(rq.need, true) && (!have_head || [&] {
      // the resident buffers go high; the older request's transient buffers must still fit
      Arena probe = arena;
      for (size_t b : rq.need) probe.alloc(b, true);
      return probe.fits(head_need);
    }()) : arena.fits(with_head);
    if (!fit) {
      if (!have_head) {
        have_head = true;
        head_need = rq.need;
        head_id = rq.id;
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        ++deferred_memory;
      }
      blocked[rq.r.series] = 1;
      ++it;
      continue;
    }
    rq.offs.clear();
    {
      std::lock_guard<std::mutex> lk(mu);
      for (size_t b : rq.need) rq.offs.push_back(arena.alloc(b, rq.reference));
    }
    if (rq.reference) {                            // resident from now on
      s.recon = rq.offs[0];
      s.base = rq.offs[1];
      s.blob = rq.offs[2];
      const numarck_params q = series_params(rq.r.params);
      s.blob_cap = numarck_compress_bound(rq.r.n, &q);
      s.n = rq.r.n;
      s.dtype = rq.r.params.dtype;
      rq.offs.clear();
      rq.need.clear();
    }
    s.busy = true;
    Req run_rq = std::move(rq);
    it = waiting.erase(it);
    start(slots[free_slot], std::move(run_rq));
    any = true;
  }
  // nothing runs and the oldest runnable request does not fit: no memory will be freed (the
  // rest of the arena holds resident series), so it never will
  if (!any && inflight == 0 && have_head) {
    for (auto it = waiting.begin(); it != waiting.end(); ++it) {
      if (it->id != head_id) continue;
      Req bad = std::move(*it);
      waiting.erase(it);
      fail(bad, NUMARCK_ERR_CAPACITY);
      return true;
    }
  }
  return any;
}

void numarck_server::start(Slot& sl, Req&& rq) {
  sl.busy = true;
  sl.stage = 0;
  sl.status = NUMARCK_OK;
  sl.out_bytes = 0;
  sl.req = std::move(rq);
  sl.req.t_start = now();
  {
    std::lock_guard<std::mutex> lk(mu);
    ++started;
    ++inflight;
    max_inflight = std::max(max_inflight, inflight);
  }
  const numarck_request& r = sl.req.r;
  Series& s = series[r.series];
  const size_t L = elem_bytes(s.dtype ? s.dtype : r.params.dtype);
  if (cfg.dry_run) {
    sl.deadline = now() + cfg.dry_run_us * 1e-6;
    if (r.kind == NUMARCK_REQ_COMPRESS && !sl.req.reference) s.has_blob = true;
    if (r.kind == NUMARCK_REQ_DECOMPRESS && !s.has_blob) sl.status = NUMARCK_ERR_INVALID_ARG;
    return;
  }
  cudaStream_t st = sl.stream;
  unsigned char* a = base;
  int rc = NUMARCK_OK;
  if (r.kind == NUMARCK_REQ_COMPRESS && sl.req.reference) {
    if (cudaMemcpyAsync(a + s.recon, r.host_in, r.n * L, cudaMemcpyHostToDevice, st) != cudaSuccess)
      rc = NUMARCK_ERR_CUDA;
  } else if (r.kind == NUMARCK_REQ_COMPRESS) {
    unsigned char* cur = a + sl.req.offs[0];
    unsigned char* ws = a + sl.req.offs[1];
    const size_t ws_bytes = sl.req.need[1];
    if (cudaMemcpyAsync(cur, r.host_in, r.n * L, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(ws, 0, ws_bytes, st) != cudaSuccess) {
      rc = NUMARCK_ERR_CUDA;
    } else {
      rc = numarck_compress(a + s.recon, cur, r.n, &r.params, a + s.blob, s.blob_cap, ws, ws_bytes,
                            reinterpret_cast<numarck_stream_t>(st));
      // the new reconstruction goes to the other resident buffer; the one compressed against
      // becomes the base of this blob
      if (!rc)
        rc = numarck_decompress(a + s.blob, nullptr, a + s.recon, a + s.base, r.n, nullptr,
                                reinterpret_cast<numarck_stream_t>(st));
      if (!rc && cudaMemcpyAsync(sl.hdr, a + s.blob, NUMARCK_HEADER_BYTES,
                                 cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = NUMARCK_ERR_CUDA;
      if (!rc) {
        std::swap(s.recon, s.base);
        s.has_blob = true;
      }
    }
  } else {
    if (!s.has_blob) {
      rc = NUMARCK_ERR_INVALID_ARG;
    } else if (r.start < 0 || r.count < 0 || r.start > s.n || r.count > s.n - r.start) {
      rc = NUMARCK_ERR_RANGE;
    } else if (r.host_out_cap < (size_t)r.count * L || (r.count > 0 && !r.host_out)) {
      rc = NUMARCK_ERR_CAPACITY;
    } else if (r.count > 0) {
      unsigned char* out = a + sl.req.offs[0];
      rc = numarck_decompress_range(a + s.blob, nullptr, a + s.base + r.start * L, r.start,
                                    r.count, out, nullptr, reinterpret_cast<numarck_stream_t>(st));
      if (!rc && cudaMemcpyAsync(r.host_out, out, r.count * L, cudaMemcpyDeviceToHost, st) !=
                     cudaSuccess)
        rc = NUMARCK_ERR_CUDA;
      sl.out_bytes = (uint64_t)r.count * L;
    }
  }
  sl.status = rc;
  if (rc == NUMARCK_OK && cudaEventRecord(sl.ev, st) != cudaSuccess) sl.status = NUMARCK_ERR_CUDA;
}

// Advances in-flight requests whose queued work has finished; true on any progress.
bool numarck_server::poll() {
  bool any = false;
  for (Slot& sl : slots) {
    if (!sl.busy) continue;
    if (cfg.dry_run) {
      if (now() < sl.deadline) continue;
      if (sl.stage == 0 && sl.req.r.kind == NUMARCK_REQ_COMPRESS && !sl.req.reference) {
        sl.stage = 1;                             // the blob copy-out stage
        sl.deadline = now() + cfg.dry_run_us * 1e-6;
        any = true;
        continue;
      }
      finish(sl);
      any = true;
      continue;
    }
    if (sl.status == NUMARCK_OK) {
      const cudaError_t q = cudaEventQuery(sl.ev);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) sl.status = NUMARCK_ERR_CUDA;
    }
    const numarck_request& r = sl.req.r;
    if (sl.status == NUMARCK_OK && sl.stage == 0 && r.kind == NUMARCK_REQ_COMPRESS &&
        !sl.req.reference) {
      // the header is on the host: copy out the blob's used bytes
      size_t size = 0;
      int rc = numarck_blob_size(sl.hdr, &size);
      Series& s = series[r.series];
      if (!rc && (size > r.host_out_cap || !r.host_out)) rc = NUMARCK_ERR_CAPACITY;
      if (!rc && cudaMemcpyAsync(r.host_out, base + s.blob, size, cudaMemcpyDeviceToHost,
                                 sl.stream) != cudaSuccess)
        rc = NUMARCK_ERR_CUDA;
      if (!rc && cudaEventRecord(sl.ev, sl.stream) != cudaSuccess) rc = NUMARCK_ERR_CUDA;
      sl.status = rc;
      sl.out_bytes = size;
      sl.stage = 1;
      any = true;
      if (rc == NUMARCK_OK) continue;
    }
    finish(sl);
    any = true;
  }
  return any;
}

void numarck_server::finish(Slot& sl) {
  Req& rq = sl.req;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (size_t i = 0; i < rq.offs.size(); ++i) arena.release(rq.offs[i], rq.need[i]);
    --inflight;
  }
  Series& s = series[rq.r.series];
  if (rq.reference && sl.status == NUMARCK_OK) s.live = true;
  s.busy = false;
  numarck_completion c{};
  c.id = rq.id;
  c.status = sl.status;
  c.kind = rq.r.kind;
  c.series = rq.r.series;
  c.reference = rq.reference ? 1 : 0;
  c.out_bytes = sl.status == NUMARCK_OK ? sl.out_bytes : 0;
  c.t_submit = rq.t_submit;
  c.t_start = rq.t_start;
  c.t_end = now();
  sl.busy = false;
  std::lock_guard<std::mutex> lk(mu);
  done.push_back(c);
  ++completed;
  cv_done.notify_all();
}

void numarck_server::run() {
  if (!cfg.dry_run) cudaSetDevice(device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(mu);
      while (!incoming.empty()) {
        waiting.push_back(std::move(incoming.front()));
        incoming.pop_front();
      }
      if (stop && waiting.empty() && inflight == 0) break;
    }
    // admit() and poll() run on this thread only; they lock mu around shared fields
    const bool progress = admit() | poll();
    if (!progress) {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait_for(lk, std::chrono::microseconds(inflight ? 20 : 2000),
                       [&] { return !incoming.empty() || (stop && inflight == 0); });
    }
  }
}

extern "C" {

numarck_server* numarck_server_create(const numarck_server_config* cfg, int* status) {
  int rc = NUMARCK_OK;
  if (!cfg || cfg->slots < 1 || cfg->slots > kMaxSlots || cfg->max_series < 1 ||
      cfg->max_series > (1 << 20) || (!cfg->dry_run && (!cfg->arena || cfg->arena_bytes == 0)) ||
      (cfg->arena && (uintptr_t)cfg->arena % kGranule) || cfg->dry_run_us < 0)
    rc = NUMARCK_ERR_INVALID_ARG;
  if (rc) {
    if (status) *status = rc;
    return nullptr;
  }
  auto* S = new numarck_server();
  S->cfg = *cfg;
  S->t0 = Clock::now();
  S->arena = Arena(cfg->arena_bytes);
  S->base = static_cast<unsigned char*>(cfg->arena);
  S->series.resize(cfg->max_series);
  S->slots.resize(cfg->slots);
  if (!cfg->dry_run) {
    if (cudaGetDevice(&S->device) != cudaSuccess) rc = NUMARCK_ERR_CUDA;
    for (Slot& sl : S->slots) {
      if (rc) break;
      if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess ||
          cudaHostAlloc(reinterpret_cast<void**>(&sl.hdr), NUMARCK_HEADER_BYTES,
                        cudaHostAllocDefault) != cudaSuccess)
        rc = NUMARCK_ERR_CUDA;
    }
  }
  if (rc) {
    numarck_server_destroy(S);
    if (status) *status = rc;
    return nullptr;
  }
  S->worker = std::thread([S] { S->run(); });
  if (status) *status = NUMARCK_OK;
  return S;
}

int numarck_server_submit(numarck_server* S, const numarck_request* r, uint64_t* id) {
  if (!S || !r) return NUMARCK_ERR_INVALID_ARG;
  if (r->kind != NUMARCK_REQ_COMPRESS && r->kind != NUMARCK_REQ_DECOMPRESS)
    return NUMARCK_ERR_INVALID_ARG;
  if (r->series < 0 || r->series >= S->cfg.max_series || r->n < 0 || r->n > ((int64_t)1 << 40))
    return NUMARCK_ERR_INVALID_ARG;
  if (r->params.dtype != NUMARCK_F32 && r->params.dtype != NUMARCK_F64)
    return NUMARCK_ERR_INVALID_ARG;
  if (r->kind == NUMARCK_REQ_COMPRESS) {
    if (numarck_workspace_bytes(r->n, &r->params) == 0 || r->params.B == 0 ||
        (r->n > 0 && !r->host_in))
      return NUMARCK_ERR_INVALID_ARG;
  }
  Req rq;
  rq.r = *r;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return NUMARCK_ERR_INVALID_ARG;
  rq.id = S->next_id++;
  rq.t_submit = S->now();
  if (id) *id = rq.id;
  S->incoming.push_back(std::move(rq));
  S->cv_work.notify_one();
  return NUMARCK_OK;
}

int numarck_server_poll(numarck_server* S, numarck_completion* out, int max, int* got,
                        int wait_ms) {
  if (!S || !got || max < 0 || (max > 0 && !out)) return NUMARCK_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->done.empty() && wait_ms > 0)
    S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !S->done.empty(); });
  int k = 0;
  while (k < max && !S->done.empty()) {
    out[k++] = S->done.front();
    S->done.pop_front();
  }
  *got = k;
  return NUMARCK_OK;
}

int numarck_server_get_stats(numarck_server* S, numarck_server_stats* st) {
  if (!S || !st) return NUMARCK_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  st->submitted = S->next_id - 1;
  st->started = S->started;
  st->completed = S->completed;
  st->deferred_memory = S->deferred_memory;
  st->arena_bytes = S->arena.size();
  st->arena_used = S->arena.used();
  st->arena_peak = S->arena.peak();
  st->max_inflight = S->max_inflight;
  st->now = S->now();
  return NUMARCK_OK;
}

int numarck_server_destroy(numarck_server* S) {
  if (!S) return NUMARCK_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv_work.notify_all();
  }
  if (S->worker.joinable()) S->worker.join();
  int rc = NUMARCK_OK;
  for (Slot& sl : S->slots) {
    if (sl.stream && cudaStreamDestroy(sl.stream) != cudaSuccess) rc = NUMARCK_ERR_CUDA;
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.hdr) cudaFreeHost(sl.hdr);
  }
  delete S;
  return rc;
}

}  // extern "C"
