// Request server: continuous batching of contact-query batches from many
// simulator clients on one detector handle (declared in include/locc.h,
// "serving").  Host runtime in C++; the only kernel here packs the pairs of
// one launch, the contact path itself is the handle's (crop gather, encoder,
// head) through run_path.
//
// Threads and streams
//   client threads   locc_server_submit / locc_server_wait (any number)
//   scheduler thread admission, launch formation, all CUDA calls
//   CUDA host-func   per launch, after its results reached host memory:
//                    marks requests done, frees their arena blocks
// Streams: s_h2d (inputs of newly admitted requests -> arena), s_comp (pack
// kernel + contact path, one launch after another), s_d2h (results -> the
// clients' `out` arrays).  A launch waits for the inputs of its requests with
// events; the results of launch k copy out while launch k + 1 computes.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "arena.hpp"
#include "common.cuh"
#include "handle.cuh"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kSlots = 3;          // launches in flight (pack / compute / copy-out)
constexpr int kMaxActive = 1024;   // admitted requests at once (segment table size)

// One contiguous run of a request's pairs inside a launch (device table).
struct alignas(16) Segment {
  const float* poses;      // request's poses in the arena [n_obj][7]
  const int32_t* shape;    // request's obj_shape in the arena [n_obj]
  const int32_t* pairs;    // request's pairs in the arena [n_pairs][2]
  int32_t first;           // first pair of the run (request-local index)
  int32_t dst;             // first packed row of the run in this launch
};

// Packed inputs of launch rows [0, n): row j of the launch is the segment
// whose dst is the last one <= j.  Objects are renumbered 2j (A) and 2j + 1
// (B), so the contact path sees one self-contained batch; its outputs are
// therefore those of the pair computed alone.
__global__ void pack_kernel(const Segment* __restrict__ tab, int n_seg, int n,
                            float* __restrict__ poses, int32_t* __restrict__ shape,
                            int2* __restrict__ pairs) {
  __shared__ int s_dst[kMaxActive];
  for (int i = threadIdx.x; i < n_seg; i += blockDim.x) s_dst[i] = tab[i].dst;
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int lo = 0, hi = n_seg - 1;  // last segment with dst <= j
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (s_dst[mid] <= j) lo = mid;
    else hi = mid - 1;
  }
  const Segment sg = tab[lo];
  const int p = sg.first + (j - s_dst[lo]);
  const int2 ab = reinterpret_cast<const int2*>(sg.pairs)[p];
  const int obj[2] = {ab.x, ab.y};
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float* src = sg.poses + 7 * (size_t)obj[k];
    float* dstp = poses + 7 * (size_t)(2 * j + k);
#pragma unroll
    for (int c = 0; c < 7; ++c) dstp[c] = src[c];
    shape[2 * j + k] = sg.shape[obj[k]];
  }
  pairs[j] = make_int2(2 * j, 2 * j + 1);
}

enum ReqState { kQueued = 0, kActive = 1, kDone = 2 };

struct Request {
  int64_t id = 0;
  locc_request rq{};
  size_t bytes = 0, off = 0, off_shape = 0, off_pairs = 0;
  int64_t cursor = 0;        // pairs handed to launches (scheduler, under the lock)
  int in_flight = 0;         // launches carrying its pairs not yet copied out
  int launches = 0;
  int status = 0;
  ReqState state = kQueued;
  cudaEvent_t ready = nullptr;  // its inputs are in the arena
  Clock::time_point t_submit, t_admit, t_done;
};

struct SegHost {
  Request* r;
  int64_t first, count, dst;
};

struct Slot {
  locc_server* srv = nullptr;
  bool busy = false;
  int n = 0;
  Segment* h_tab = nullptr;  // pinned
  Segment* d_tab = nullptr;
  float* d_poses = nullptr;
  int32_t* d_shape = nullptr;
  int2* d_pairs = nullptr;
  float* d_out = nullptr;
  cudaEvent_t ev_comp = nullptr;
  std::vector<SegHost> segs;
};

double us_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::micro>(b - a).count();
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  const size_t k = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
  std::nth_element(v.begin(), v.begin() + (ptrdiff_t)k, v.end());
  return v[k];
}

}  // namespace

struct locc_server {
  locc_handle* h = nullptr;
  locc_server_config cfg{};
  cudaStream_t s_h2d = nullptr, s_comp = nullptr, s_d2h = nullptr;
  char* d_arena = nullptr;
  locc::Arena arena;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<Request*> queue;              // waiting for admission, arrival order
  std::vector<Request*> active;            // admitted, admission order
  std::unordered_map<int64_t, Request*> live;  // every request not yet waited for
  std::vector<cudaEvent_t> free_events;
  Slot slots[kSlots];
  std::thread th;
  bool stop = false;
  int64_t next_id = 1;
  int64_t queued_pairs = 0;
  // statistics (under mu)
  int64_t n_submitted = 0, n_rejected = 0, n_completed = 0, n_failed = 0;
  int64_t pairs_completed = 0, launches = 0, launched_pairs = 0;
  int max_active_seen = 0;
  std::vector<double> latencies;

  void scheduler();
  int launch(Slot& sl, std::vector<Request*>& cand);
  void finish_locked(Request* r, Clock::time_point now);
};

namespace {

// Runs on a CUDA callback thread once a launch's results are in the clients'
// arrays: no CUDA calls here, only bookkeeping under the server lock.
void CUDART_CB on_launch_done(void* p) {
  Slot* sl = static_cast<Slot*>(p);
  locc_server* S = sl->srv;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    const Clock::time_point now = Clock::now();
    for (const SegHost& sg : sl->segs) {
      Request* r = sg.r;
      if (--r->in_flight == 0 && r->cursor == r->rq.n_pairs) S->finish_locked(r, now);
    }
    sl->segs.clear();
    sl->busy = false;
  }
  S->cv_sched.notify_all();
  S->cv_done.notify_all();
}

}  // namespace

// Under mu.  A finished request leaves the admitted list here, before any
// client can see it done (locc_server_wait frees it), and returns its arena
// block and event.
void locc_server::finish_locked(Request* r, Clock::time_point now) {
  r->state = kDone;
  r->t_done = now;
  auto it = std::find(active.begin(), active.end(), r);
  if (it != active.end()) active.erase(it);
  if (r->ready) {
    free_events.push_back(r->ready);
    r->ready = nullptr;
  }
  if (r->bytes) arena.release(r->off);
  if (r->status == 0) {
    ++n_completed;
    pairs_completed += r->rq.n_pairs;
    latencies.push_back(us_between(r->t_submit, now));
  } else {
    ++n_failed;
  }
}

// Build and enqueue one launch from the admitted requests `cand` (admission
// order, each with pairs left).  Returns 0 or an error code.
int locc_server::launch(Slot& sl, std::vector<Request*>& cand) {
  const int n = (int)cand.size();
  std::vector<int64_t> rem(n), take(n);
  for (int i = 0; i < n; ++i) rem[i] = cand[i]->rq.n_pairs - cand[i]->cursor;
  const int64_t total = locc::pack_launch(rem.data(), n, cfg.max_batch_pairs, take.data());
  if (total == 0) return 0;
  sl.segs.clear();
  int64_t dst = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (int i = 0; i < n; ++i) {
      if (!take[i]) continue;
      Request* r = cand[i];
      sl.segs.push_back({r, r->cursor, take[i], dst});
      r->cursor += take[i];
      ++r->in_flight;
      ++r->launches;
      dst += take[i];
    }
    sl.busy = true;
    ++launches;
    launched_pairs += total;
  }
  sl.n = (int)total;
  const int n_seg = (int)sl.segs.size();
  for (int i = 0; i < n_seg; ++i) {
    const SegHost& sg = sl.segs[i];
    char* base = d_arena + sg.r->off;
    sl.h_tab[i] = Segment{reinterpret_cast<const float*>(base),
                          reinterpret_cast<const int32_t*>(d_arena + sg.r->off_shape),
                          reinterpret_cast<const int32_t*>(d_arena + sg.r->off_pairs),
                          (int32_t)sg.first, (int32_t)sg.dst};
  }
  cudaError_t e = cudaSuccess;
  int st = 0;
  for (int i = 0; i < n_seg && e == cudaSuccess; ++i)
    e = cudaStreamWaitEvent(s_comp, sl.segs[i].r->ready, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sl.d_tab, sl.h_tab, sizeof(Segment) * n_seg, cudaMemcpyHostToDevice, s_comp);
  if (e == cudaSuccess) {
    pack_kernel<<<(sl.n + 255) / 256, 256, 0, s_comp>>>(sl.d_tab, n_seg, sl.n, sl.d_poses,
                                                        sl.d_shape, sl.d_pairs);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    locc::PairInputs in{sl.d_poses, sl.d_shape, reinterpret_cast<const int32_t*>(sl.d_pairs), 2 * sl.n,
                  sl.n};
    st = locc::run_path(h, in, sl.n, nullptr, sl.d_out, s_comp);
  }
  if (e == cudaSuccess && st == 0) e = cudaEventRecord(sl.ev_comp, s_comp);
  if (e == cudaSuccess && st == 0) e = cudaStreamWaitEvent(s_d2h, sl.ev_comp, 0);
  for (int i = 0; i < n_seg && e == cudaSuccess && st == 0; ++i) {
    const SegHost& sg = sl.segs[i];
    e = cudaMemcpyAsync(sg.r->rq.out + 8 * sg.first, sl.d_out + 8 * sg.dst,
                        (size_t)sg.count * 8 * sizeof(float), cudaMemcpyDeviceToHost, s_d2h);
  }
  if (e == cudaSuccess && st == 0) e = cudaLaunchHostFunc(s_d2h, on_launch_done, &sl);
  if (e == cudaSuccess && st == 0) return 0;
  // The launch could not be enqueued: fail its requests once the streams are idle.
  if (st == 0) st = LOCC_ERR_CUDA;
  cudaGetLastError();
  cudaStreamSynchronize(s_comp);
  cudaStreamSynchronize(s_d2h);
  {
    std::lock_guard<std::mutex> lk(mu);
    const Clock::time_point now = Clock::now();
    for (const SegHost& sg : sl.segs) {
      Request* r = sg.r;
      r->status = st;
      if (--r->in_flight == 0 && r->cursor == r->rq.n_pairs) finish_locked(r, now);
    }
    sl.segs.clear();
    sl.busy = false;
  }
  cv_done.notify_all();
  return st;
}

void locc_server::scheduler() {
  cudaSetDevice(h->device);
  std::vector<Request*> admitted, cand;
  for (;;) {
    Slot* slot = nullptr;
    admitted.clear();
    cand.clear();
    {
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        // admission in arrival order while the arena has room
        // launch pressure of the admitted requests: the pairs each still has to
        // launch, counted up to one launch, so a large request does not keep
        // small ones out while many large ones are bounded
        int64_t pressure = 0;
        for (Request* r : active)
          pressure += std::min<int64_t>(r->rq.n_pairs - r->cursor, cfg.max_batch_pairs);
        while (!queue.empty() && (int)active.size() < cfg.max_active && !free_events.empty() &&
               (active.empty() || pressure < cfg.max_active_pairs)) {
          Request* r = queue.front();
          size_t off = 0;
          if (!arena.alloc(r->bytes, &off)) break;
          queue.pop_front();
          queued_pairs -= r->rq.n_pairs;
          pressure += std::min<int64_t>(r->rq.n_pairs, cfg.max_batch_pairs);
          r->off = off;
          r->off_shape = off + (((size_t)r->rq.n_obj * 28 + 255) / 256 * 256);
          r->off_pairs = r->off_shape + (((size_t)r->rq.n_obj * 4 + 255) / 256 * 256);
          r->ready = free_events.back();
          free_events.pop_back();
          r->state = kActive;
          r->t_admit = Clock::now();
          active.push_back(r);
          admitted.push_back(r);
        }
        max_active_seen = std::max(max_active_seen, (int)active.size());
        for (Slot& s : slots)
          if (!s.busy) {
            slot = &s;
            break;
          }
        for (Request* r : active)
          if (r->cursor < r->rq.n_pairs) cand.push_back(r);
        if (!admitted.empty() || (slot && !cand.empty())) break;
        bool idle = queue.empty() && active.empty();
        for (Slot& s : slots) idle = idle && !s.busy;
        if (stop && idle) return;
        cand.clear();
        cv_sched.wait_for(lk, std::chrono::milliseconds(50));
      }
    }
    // inputs of newly admitted requests -> arena (outside the lock: these
    // calls may block while a callback wants the lock)
    for (Request* r : admitted) {
      char* base = d_arena + r->off;
      cudaError_t e = cudaMemcpyAsync(base, r->rq.poses, (size_t)r->rq.n_obj * 28,
                                      cudaMemcpyHostToDevice, s_h2d);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_arena + r->off_shape, r->rq.obj_shape, (size_t)r->rq.n_obj * 4,
                            cudaMemcpyHostToDevice, s_h2d);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_arena + r->off_pairs, r->rq.pairs, (size_t)r->rq.n_pairs * 8,
                            cudaMemcpyHostToDevice, s_h2d);
      if (e == cudaSuccess) e = cudaEventRecord(r->ready, s_h2d);
      if (e != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(s_h2d);
        std::lock_guard<std::mutex> lk(mu);
        r->status = LOCC_ERR_CUDA;
        r->cursor = r->rq.n_pairs;  // nothing more to launch
        if (r->in_flight == 0) finish_locked(r, Clock::now());
        cv_done.notify_all();
      }
    }
    if (!slot || cand.empty()) continue;
    // requests whose copy-in just failed are finished: skip them
    cand.erase(std::remove_if(cand.begin(), cand.end(),
                              [](Request* r) { return r->cursor >= r->rq.n_pairs; }),
               cand.end());
    if (!cand.empty()) launch(*slot, cand);
  }
}

extern "C" {

int locc_server_create(locc_handle* h, const locc_server_config* cfg_in, locc_server** out) {
  using locc::set_error;
  if (out) *out = nullptr;
  if (!h || !out) {
    set_error("locc_server_create: NULL handle or output");
    return LOCC_ERR_INVALID_ARG;
  }
  locc_server_config cfg{};
  if (cfg_in) cfg = *cfg_in;
  if (cfg.max_batch_pairs == 0) cfg.max_batch_pairs = 131072;
  if (cfg.max_active == 0) cfg.max_active = 256;
  if (cfg.max_active_pairs == 0) cfg.max_active_pairs = 4 * (int64_t)cfg.max_batch_pairs;
  if (cfg.max_batch_pairs < 1 || cfg.max_active < 1 || cfg.max_active > kMaxActive ||
      cfg.arena_bytes < 0 || cfg.max_queued_pairs < 0 || cfg.max_active_pairs < 0) {
    set_error("locc_server_create: max_batch_pairs >= 1, 1 <= max_active <= 1024, "
              "arena_bytes, max_queued_pairs and max_active_pairs >= 0 are required");
    return LOCC_ERR_INVALID_ARG;
  }
  if (cudaSetDevice(h->device) != cudaSuccess) {
    set_error("locc_server_create: cudaSetDevice failed");
    return LOCC_ERR_CUDA;
  }
  int st = locc_reserve(h, cfg.max_batch_pairs, 0);
  if (st) return st;
  if (cfg.arena_bytes == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      set_error("locc_server_create: cudaMemGetInfo failed");
      return LOCC_ERR_CUDA;
    }
    cfg.arena_bytes = (int64_t)(fr / 2);
  }
  locc_server* S = new (std::nothrow) locc_server;
  if (!S) {
    set_error("locc_server_create: host allocation failed");
    return LOCC_ERR_OOM;
  }
  S->h = h;
  S->cfg = cfg;
  bool ok = cudaStreamCreateWithFlags(&S->s_h2d, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&S->s_comp, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&S->s_d2h, cudaStreamNonBlocking) == cudaSuccess;
  const size_t M = (size_t)cfg.max_batch_pairs;
  bool oom = false;
  if (ok) {
    oom = cudaMalloc(&S->d_arena, (size_t)cfg.arena_bytes) != cudaSuccess;
    S->arena.reset((size_t)cfg.arena_bytes, 256);
  }
  for (int i = 0; ok && !oom && i < kSlots; ++i) {
    Slot& sl = S->slots[i];
    sl.srv = S;
    oom = cudaMallocHost(&sl.h_tab, sizeof(Segment) * kMaxActive) != cudaSuccess ||
          cudaMalloc(&sl.d_tab, sizeof(Segment) * kMaxActive) != cudaSuccess ||
          cudaMalloc(&sl.d_poses, M * 2 * 7 * sizeof(float)) != cudaSuccess ||
          cudaMalloc(&sl.d_shape, M * 2 * sizeof(int32_t)) != cudaSuccess ||
          cudaMalloc(&sl.d_pairs, M * sizeof(int2)) != cudaSuccess ||
          cudaMalloc(&sl.d_out, M * 8 * sizeof(float)) != cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&sl.ev_comp, cudaEventDisableTiming) == cudaSuccess;
  }
  for (int i = 0; ok && !oom && i < cfg.max_active; ++i) {
    cudaEvent_t e = nullptr;
    ok = cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (ok) S->free_events.push_back(e);
  }
  if (!ok || oom) {
    cudaGetLastError();
    locc_server_destroy(S);
    set_error(oom ? "locc_server_create: device or pinned allocation failed"
                  : "locc_server_create: stream or event creation failed");
    return oom ? LOCC_ERR_OOM : LOCC_ERR_CUDA;
  }
  S->th = std::thread([S] { S->scheduler(); });
  *out = S;
  return LOCC_OK;
}

int locc_server_submit(locc_server* S, const locc_request* req, int64_t* id_out) {
  using locc::set_error;
  if (!S || !req || !id_out) {
    set_error("locc_server_submit: NULL argument");
    return LOCC_ERR_INVALID_ARG;
  }
  const locc_request& q = *req;
  if (q.n_obj < 0 || q.n_pairs < 0) {
    set_error("locc_server_submit: negative size");
    return LOCC_ERR_INVALID_ARG;
  }
  if (q.n_pairs > 0 && (!q.poses || !q.obj_shape || !q.pairs || !q.out)) {
    set_error("locc_server_submit: NULL array");
    return LOCC_ERR_INVALID_ARG;
  }
  // host-side validation, so that no launch meets a bad index
  for (int64_t i = 0; i < 2 * (int64_t)q.n_pairs; ++i)
    if (q.pairs[i] < 0 || q.pairs[i] >= q.n_obj) {
      set_error("locc_server_submit: a pair index is outside [0, n_obj)");
      return LOCC_ERR_INVALID_ARG;
    }
  if (q.n_pairs > 0)
    for (int32_t i = 0; i < q.n_obj; ++i)
      if (q.obj_shape[i] < 0 || q.obj_shape[i] >= S->h->n_shapes) {
        set_error("locc_server_submit: a shape id is outside [0, n_shapes)");
        return LOCC_ERR_INVALID_ARG;
      }
  Request* r = new (std::nothrow) Request;
  if (!r) {
    set_error("locc_server_submit: host allocation failed");
    return LOCC_ERR_OOM;
  }
  r->rq = q;
  r->t_submit = Clock::now();
  if (q.n_pairs > 0) {
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    r->bytes = al((size_t)q.n_obj * 28) + al((size_t)q.n_obj * 4) + al((size_t)q.n_pairs * 8);
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (r->bytes && !S->arena.fits_empty(r->bytes)) {
      ++S->n_rejected;
      delete r;
      set_error("locc_server_submit: the request's inputs exceed the whole arena");
      return LOCC_ERR_OOM;
    }
    if (S->cfg.max_queued_pairs > 0 && S->queued_pairs > 0 &&
        S->queued_pairs + q.n_pairs > S->cfg.max_queued_pairs) {
      ++S->n_rejected;
      delete r;
      set_error("locc_server_submit: queue full (max_queued_pairs)");
      return LOCC_ERR_BUSY;
    }
    r->id = S->next_id++;
    ++S->n_submitted;
    S->live[r->id] = r;
    if (q.n_pairs == 0) {
      r->t_admit = r->t_submit;
      S->finish_locked(r, r->t_submit);
    } else {
      S->queue.push_back(r);
      S->queued_pairs += q.n_pairs;
    }
    *id_out = r->id;
  }
  S->cv_sched.notify_all();
  S->cv_done.notify_all();
  return LOCC_OK;
}

int locc_server_wait(locc_server* S, int64_t id, int32_t timeout_ms, locc_request_info* info) {
  using locc::set_error;
  if (!S) {
    set_error("locc_server_wait: NULL server");
    return LOCC_ERR_INVALID_ARG;
  }
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->live.find(id);
  if (it == S->live.end()) {
    set_error("locc_server_wait: unknown request id");
    return LOCC_ERR_INVALID_ARG;
  }
  Request* r = it->second;
  auto done = [r] { return r->state == kDone; };
  if (timeout_ms < 0) {
    S->cv_done.wait(lk, done);
  } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
    set_error("locc_server_wait: request still running");
    return LOCC_ERR_TIMEOUT;
  }
  if (info) {
    info->admit_us = us_between(r->t_submit, r->t_admit);
    info->done_us = us_between(r->t_submit, r->t_done);
    info->launches = r->launches;
    info->status = r->status;
  }
  const int st = r->status;
  S->live.erase(it);
  delete r;
  if (st) set_error("locc_server_wait: a launch carrying this request failed");
  return st;
}

int locc_server_stats(locc_server* S, locc_server_counters* st, int32_t reset) {
  if (!S || !st) {
    locc::set_error("locc_server_stats: NULL argument");
    return LOCC_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = S->n_submitted;
  st->rejected = S->n_rejected;
  st->completed = S->n_completed;
  st->failed = S->n_failed;
  st->queued = (int64_t)S->queue.size();
  st->active = (int64_t)S->active.size();
  st->pairs_completed = S->pairs_completed;
  st->launches = S->launches;
  st->arena_bytes = (int64_t)S->arena.capacity();
  st->arena_used = (int64_t)S->arena.used();
  st->arena_peak = (int64_t)S->arena.peak();
  st->latency_p50_us = percentile(S->latencies, 0.50);
  st->latency_p99_us = percentile(S->latencies, 0.99);
  st->latency_max_us =
      S->latencies.empty() ? 0.0 : *std::max_element(S->latencies.begin(), S->latencies.end());
  st->mean_pairs_per_launch = S->launches ? (double)S->launched_pairs / (double)S->launches : 0.0;
  st->max_active_seen = S->max_active_seen;
  if (reset) {
    S->n_submitted = S->n_rejected = S->n_completed = S->n_failed = 0;
    S->pairs_completed = S->launches = S->launched_pairs = 0;
    S->max_active_seen = 0;
    S->latencies.clear();
  }
  return LOCC_OK;
}

void locc_server_destroy(locc_server* S) {
  if (!S) return;
  if (S->th.joinable()) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->stop = true;
    }
    S->cv_sched.notify_all();
    S->th.join();
  }
  if (S->s_h2d) cudaStreamSynchronize(S->s_h2d);
  if (S->s_comp) cudaStreamSynchronize(S->s_comp);
  if (S->s_d2h) cudaStreamSynchronize(S->s_d2h);
  for (auto& kv : S->live) {
    if (kv.second->ready) cudaEventDestroy(kv.second->ready);
    delete kv.second;
  }
  for (cudaEvent_t e : S->free_events) cudaEventDestroy(e);
  for (Slot& sl : S->slots) {
    cudaFreeHost(sl.h_tab);
    cudaFree(sl.d_tab);
    cudaFree(sl.d_poses);
    cudaFree(sl.d_shape);
    cudaFree(sl.d_pairs);
    cudaFree(sl.d_out);
    if (sl.ev_comp) cudaEventDestroy(sl.ev_comp);
  }
  cudaFree(S->d_arena);
  if (S->s_h2d) cudaStreamDestroy(S->s_h2d);
  if (S->s_comp) cudaStreamDestroy(S->s_comp);
  if (S->s_d2h) cudaStreamDestroy(S->s_d2h);
  delete S;
}

}  // extern "C"
