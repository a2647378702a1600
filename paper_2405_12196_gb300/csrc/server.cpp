// Continuous-batching server for contraction requests (include/ytn.h, "Serving").
//
// An admission thread keeps a FIFO of submitted requests and a set of stream
// slots. A request is admitted when a slot is free and its workspace fits in
// the caller's device arena (first-fit, 256-byte aligned ranges, freed ranges
// coalesced). Admitted requests are launched with ytn_tensordot on their slot's
// stream, so several requests overlap on the device; completion is detected
// with one event per slot. A request that finishes releases its slot and its
// arena range at once, so waiting requests are admitted while others run.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <new>
#include <system_error>
#include <thread>

#include "ytn_internal.hpp"

namespace ytn {

namespace {

constexpr size_t kAlign = 256;

// First-fit allocator over [0, cap) with coalescing of freed ranges.
class Arena {
 public:
  explicit Arena(size_t cap) : cap_(cap) {
    if (cap_) free_[0] = cap_;
  }
  bool alloc(size_t bytes, size_t &off) {
    const size_t need = (bytes + kAlign - 1) / kAlign * kAlign;
    if (need == 0) {
      off = 0;
      return true;
    }
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= need) {
        off = it->first;
        const size_t rest = it->second - need;
        free_.erase(it);
        if (rest) free_[off + need] = rest;
        used_ += need;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    const size_t need = (bytes + kAlign - 1) / kAlign * kAlign;
    if (need == 0) return;
    used_ -= need;
    auto it = free_.emplace(off, need).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  size_t cap_ = 0, used_ = 0;
  std::map<size_t, size_t> free_;
};

struct Request {
  int64_t id = 0;
  ytn_plan_t *plan = nullptr;
  const double *a = nullptr, *b = nullptr;
  double *c = nullptr;
  ytn_precision prec = YTN_FP64;
  double rtol = 0;
  double t_arrive = 0, t_admit = 0;
  size_t ws = 0, ws_off = 0;
  int slot = -1;
};

}  // namespace

}  // namespace ytn

struct ytn_server_s {
  ytn_ctx *ctx = nullptr;
  char *arena = nullptr;
  size_t arena_bytes = 0;
  ytn::Arena alloc{0};
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<bool> busy;
  std::vector<ytn::Request> running;
  std::deque<ytn::Request> pending;
  std::deque<ytn_request_info> done;
  std::mutex mu;
  std::condition_variable cv;
  std::thread th;
  bool stop = false;
  int64_t submitted = 0, finished = 0;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

  double now() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }

  void finish(const ytn::Request &r, int status, double t_done) {
    ytn_request_info info{};
    info.id = r.id;
    info.status = status;
    info.slot = r.slot;
    info.t_arrive = r.t_arrive;
    info.t_admit = r.t_admit;
    info.t_done = t_done;
    info.workspace = r.ws;
    done.push_back(info);
    finished++;
    if (r.plan) ytn_plan_release(r.plan);
  }

  // One pass of the admission loop (called with mu held). Returns true if it
  // changed anything.
  bool step() {
    bool acted = false;
    for (size_t s = 0; s < streams.size(); s++) {
      if (!busy[s]) continue;
      const cudaError_t q = cudaEventQuery(events[s]);
      if (q == cudaErrorNotReady) continue;
      const ytn::Request &r = running[s];
      alloc.release(r.ws_off, r.ws);
      finish(r, q == cudaSuccess ? YTN_OK : YTN_E_CUDA, now());
      busy[s] = false;
      acted = true;
    }
    while (!pending.empty()) {
      size_t s = 0;
      while (s < streams.size() && busy[s]) s++;
      if (s == streams.size()) break;
      ytn::Request &r = pending.front();
      size_t off = 0;
      if (!alloc.alloc(r.ws, off)) break;   // FIFO: wait until the head fits
      ytn::Request req = r;
      pending.pop_front();
      req.ws_off = off;
      req.slot = (int)s;
      req.t_admit = now();
      const ytn_status st = ytn_tensordot(req.plan, req.a, req.b, req.c, req.prec, req.rtol,
                                          req.ws ? arena + off : nullptr, req.ws, nullptr,
                                          reinterpret_cast<ytn_stream>(streams[s]));
      if (st != YTN_OK || cudaEventRecord(events[s], streams[s]) != cudaSuccess) {
        alloc.release(off, req.ws);
        finish(req, st != YTN_OK ? st : YTN_E_CUDA, now());
      } else {
        running[s] = req;
        busy[s] = true;
      }
      acted = true;
    }
    return acted;
  }

  void loop() {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      const bool acted = step();
      bool any_busy = false;
      for (bool b : busy) any_busy = any_busy || b;
      if (stop && pending.empty() && !any_busy) break;
      if (!acted) {
        if (any_busy) cv.wait_for(lk, std::chrono::microseconds(20));
        else cv.wait_for(lk, std::chrono::milliseconds(2));
      }
    }
  }
};

using namespace ytn;

extern "C" {

ytn_status ytn_server_create(ytn_ctx *ctx, int nslots, void *arena, size_t arena_bytes, ytn_server_t **server) {
  if (!ctx || !server || nslots < 1 || nslots > 64) return fail(YTN_E_INVALID, "bad server arguments");
  if (ctx->device < 0) return fail(YTN_E_INVALID, "host-only context");
  if ((arena_bytes && !arena) || ((uintptr_t)arena & (kAlign - 1)))
    return fail(YTN_E_INVALID, "arena missing or not 256-byte aligned");
  *server = nullptr;
  ytn_server_t *s = new (std::nothrow) ytn_server_t;
  if (!s) return fail(YTN_E_NOMEM, "host allocation failed");
  s->ctx = ctx;
  s->arena = static_cast<char *>(arena);
  s->arena_bytes = arena_bytes;
  s->alloc = Arena(arena_bytes);
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  auto release = [&]() {
    for (auto x : s->streams) cudaStreamDestroy(x);
    for (auto x : s->events) cudaEventDestroy(x);
    cudaSetDevice(prev);
    delete s;
  };
  for (int i = 0; i < nslots; i++) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      release();
      return fail(YTN_E_CUDA, "cannot create server streams");
    }
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaStreamDestroy(st);
      release();
      return fail(YTN_E_CUDA, "cannot create server events");
    }
    s->streams.push_back(st);
    s->events.push_back(ev);
  }
  s->busy.assign(nslots, false);
  s->running.resize(nslots);
  try {
    s->th = std::thread([s] { s->loop(); });
  } catch (const std::system_error &) {
    release();
    return fail(YTN_E_NOMEM, "cannot start the admission thread");
  }
  cudaSetDevice(prev);
  *server = s;
  return YTN_OK;
}

ytn_status ytn_server_submit(ytn_server_t *s, int64_t id, ytn_plan_t *plan, const double *a, const double *b,
                             double *c, ytn_precision prec, double rtol, double t_arrive) {
  if (!s || !plan) return fail(YTN_E_INVALID, "null argument");
  if (plan->ctx != s->ctx) return fail(YTN_E_INVALID, "plan belongs to another context");
  size_t ws = 0;
  ytn_status st = ytn_workspace_size(plan, prec, rtol, &ws);
  Request r;
  r.id = id;
  r.a = a;
  r.b = b;
  r.c = c;
  r.prec = prec;
  r.rtol = rtol;
  r.ws = ws;
  std::lock_guard<std::mutex> lk(s->mu);
  r.t_arrive = t_arrive >= 0 ? t_arrive : s->now();
  s->submitted++;
  if (st != YTN_OK || ws > s->arena_bytes) {
    s->finish(r, st != YTN_OK ? st : YTN_E_WORKSPACE, s->now());
    return YTN_OK;
  }
  plan->refs++;
  r.plan = plan;
  s->pending.push_back(r);
  s->cv.notify_one();
  return YTN_OK;
}

ytn_status ytn_server_poll(ytn_server_t *s, ytn_request_info *out, int64_t max, int64_t *n) {
  if (!s || !n || (max > 0 && !out)) return fail(YTN_E_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  int64_t k = 0;
  while (k < max && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  *n = k;
  return YTN_OK;
}

ytn_status ytn_server_drain(ytn_server_t *s, int64_t timeout_ms) {
  if (!s) return fail(YTN_E_INVALID, "null server");
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->finished == s->submitted) return YTN_OK;
      s->cv.notify_one();
    }
    if (timeout_ms >= 0 &&
        std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count() >
            timeout_ms)
      return fail(YTN_E_TIMEOUT, "requests still running after the timeout");
    std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
}

double ytn_server_now_ms(const ytn_server_t *s) { return s ? s->now() : 0.0; }

void ytn_server_destroy(ytn_server_t *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_one();
  }
  if (s->th.joinable()) s->th.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->ctx->device);
  for (auto x : s->streams) cudaStreamDestroy(x);
  for (auto x : s->events) cudaEventDestroy(x);
  cudaSetDevice(prev);
  delete s;
}

}  // extern "C"
