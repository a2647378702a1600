// C ABI of the library (include/ytn.h): contexts, planning with a plan cache,
// upload of the job tables, and the execution entry points that launch the
// device kernels on the caller's stream.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <algorithm>
#include <array>
#include <functional>
#include <cstring>
#include <new>
#include <thread>

#include "kernels.hpp"

namespace ytn {

static thread_local std::string g_last_error;

ytn_status fail(ytn_status st, const std::string &msg) {
  g_last_error = msg;
  return st;
}

static ytn_status cuda_fail(cudaError_t e, const char *what) {
  return fail(YTN_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Makes ctx->device current for the scope of an entry point and restores the
// caller's device afterwards.
class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    ok_ = cudaGetDevice(&prev_) == cudaSuccess;
    if (ok_ && prev_ != dev) ok_ = cudaSetDevice(dev) == cudaSuccess, changed_ = true;
  }
  ~DeviceGuard() {
    if (changed_) cudaSetDevice(prev_);
  }
  bool ok() const { return ok_; }

 private:
  int prev_ = 0;
  bool ok_ = false, changed_ = false;
};

static size_t align256(size_t b) { return (b + 255) / 256 * 256; }

template <class T>
static void put_table(std::vector<char> &buf, const std::vector<T> &v, size_t &off) {
  off = align256(buf.size());
  buf.resize(off + v.size() * sizeof(T));
  if (!v.empty()) std::memcpy(buf.data() + off, v.data(), v.size() * sizeof(T));
}

static ytn_status upload(ytn_plan_t *p) {
  std::vector<char> buf;
  size_t o_jobs, o_items, o_sec, o_tiles, o_tro, o_trc;
  put_table(buf, p->jobs, o_jobs);
  put_table(buf, p->items, o_items);
  put_table(buf, p->sectors_dev, o_sec);
  put_table(buf, p->tiles, o_tiles);
  put_table(buf, p->tr_out, o_tro);
  size_t o_csj;
  put_table(buf, p->cs_jobs, o_csj);
  put_table(buf, p->tr_contrib, o_trc);
  size_t o_vdp, o_vdc;
  put_table(buf, p->vd_pieces, o_vdp);
  put_table(buf, p->vd_chunks, o_vdc);
  size_t o_spo, o_spe, o_sps, o_spsec, o_spt, o_spfi, o_spsg;
  put_table(buf, p->sp_ops, o_spo);
  put_table(buf, p->sp_exp_items, o_spe);
  put_table(buf, p->sp_slice_items, o_sps);
  put_table(buf, p->sp_sectors, o_spsec);
  put_table(buf, p->sp_tiles, o_spt);
  size_t o_sptm;
  put_table(buf, p->sp_tiles_mix, o_sptm);
  put_table(buf, p->sp_fitems, o_spfi);
  put_table(buf, p->sp_segs, o_spsg);
  p->dev_bytes = align256(buf.size()) + 256;
  cudaError_t e = cudaMalloc(&p->dev, p->dev_bytes);
  if (e != cudaSuccess) {
    p->dev = nullptr;
    return e == cudaErrorMemoryAllocation ? fail(YTN_E_NOMEM, "cudaMalloc of plan tables failed")
                                          : cuda_fail(e, "cudaMalloc");
  }
  if (!buf.empty()) {
    e = cudaMemcpy(p->dev, buf.data(), buf.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy of plan tables");
  }
  char *d = static_cast<char *>(p->dev);
  p->d_jobs = reinterpret_cast<const CopyJob *>(d + o_jobs);
  p->d_items = reinterpret_cast<const CopyItem *>(d + o_items);
  p->d_sectors = reinterpret_cast<const SectorDev *>(d + o_sec);
  p->d_tiles = reinterpret_cast<const GemmTile *>(d + o_tiles);
  p->d_tr_out = reinterpret_cast<const TraceOut *>(d + o_tro);
  p->d_cs_jobs = reinterpret_cast<const CScatterJob *>(d + o_csj);
  p->d_tr_contrib = reinterpret_cast<const TraceContrib *>(d + o_trc);
  p->d_vd_pieces = reinterpret_cast<const VdotPiece *>(d + o_vdp);
  p->d_vd_chunks = reinterpret_cast<const VdotChunk *>(d + o_vdc);
  p->d_sp_ops = reinterpret_cast<const SplitOperand *>(d + o_spo);
  p->d_sp_exp_items = reinterpret_cast<const SplitItem *>(d + o_spe);
  p->d_sp_slice_items = reinterpret_cast<const SplitItem *>(d + o_sps);
  p->d_sp_sectors = reinterpret_cast<const SplitSector *>(d + o_spsec);
  p->d_sp_tiles = reinterpret_cast<const SplitTile *>(d + o_spt);
  p->d_sp_tiles_mix = reinterpret_cast<const SplitTile *>(d + o_sptm);
  p->d_sp_fitems = reinterpret_cast<const SliceItem *>(d + o_spfi);
  p->d_sp_segs = reinterpret_cast<const SliceSeg *>(d + o_spsg);
  return YTN_OK;
}

static void destroy_plan(ytn_plan_t *p) {
  if (!p) return;
  if (p->dev) {
    DeviceGuard g(p->ctx->device);
    cudaFree(p->dev);
  }
  delete p;
}

// Records a CUDA event pair around one kernel phase when profiling is on.
class PhaseTimer {
 public:
  PhaseTimer(ytn_ctx *ctx, int phase, cudaStream_t st) : ctx_(ctx), st_(st) {
    if (!ctx_->prof) return;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st_, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> lk(ctx_->prof_mu);
    if (ctx_->ev_next + 2 > ctx_->ev_pool.size()) {
      ctx_->dropped++;
      return;
    }
    idx_ = (int)ctx_->ev_next;
    ctx_->ev_next += 2;
    ctx_->pending.push_back({phase, idx_});
    cudaEventRecord(static_cast<cudaEvent_t>(ctx_->ev_pool[idx_]), st_);
  }
  ~PhaseTimer() {
    if (idx_ >= 0) cudaEventRecord(static_cast<cudaEvent_t>(ctx_->ev_pool[idx_ + 1]), st_);
  }

 private:
  ytn_ctx *ctx_;
  cudaStream_t st_;
  int idx_ = -1;
};

// The address the kernels use for a caller's data buffer: device memory of the
// context's device as is; page-locked host memory (cudaHostAlloc, or registered
// with cudaHostRegister) through its device mapping, so that the data movers
// read or write it over the host link with no separate copy. Pageable host
// memory and other devices' memory are rejected before anything is launched.
static ytn_status device_view(const ytn_ctx *ctx, const void *ptr, const void **out, const char *what,
                              bool *on_host = nullptr) {
  *out = ptr;
  if (on_host) *on_host = false;
  if (!ptr) return YTN_OK;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(YTN_E_INVALID, std::string(what) + ": not a CUDA-visible pointer");
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
    if (at.type == cudaMemoryTypeDevice && at.device != ctx->device)
      return fail(YTN_E_INVALID, std::string(what) + ": device memory of another GPU");
    return YTN_OK;
  }
  if (at.type == cudaMemoryTypeHost) {
    if (!at.devicePointer) return fail(YTN_E_INVALID, std::string(what) + ": page-locked host memory without a device mapping");
    *out = at.devicePointer;
    if (on_host) *on_host = true;
    return YTN_OK;
  }
  return fail(YTN_E_INVALID, std::string(what) + ": pageable host memory (page-lock it with cudaHostRegister first)");
}

template <class T>
static ytn_status device_view(const ytn_ctx *ctx, T *ptr, T **out, const char *what, bool *on_host = nullptr) {
  const void *v = nullptr;
  ytn_status st = device_view(ctx, static_cast<const void *>(ptr), &v, what, on_host);
  *out = static_cast<T *>(const_cast<void *>(v));
  return st;
}

// A plan used by a launch that is being recorded into a graph stays alive
// until the graph is destroyed.
static void note_capture(ytn_plan_t *p, cudaStream_t st) {
  ytn_ctx *c = p->ctx;
  if (!c->capturing.load()) return;
  std::lock_guard<std::mutex> lk(c->cap_mu);
  if (c->cap_stream != static_cast<void *>(st)) return;
  p->refs++;
  c->cap_plans.push_back(p);
}

// Workspace: WA | WB | WC (FP64 sector matrices), then for the split path
// SA | SB (BF16 slice blocks) | EA | EB (row / column exponents) and the accuracy
// check: EMAX | NORMSQ | REC | SECV | FLAGGED | TILE_END (see SplitRecord);
// 256-byte aligned regions, except that EMAX follows EB and REC follows NORMSQ
// directly so that one memset covers each pair.
struct WsLayout {
  size_t wa = 0, wb = 0, wc = 0, sa = 0, sb = 0, ea = 0, eb = 0;
  size_t emax = 0, emax_end = 0, normsq = 0, rec = 0, rec_end = 0, secv = 0, flagged = 0, tile_end = 0;
  size_t item_end_a = 0, item_end_b = 0;
};

static size_t workspace_layout(const ytn_plan_t *p, bool split, WsLayout &w) {
  size_t o = 0;
  w.wa = o;
  o += align256((size_t)p->a_elems * 8);
  w.wb = o;
  o += align256((size_t)p->b_elems * 8);
  w.wc = o;
  o += align256((size_t)p->c_elems * 8);
  if (!split) return o;
  w.sa = o;
  o += align256((size_t)p->sp_sa_bytes);
  w.sb = o;
  o += align256((size_t)p->sp_sb_bytes);
  w.ea = o;
  o += align256((size_t)p->sp_ea * 4);
  w.eb = o;
  o += (size_t)p->sp_eb * 4;
  const size_t nsec = p->sp_sectors.size();
  w.emax = o;
  o += 2 * nsec * 4;
  w.emax_end = o;
  o = align256(o);
  w.normsq = o;
  o += align256(nsec * 4);
  w.rec = o;
  o += sizeof(SplitRecord);
  w.rec_end = o;
  o = align256(o);
  w.secv = o;
  o += align256(nsec * 8);
  w.flagged = o;
  o += align256(nsec * 4);
  w.tile_end = o;
  o += align256(nsec * 4);
  w.item_end_a = o;
  o += align256(nsec * 4);
  w.item_end_b = o;
  o += align256(nsec * 4);
  return o;
}

// Data-aware estimate (split_check.cu): per element of C_q, the error relative to
// the product of the row and column scales 2^(e_i + f_j), per square root of K.
// Digit rounding and the dropped orders contribute about 2^(-8s-1); the FP32
// rounding of the accumulator of the orders >= 3 about 2^-43 (it is rounded over
// 256 of K at a time at that accumulator's own magnitude, which the digits bound
// relative to the scales). Measured on this GPU over seven value distributions
// (normal, uniform, elements just below a power of two, log-uniform over 2^30,
// rows scaled over 10^60, one dominant element per row and column, cancelling
// products), K from 64 to 16384 and s = 4, 5, 6, the split error stayed below
// half of this estimate. An FP64 product: 2^-52.
static double split_eta(int s) { return std::ldexp(1.0, -8 * s - 1) + std::ldexp(1.0, -43); }
static const double kEtaFp64 = std::ldexp(1.0, -52);

// A-priori estimate that picks the slice count (reported as ytn_result.err_est):
// the data-aware estimate for data spread like a normal distribution, whose row
// and column scales exceed the result by about sqrt(K) times 100 (a scale is
// about (4 max|x|)^2, with max|x| three to four standard deviations over
// thousands of elements, and |c| about sqrt(K) times the variance), so that the
// estimate is 128 eta(s) whatever K. It is a forecast, not a bound: every call
// checks its result on the device (split_check.cu) and recomputes on the FP64
// path the sectors whose data make the estimate exceed rtol. The slice count is
// the smallest s >= 4 whose forecast is at most rtol (s = 5 for rtol = 1e-10).
static double split_error_estimate(int s) { return 128.0 * split_eta(s); }

static ytn_status choose_slices(const ytn_plan_t *p, double rtol, int &s, double &est) {
  if (p->max_k > 16384) return fail(YTN_E_UNSUPPORTED, "split path supports K up to 16384 per sector");
  if (!(rtol > 0.0)) return fail(YTN_E_TOLERANCE, "split path needs rtol > 0");
  for (s = 4; s <= kSlices; s++) {   // orders 0..2 are exact, so at least 4 slices
    est = split_error_estimate(s);
    if (est <= rtol) return YTN_OK;
  }
  est = split_error_estimate(kSlices);
  return fail(YTN_E_TOLERANCE, "rtol below what the split path can reach for this plan");
}

// Times contraction runs enqueued one after another on st (each a callable) and
// returns their durations in ms; synchronises the stream.
static ytn_status time_runs(cudaStream_t st, const std::vector<std::function<ytn_status()>> &runs,
                            std::vector<float> &ms) {
  std::vector<cudaEvent_t> ev(runs.size() + 1);
  for (auto &x : ev) cudaEventCreate(&x);
  cudaEventRecord(ev[0], st);
  ytn_status r = YTN_OK;
  for (size_t i = 0; i < runs.size(); i++) {
    if (r == YTN_OK) r = runs[i]();
    cudaEventRecord(ev[i + 1], st);
  }
  cudaError_t e = cudaEventSynchronize(ev.back());
  ms.assign(runs.size(), 0.f);
  for (size_t i = 0; i < runs.size() && e == cudaSuccess; i++) e = cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
  for (auto &x : ev) cudaEventDestroy(x);
  if (r != YTN_OK) return r;
  return e == cudaSuccess ? YTN_OK : cuda_fail(e, "timing the contraction paths");
}

// The copy launch of items [b, e) of the plan's job table, with the kernel built for
// the most dims those items have (cached per range: a range's items never change).
static cudaError_t copy_range(ytn_plan_t *p, int64_t b, int64_t e, const double *src, double *dst,
                              cudaStream_t st) {
  int nd = kMaxCopyDims;
  if (e > b && e <= (int64_t)p->items.size()) {
    const int64_t key = (b << 32) + e;
    std::lock_guard<std::mutex> lk(p->nd_mu);
    auto it = p->nd_max.find(key);
    if (it != p->nd_max.end()) {
      nd = it->second;
    } else {
      int m = 1;
      for (int64_t i = b; i < e; i++) m = std::max(m, p->items[i].kind & 255);
      p->nd_max.emplace(key, m);
      nd = m;
    }
  }
  return launch_copy(p->d_jobs, p->d_items + b, e - b, src, dst, st, nd);
}

}  // namespace ytn

using namespace ytn;

extern "C" {

const char *ytn_version(void) { return "ytn 0.1 (sm_103a)"; }

const char *ytn_last_error(void) { return g_last_error.c_str(); }

ytn_status ytn_ctx_create(ytn_ctx **ctx, int device) {
  if (!ctx) return fail(YTN_E_INVALID, "null ctx pointer");
  *ctx = nullptr;
  if (device < 0) {  // host-only context: plans without device tables
    ytn_ctx *c = new (std::nothrow) ytn_ctx;
    if (!c) return fail(YTN_E_NOMEM, "host allocation failed");
    c->device = -1;
    *ctx = c;
    return YTN_OK;
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return fail(YTN_E_INVALID, "device out of range");
  ytn_ctx *c = new (std::nothrow) ytn_ctx;
  if (!c) return fail(YTN_E_NOMEM, "host allocation failed");
  c->device = device;
  DeviceGuard g(device);
  if (!g.ok()) {
    delete c;
    return fail(YTN_E_CUDA, "cannot select device");
  }
  e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaDeviceGetAttribute");
  }
  e = configure_split_gemm();
  if (e == cudaSuccess) e = configure_split_blocks();
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "configure split-precision GEMM");
  }
  e = cudaMalloc(&c->status_dev, sizeof(int) * 4);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaMalloc status word");
  }
  e = cudaMemset(c->status_dev, 0, sizeof(int) * 4);
  if (e != cudaSuccess) {
    cudaFree(c->status_dev);
    delete c;
    return cuda_fail(e, "cudaMemset status word");
  }
  // pipelined fused split: the GEMM chain on the highest-priority stream, so that
  // its CTAs take the SMs before the slicing that runs beside them
  {
    int least = 0, greatest = 0;
    cudaStream_t hi = nullptr, lo = nullptr;
    e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&hi, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&lo, cudaStreamNonBlocking, least);
    for (int i = 0; e == cudaSuccess && i < kPipeGroups + 2; i++) {
      cudaEvent_t ev = nullptr;
      e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) c->pipe_ev.push_back(ev);
    }
    c->pipe_hi = hi;
    c->pipe_lo = lo;
    if (e != cudaSuccess) {
      for (void *ev : c->pipe_ev) cudaEventDestroy(static_cast<cudaEvent_t>(ev));
      if (hi) cudaStreamDestroy(hi);
      if (lo) cudaStreamDestroy(lo);
      cudaFree(c->status_dev);
      delete c;
      return cuda_fail(e, "pipeline streams and events");
    }
  }
  *ctx = c;
  return YTN_OK;
}

void ytn_ctx_destroy(ytn_ctx *ctx) {
  if (!ctx) return;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    for (auto &kv : ctx->cache) {
      ytn_plan_t *p = kv.second;
      if (--p->refs == 0) destroy_plan(p);
    }
    ctx->cache.clear();
  }
  if (ctx->device >= 0) {
    DeviceGuard g(ctx->device);
    for (void *ev : ctx->ev_pool) cudaEventDestroy(static_cast<cudaEvent_t>(ev));
    for (void *ev : ctx->pipe_ev) cudaEventDestroy(static_cast<cudaEvent_t>(ev));
    if (ctx->pipe_hi) cudaStreamDestroy(static_cast<cudaStream_t>(ctx->pipe_hi));
    if (ctx->pipe_lo) cudaStreamDestroy(static_cast<cudaStream_t>(ctx->pipe_lo));
    if (ctx->status_dev) cudaFree(ctx->status_dev);
    svd_release(ctx);
  }
  delete ctx;
}

static ytn_status plan_op(ytn_ctx *ctx, const ytn_op *op, int32_t rank, int32_t world, ytn_plan_t **plan) {
  if (!ctx || !op || !plan) return fail(YTN_E_INVALID, "null argument");
  *plan = nullptr;
  if (world < 1 || rank < 0 || rank >= world) return fail(YTN_E_INVALID, "shard rank outside [0, world)");
  if (world > 1 && op->kind != YTN_OP_TENSORDOT) return fail(YTN_E_INVALID, "only tensordot plans are sharded");
  std::string key;
  try {
    key = plan_key(op);
    if (world > 1) {
      key += "|shard";
      key.append(reinterpret_cast<const char *>(&rank), sizeof(rank));
      key.append(reinterpret_cast<const char *>(&world), sizeof(world));
    }
  } catch (...) {
    return fail(YTN_E_NOMEM, "host allocation failed");
  }
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->cache.find(key);
    if (it != ctx->cache.end()) {
      it->second->refs++;
      *plan = it->second;
      return YTN_OK;
    }
  }
  ytn_plan_t *p = new (std::nothrow) ytn_plan_t;
  if (!p) return fail(YTN_E_NOMEM, "host allocation failed");
  p->ctx = ctx;
  p->key = key;
  p->shard_rank = rank;
  p->shard_world = world;
  std::string err;
  ytn_status st = YTN_OK;
  try {
    Tensor A, B;
    st = load_struct(op->a, A, err);
    if (st == YTN_OK) {
      switch (op->kind) {
        case YTN_OP_TENSORDOT:
          st = load_struct(op->b, B, err);
          if (st == YTN_OK) st = plan_tensordot(p, A, B, op->naxes, op->axa, op->axb, err);
          break;
        case YTN_OP_FUSE:
          st = plan_fuse(p, A, op->ngroups, op->group_size, op->order, err);
          break;
        case YTN_OP_UNFUSE:
          if (op->naxes < 1 || op->naxes > YTN_MAX_RANK) {
            st = YTN_E_INVALID;
            err = "naxes out of range";
          } else {
            st = plan_unfuse(p, A, op->naxes, op->axa, err);
          }
          break;
        case YTN_OP_CONJ:
          st = plan_conj(p, A, err);
          break;
        case YTN_OP_SVD:
          st = plan_svd(p, A, op->ngroups, op->group_size, op->order, err);
          if (st == YTN_OK && ctx->device >= 0) {
            DeviceGuard g(ctx->device);
            st = svd_prepare(p);
            if (st != YTN_OK) err = "dense solver set-up failed";
          }
          break;
        case YTN_OP_EIGH:
          st = plan_eigh(p, A, op->ngroups, op->group_size, op->order, err);
          if (st == YTN_OK && ctx->device >= 0) {
            DeviceGuard g(ctx->device);
            st = svd_prepare(p);
            if (st != YTN_OK) err = "dense solver set-up failed";
          }
          break;
        case YTN_OP_SLICE:
          st = plan_slice(p, A, op->naxes, op->axa, op->nkeep, op->keep_t, op->keep_D, err);
          break;
        case YTN_OP_SWAP_GATE:
          st = plan_swap_gate(p, A, op->ngroups, op->group_size, op->order, op->fermionic, err);
          break;
        case YTN_OP_VDOT:
          st = load_struct(op->b, B, err);
          if (st == YTN_OK) st = plan_vdot(p, A, B, err);
          break;
        case YTN_OP_TRACE:
          if (op->naxes < 1 || op->naxes > YTN_MAX_RANK) {
            st = YTN_E_INVALID;
            err = "naxes out of range";
          } else {
            st = plan_trace(p, A, op->naxes, op->axa, op->axb, err);
          }
          break;
        default:
          st = YTN_E_INVALID;
          err = "unknown operation";
      }
    }
    if (st == YTN_OK) finish_output_view(p);
  } catch (const std::bad_alloc &) {
    st = YTN_E_NOMEM;
    err = "host allocation failed";
  }
  if (st != YTN_OK) {
    delete p;
    return fail(st, err);
  }
  if (ctx->device >= 0) {
    DeviceGuard g(ctx->device);
    if (!g.ok()) {
      delete p;
      return fail(YTN_E_CUDA, "cannot select device");
    }
    st = upload(p);
  }
  if (st != YTN_OK) {
    destroy_plan(p);
    return st;
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->cache.find(key);
  if (it != ctx->cache.end()) {  // planned concurrently by another thread
    destroy_plan(p);
    it->second->refs++;
    *plan = it->second;
    return YTN_OK;
  }
  p->refs = 2;  // the caller's reference and the cache's
  ctx->cache[key] = p;
  *plan = p;
  return YTN_OK;
}

ytn_status ytn_plan(ytn_ctx *ctx, const ytn_op *op, ytn_plan_t **plan) { return plan_op(ctx, op, 0, 1, plan); }

ytn_status ytn_plan_shard(ytn_ctx *ctx, const ytn_op *op, int32_t rank, int32_t world, ytn_plan_t **plan) {
  return plan_op(ctx, op, rank, world, plan);
}

// Structure from legs: not cached (the caller holds the only reference).
ytn_status ytn_plan_blocks(ytn_ctx *ctx, ytn_sym sym, int32_t rank, const ytn_leg *legs, const int32_t *n,
                           ytn_plan_t **plan) {
  if (!ctx || !plan) return fail(YTN_E_INVALID, "null argument");
  *plan = nullptr;
  ytn_plan_t *p = new (std::nothrow) ytn_plan_t;
  if (!p) return fail(YTN_E_NOMEM, "host allocation failed");
  p->ctx = ctx;
  std::string err;
  ytn_status st;
  try {
    st = plan_blocks(p, sym, rank, legs, n, err);
    if (st == YTN_OK) finish_output_view(p);
  } catch (const std::bad_alloc &) {
    st = YTN_E_NOMEM;
    err = "host allocation failed";
  }
  if (st != YTN_OK) {
    delete p;
    return fail(st, err);
  }
  if (ctx->device >= 0) {
    DeviceGuard g(ctx->device);
    if (!g.ok()) {
      delete p;
      return fail(YTN_E_CUDA, "cannot select device");
    }
    if ((st = upload(p)) != YTN_OK) {
      destroy_plan(p);
      return st;
    }
  }
  p->refs = 1;
  *plan = p;
  return YTN_OK;
}

ytn_status ytn_fill_normal(ytn_plan_t *p, uint64_t seed, double *out, ytn_stream stream) {
  if (!p) return fail(YTN_E_INVALID, "null plan");
  if (!p->dev) return fail(YTN_E_INVALID, "plan of a host-only context cannot run");
  if (p->out.dtype != YTN_REAL64) return fail(YTN_E_UNSUPPORTED, "normal fill of complex data");
  if (p->out.size && !out) return fail(YTN_E_INVALID, "null data buffer");
  DeviceGuard g(p->ctx->device);
  if (!g.ok()) return fail(YTN_E_CUDA, "cannot select device");
  ytn_status vs = device_view(p->ctx, out, &out, "output");
  if (vs != YTN_OK) return vs;
  cudaError_t e = launch_fill_normal(seed, p->out.size, out, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? YTN_OK : cuda_fail(e, "normal fill");
}

const ytn_struct *ytn_plan_output(const ytn_plan_t *plan) { return plan ? &plan->out_view : nullptr; }

const ytn_struct *ytn_plan_output_at(const ytn_plan_t *plan, int32_t i) {
  if (!plan || i < 0) return nullptr;
  if (i == 0) return &plan->out_view;
  return (size_t)i <= plan->outs_view.size() ? &plan->outs_view[(size_t)i - 1] : nullptr;
}

ytn_status ytn_plan_get_info(const ytn_plan_t *p, ytn_plan_info *info) {
  if (!p || !info) return fail(YTN_E_INVALID, "null argument");
  std::memset(info, 0, sizeof(*info));
  info->useful_flops = p->flops;
  info->nsectors = (int64_t)p->sectors.size();
  info->max_m = p->max_m;
  info->max_n = p->max_n;
  info->max_k = p->max_k;
  info->a_elems = p->a_elems;
  info->b_elems = p->b_elems;
  info->c_elems = p->c_elems;
  info->moved_elems = p->moved;
  info->out_size = p->out.size;
  info->njobs = (int64_t)p->jobs.size();
  info->split_fused = p->sp_fused ? 1 : 0;
  int nd = 0;
  for (const CopyItem &it : p->items) nd = std::max(nd, it.kind & 255);
  info->max_copy_dims = nd;
  info->split_pipe_groups = (int32_t)p->sp_pipe_tile_end.size();
  return YTN_OK;
}

ytn_status ytn_plan_tuning(const ytn_plan_t *p, int32_t slices, ytn_tuning *out) {
  if (!p || !out) return fail(YTN_E_INVALID, "null argument");
  if (slices < 1 || slices > kSlices) return fail(YTN_E_INVALID, "slice count out of range");
  std::lock_guard<std::mutex> lk(const_cast<ytn_plan_t *>(p)->auto_mu);
  std::memset(out, 0, sizeof(*out));
  out->slices = slices;
  out->auto_choice = p->auto_choice[slices];
  out->split_variant = p->split_variant[slices];
  out->tile_policy = p->tile_policy[slices];
  out->fp64_ms = p->auto_ms[slices][0];
  out->split_ms = p->auto_ms[slices][1];
  out->staged_ms = p->variant_ms[slices][0];
  out->fused_ms = p->variant_ms[slices][1];
  out->pipelined_ms = p->variant_ms[slices][2];
  out->wide_ms = p->tile_ms[slices][0];
  out->narrow_ms = p->tile_ms[slices][1];
  return YTN_OK;
}

void ytn_plan_release(ytn_plan_t *plan) {
  if (!plan) return;
  ytn_ctx *ctx = plan->ctx;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (--plan->refs == 0) destroy_plan(plan);
}

// Staging of page-locked host operands through the workspace (copy engines):
// device copies of A, B and C after the contraction's own workspace.
static size_t staging_bytes(const ytn_plan_t *p) {
  const size_t wa = p->a_size * (p->ca == 2 ? 16 : 8), wb = p->b_size * (p->cb == 2 ? 16 : 8);
  const size_t wc = (size_t)p->out.size * (p->out.dtype == YTN_COMPLEX128 ? 16 : 8);
  return align256(wa) + align256(wb) + align256(wc);
}

ytn_status ytn_workspace_size_staged(const ytn_plan_t *p, ytn_precision prec, double rtol, size_t *bytes) {
  ytn_status st = ytn_workspace_size(p, prec, rtol, bytes);
  if (st != YTN_OK) return st;
  if (p->kind != Kind::Tensordot) return fail(YTN_E_INVALID, "staging is for tensordot plans");
  *bytes = align256(*bytes) + staging_bytes(p);
  return YTN_OK;
}

ytn_status ytn_workspace_size(const ytn_plan_t *p, ytn_precision prec, double rtol, size_t *bytes) {
  if (!p || !bytes) return fail(YTN_E_INVALID, "null argument");
  *bytes = 0;
  if (p->kind == Kind::Vdot) {
    *bytes = align256(p->vd_chunks.size() * sizeof(double) * p->cw);
    return YTN_OK;
  }
  if (p->kind == Kind::Svd || p->kind == Kind::Eigh) {
    *bytes = align256((p->svd_ws_doubles + kSolverLanes * p->svd_lwork) * sizeof(double));
    return YTN_OK;
  }
  if (p->kind != Kind::Tensordot) return YTN_OK;
  WsLayout w;
  if (prec == YTN_FP64) {
    *bytes = workspace_layout(p, false, w);
    return YTN_OK;
  }
  if (prec == YTN_SPLIT_BF16) {
    int s;
    double est;
    ytn_status st = choose_slices(p, rtol, s, est);
    if (st != YTN_OK) return st;
    *bytes = workspace_layout(p, true, w);
    return YTN_OK;
  }
  if (prec == YTN_AUTO) {
    int s;
    double est;
    const bool split_ok = choose_slices(p, rtol, s, est) == YTN_OK;
    *bytes = workspace_layout(p, split_ok, w);   // the split layout extends the FP64 one
    return YTN_OK;
  }
  return fail(YTN_E_INVALID, "unknown precision");
}

// One contraction on the chosen path; arguments already checked and mapped.
static ytn_status exec_tensordot(ytn_plan_t *p, const double *a, const double *b, double *c, bool split, int slices,
                                 double rtol, void *workspace, cudaStream_t st, bool fused_variant = false,
                                 bool narrow_tails = false, bool pipelined = false) {
  WsLayout w;
  workspace_layout(p, split, w);
  char *ws = static_cast<char *>(workspace);
  double *wa = reinterpret_cast<double *>(ws + w.wa), *wb = reinterpret_cast<double *>(ws + w.wb),
         *wc = reinterpret_cast<double *>(ws + w.wc);
  cudaError_t e;
  // the fused split builds its slices straight from the blocks and gathers FP64
  // sector matrices only for the sectors its accuracy check recomputes
  const bool fused = split && p->sp_fused && fused_variant;
  if (!fused) {
    if (p->zero_a && (e = cudaMemsetAsync(wa, 0, (size_t)p->a_elems * 8, st)) != cudaSuccess)
      return cuda_fail(e, "memset A workspace");
    if (p->zero_b && (e = cudaMemsetAsync(wb, 0, (size_t)p->b_elems * 8, st)) != cudaSuccess)
      return cuda_fail(e, "memset B workspace");
    {
      PhaseTimer t(p->ctx, YTN_PHASE_GATHER_A, st);
      e = copy_range(p, p->items_a_begin, p->items_a_end, a, wa, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "gather A");
    {
      PhaseTimer t(p->ctx, YTN_PHASE_GATHER_B, st);
      e = copy_range(p, p->items_b_begin, p->items_b_end, b, wb, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "gather B");
  }
  if (!split) {
    PhaseTimer t(p->ctx, YTN_PHASE_GEMM, st);
    e = launch_gemm_fp64(p->d_sectors, p->d_tiles, (int64_t)p->tiles.size(), wa, wb, wc, st);
    if (e != cudaSuccess) return cuda_fail(e, "grouped FP64 GEMM");
  } else {
    int32_t *ea = reinterpret_cast<int32_t *>(ws + w.ea), *eb = reinterpret_cast<int32_t *>(ws + w.eb);
    int32_t *emax = reinterpret_cast<int32_t *>(ws + w.emax);
    float *normsq = reinterpret_cast<float *>(ws + w.normsq);
    SplitRecord *rec = reinterpret_cast<SplitRecord *>(ws + w.rec);
    uint8_t *sa = reinterpret_cast<uint8_t *>(ws + w.sa), *sb = reinterpret_cast<uint8_t *>(ws + w.sb);
    const int sms = p->ctx->gemm_sms.load() > 0 ? p->ctx->gemm_sms.load() : p->ctx->num_sms;
    const size_t ngroups = p->sp_pipe_tile_end.size();
    if (fused && pipelined && ngroups >= 2 && ngroups <= (size_t)kPipeGroups && p->ctx->pipe_hi) {
      // Pipelined: the sectors in groups (the GEMM's order). Group 0 is sliced
      // alone; then each group's GEMM runs while the next groups are sliced beside
      // it on the same SMs (a slicing CTA fits next to a GEMM CTA), and each group's
      // GEMM waits for its slices. The GEMM chain runs on the highest-priority
      // stream, the slicing on the lowest, both forked from and joined to st.
      std::lock_guard<std::mutex> lk(p->ctx->pipe_mu);
      cudaStream_t hi = static_cast<cudaStream_t>(p->ctx->pipe_hi), lo = static_cast<cudaStream_t>(p->ctx->pipe_lo);
      auto ev = [&](size_t i) { return static_cast<cudaEvent_t>(p->ctx->pipe_ev[i]); };
      const std::vector<int64_t> &te = p->sp_pipe_tile_end, &ie = p->sp_pipe_item_end;
      e = cudaEventRecord(ev(0), st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(hi, ev(0), 0);
      if (e == cudaSuccess) {
        PhaseTimer t(p->ctx, YTN_PHASE_SPLIT, hi);
        e = cudaMemsetAsync(ea, 0x80, w.emax_end - w.ea, hi);
        if (e == cudaSuccess) e = cudaMemsetAsync(normsq, 0, w.rec_end - w.normsq, hi);
        if (e == cudaSuccess)
          e = launch_split_blocks(p->d_sp_ops, p->d_sp_fitems, ie[0], p->d_sp_segs, a, b, ea, eb, emax, sa, sb, slices,
                                  false, hi);
      }
      if (e == cudaSuccess) e = cudaEventRecord(ev(1), hi);
      if (e != cudaSuccess) return cuda_fail(e, "split into slices");
      {
        PhaseTimer t(p->ctx, YTN_PHASE_GEMM, hi);
        e = launch_gemm_split(p->d_sp_sectors, p->d_sp_tiles, te[0], sa, sb, ea, eb, emax, normsq, wc, slices,
                              p->ctx->status_dev, sms, false, hi);
        // enqueued after group 0's GEMM, so that its CTAs are dispatched first
        if (e == cudaSuccess) e = cudaStreamWaitEvent(lo, ev(1), 0);
        for (size_t g = 1; g < ngroups && e == cudaSuccess; g++) {
          e = launch_split_blocks(p->d_sp_ops, p->d_sp_fitems + ie[g - 1], ie[g] - ie[g - 1], p->d_sp_segs, a, b, ea,
                                  eb, emax, sa, sb, slices, true, lo);
          if (e == cudaSuccess) e = cudaEventRecord(ev(g + 1), lo);
        }
        for (size_t g = 1; g < ngroups && e == cudaSuccess; g++) {
          e = cudaStreamWaitEvent(hi, ev(g + 1), 0);
          if (e == cudaSuccess)
            e = launch_gemm_split(p->d_sp_sectors, p->d_sp_tiles + te[g - 1], te[g] - te[g - 1], sa, sb, ea, eb, emax,
                                  normsq, wc, slices, p->ctx->status_dev, sms, false, hi);
        }
      }
      if (e == cudaSuccess) e = cudaEventRecord(ev(ngroups + 1), hi);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev(ngroups + 1), 0);
      if (e != cudaSuccess) return cuda_fail(e, "pipelined split-precision GEMM");
    } else {
      {
        PhaseTimer t(p->ctx, YTN_PHASE_SPLIT, st);
        // the exponent kernels max-combine into EA, EB and EMAX: start from a value
        // below every exponent (bytes 0x80: 0x80808080 as int32); the epilogue sums
        // into NORMSQ and the check counts in the record: start from zero
        e = cudaMemsetAsync(ea, 0x80, w.emax_end - w.ea, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(normsq, 0, w.rec_end - w.normsq, st);
        if (e == cudaSuccess) {
          if (fused)
            e = launch_split_blocks(p->d_sp_ops, p->d_sp_fitems, (int64_t)p->sp_fitems.size(), p->d_sp_segs, a, b,
                                    ea, eb, emax, sa, sb, slices, false, st);
          else
            e = launch_split_prep(p->d_sp_ops, p->d_sp_exp_items, (int64_t)p->sp_exp_items.size(),
                                  p->d_sp_slice_items, (int64_t)p->sp_slice_items.size(), wa, wb, ea, eb, emax, sa,
                                  sb, slices, st);
        }
      }
      if (e != cudaSuccess) return cuda_fail(e, "split into slices");
      {
        PhaseTimer t(p->ctx, YTN_PHASE_GEMM, st);
        const bool mix = narrow_tails && !p->sp_tiles_mix.empty();
        e = launch_gemm_split(p->d_sp_sectors, mix ? p->d_sp_tiles_mix : p->d_sp_tiles,
                              (int64_t)(mix ? p->sp_tiles_mix.size() : p->sp_tiles.size()), sa, sb, ea, eb, emax,
                              normsq, wc, slices, p->ctx->status_dev, sms, mix, st);
      }
      if (e != cudaSuccess) return cuda_fail(e, "grouped split-precision GEMM");
    }
    {
      // data-aware error estimate per sector; sectors above rtol recomputed in FP64
      PhaseTimer t(p->ctx, YTN_PHASE_CHECK, st);
      int32_t *flagged = reinterpret_cast<int32_t *>(ws + w.flagged);
      int32_t *tile_end = reinterpret_cast<int32_t *>(ws + w.tile_end);
      int32_t *item_end_a = reinterpret_cast<int32_t *>(ws + w.item_end_a);
      int32_t *item_end_b = reinterpret_cast<int32_t *>(ws + w.item_end_b);
      e = launch_split_check(p->d_sp_sectors, (int64_t)p->sp_sectors.size(), ea, eb, emax, normsq,
                             reinterpret_cast<double *>(ws + w.secv), flagged, tile_end, item_end_a, item_end_b, rec,
                             split_eta(slices), kEtaFp64, rtol, slices, p->ctx->status_dev, st);
      if (e == cudaSuccess && fused && !p->sp_sectors.empty())
        e = launch_gather_flagged(p->d_jobs, p->d_items + p->items_a_begin, p->d_items + p->items_b_begin,
                                  p->d_sp_sectors, p->d_sectors, flagged, item_end_a, item_end_b, rec, a, b, wa, wb,
                                  p->zero_a, p->zero_b, p->ctx->num_sms, st);
      if (e == cudaSuccess && !p->sp_sectors.empty())
        e = launch_gemm_fp64_redo(p->d_sectors, flagged, tile_end, rec, wa, wb, wc, p->ctx->num_sms, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "accuracy check of the split products");
  }
  {
    PhaseTimer t(p->ctx, YTN_PHASE_SCATTER, st);
    if (p->ca * p->cb > 1)
      e = launch_cscatter(p->d_cs_jobs, (int64_t)p->cs_jobs.size(), wc, c, st);
    else
      e = copy_range(p, p->items_c_begin, p->items_c_end, wc, c, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "scatter C");
  return YTN_OK;
}

// Cost model of the two paths (ms): tile-padded tensor-core work at the rates
// the kernels reach on this GPU, plus the HBM traffic of the split operands.
// Used by YTN_AUTO while a stream is being captured (no timing possible).
static bool model_prefers_split(const ytn_plan_t *p, int s) {
  double f64 = 0.0, f16 = 0.0;
  for (const HostSector &h : p->sectors) {
    const double m64 = std::ceil(h.M / 64.0) * 64, n64 = std::ceil(h.N / 64.0) * 64;
    const double m128 = std::ceil(h.M / 128.0) * 128, n128 = std::ceil(h.N / 128.0) * 128;
    const double k32 = std::ceil(h.K / 32.0) * 32;
    f64 += 2.0 * m64 * n64 * (double)h.K;
    f16 += 2.0 * m128 * n128 * k32 * (s * (s + 1) / 2);
  }
  const double t64 = f64 / 1.0e12;
  const double t16 = f16 / 1.3e15 + (double)(p->a_elems + p->b_elems) * (16.0 + 2.0 * s) / 6.0e12 + 5e-6;
  return t16 < t64;
}

// Split-path variant when it cannot be timed (graph capture): the fused one for
// large blocks. The fused kernels read each block in runs along its contiguous
// direction, which pays off once blocks are large; the staged gathers read every
// block linearly, which wins for many small blocks (measured: 3.2e3 elements per
// block, fused 5.10 ms vs staged 5.24 ms per D = 20 step; 183 elements per block,
// fused 0.60 ms vs staged about 0.40 ms at D = 14).
static bool model_prefers_fused(const ytn_plan_t *p) {
  if (!p->sp_fused || p->sp_segs.empty()) return false;
  const double per_seg = (double)(p->a_elems + p->b_elems) / (double)p->sp_segs.size();
  return per_seg >= 1024.0;
}

ytn_status ytn_tensordot(ytn_plan_t *p, const double *a, const double *b, double *c, ytn_precision prec,
                         double rtol, void *workspace, size_t workspace_bytes, ytn_result *res,
                         ytn_stream stream) {
  if (!p) return fail(YTN_E_INVALID, "null plan");
  if (p->kind != Kind::Tensordot) return fail(YTN_E_INVALID, "plan is not a tensordot plan");
  if (!p->dev) return fail(YTN_E_INVALID, "plan of a host-only context cannot run");
  if ((p->a_size && !a) || (p->b_size && !b) || (p->out.size && !c))
    return fail(YTN_E_INVALID, "null data buffer");
  if (prec != YTN_FP64 && prec != YTN_SPLIT_BF16 && prec != YTN_AUTO)
    return fail(YTN_E_INVALID, "unknown precision");
  int slices = 0;
  double est = 0.0;
  bool split_ok = false;
  if (prec == YTN_SPLIT_BF16) {
    ytn_status st = choose_slices(p, rtol, slices, est);
    if (st != YTN_OK) return st;
    split_ok = true;
  } else if (prec == YTN_AUTO) {
    split_ok = choose_slices(p, rtol, slices, est) == YTN_OK;
  }
  WsLayout w;
  const size_t need = workspace_layout(p, split_ok, w);
  if (need && (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255)))
    return fail(YTN_E_WORKSPACE, "workspace missing, too small or not 256-byte aligned");
  DeviceGuard g(p->ctx->device);
  if (!g.ok()) return fail(YTN_E_CUDA, "cannot select device");
  const double *a_host = a, *b_host = b;
  double *c_host_ptr = c;
  bool ha = false, hb = false, hc = false;
  {
    ytn_status vs;
    if ((vs = device_view(p->ctx, a, &a, "A", &ha)) != YTN_OK || (vs = device_view(p->ctx, b, &b, "B", &hb)) != YTN_OK ||
        (vs = device_view(p->ctx, c, &c, "C", &hc)) != YTN_OK)
      return vs;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  note_capture(p, st);
  // Host operands with a workspace large enough for staging: copy engines move
  // them (no SM time, so calls in flight on other streams keep every SM);
  // otherwise the data movers read and write host memory directly.
  bool staged = false;
  if (ha || hb || hc) {
    const size_t base = align256(need);
    staged = workspace && workspace_bytes >= base + staging_bytes(p);
    if (staged) {
      char *sw = static_cast<char *>(workspace) + base;
      const size_t wa = p->a_size * (p->ca == 2 ? 16 : 8), wb = p->b_size * (p->cb == 2 ? 16 : 8);
      double *sa = reinterpret_cast<double *>(sw), *sb = reinterpret_cast<double *>(sw + align256(wa));
      double *sc = reinterpret_cast<double *>(sw + align256(wa) + align256(wb));
      cudaError_t e = cudaSuccess;
      if (ha && wa) e = cudaMemcpyAsync(sa, a_host, wa, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess && hb && wb) e = cudaMemcpyAsync(sb, b_host, wb, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return cuda_fail(e, "staging copy to the device");
      if (ha) a = sa;
      if (hb) b = sb;
      if (hc) c = sc;
    }
  }
  auto unstage = [&]() -> ytn_status {
    if (!staged || !hc || !p->out.size) return YTN_OK;
    const size_t wc = (size_t)p->out.size * (p->out.dtype == YTN_COMPLEX128 ? 16 : 8);
    cudaError_t e = cudaMemcpyAsync(c_host_ptr, c, wc, cudaMemcpyDeviceToHost, st);
    return e == cudaSuccess ? YTN_OK : cuda_fail(e, "staging copy to the host");
  };
  bool split = prec == YTN_SPLIT_BF16;
  auto fill_res = [&](bool sp, int variant) {
    if (!res) return;
    res->useful_flops = p->flops;
    res->precision = sp ? YTN_SPLIT_BF16 : YTN_FP64;
    res->slices = sp ? slices : 0;
    res->err_est = sp ? est : 0.0;
    res->split_variant = sp ? variant : -1;
    res->narrow_tiles = 0;
  };
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const bool capturing = cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone;
  // Choices cached per plan and slice count: YTN_AUTO's FP64 or split, the split
  // path's variant (staged, or fused when the plan has fused tables) and its tile
  // list (all 128 wide, or with 64-wide sector tails when the plan has any). The
  // first call that needs a choice times the candidates on the caller's stream
  // (this call synchronises it; C holds the last candidate's result, a split
  // result); under graph capture cost models decide.
  int choice = 1, variant = 0, tiles = 0;
  if (prec == YTN_AUTO) {
    if (!split_ok) {
      choice = 0;
    } else {
      std::lock_guard<std::mutex> lk(p->auto_mu);
      choice = p->auto_choice[slices];
    }
  }
  const bool has_mix = !p->sp_tiles_mix.empty();
  if (split_ok || split) {
    std::lock_guard<std::mutex> lk(p->auto_mu);
    variant = p->sp_fused ? p->split_variant[slices] : 0;
    tiles = has_mix ? p->tile_policy[slices] : 0;
  }
  const bool may_split = split || (prec == YTN_AUTO && split_ok && choice != 0);
  const bool need_choice = prec == YTN_AUTO && split_ok && choice < 0;
  const bool need_variant = may_split && p->sp_fused && variant < 0;
  const bool need_tiles = may_split && has_mix && tiles < 0;
  if ((need_choice || need_variant || need_tiles) && capturing) {
    std::lock_guard<std::mutex> lk(p->auto_mu);
    if (need_choice && p->auto_choice[slices] < 0) p->auto_choice[slices] = model_prefers_split(p, slices) ? 1 : 0;
    if (p->sp_fused && p->split_variant[slices] < 0) p->split_variant[slices] = model_prefers_fused(p) ? 1 : 0;
    if (has_mix && p->tile_policy[slices] < 0) p->tile_policy[slices] = 0;
    choice = prec == YTN_AUTO ? p->auto_choice[slices] : 1;
    variant = p->sp_fused ? p->split_variant[slices] : 0;
    tiles = has_mix ? p->tile_policy[slices] : 0;
  } else if (need_choice || need_variant || need_tiles) {
    // candidates in a fixed order: FP64 (YTN_AUTO), staged split, fused split (128
    // wide tiles), then the variant of the previous run with 64-wide tails
    const bool with64 = need_choice, withfused = p->sp_fused && !((ha || hb) && !staged), withmix = has_mix;
    const bool withpipe = withfused && p->sp_pipe_tile_end.size() >= 2;
    std::vector<std::function<ytn_status()>> runs;
    if (with64) runs.push_back([&]() { return exec_tensordot(p, a, b, c, false, 0, rtol, workspace, st); });
    runs.push_back([&]() { return exec_tensordot(p, a, b, c, true, slices, rtol, workspace, st, false, false); });
    if (withfused)
      runs.push_back([&]() { return exec_tensordot(p, a, b, c, true, slices, rtol, workspace, st, true, false); });
    if (withpipe)
      runs.push_back(
          [&]() { return exec_tensordot(p, a, b, c, true, slices, rtol, workspace, st, true, false, true); });
    if (withmix)
      runs.push_back(
          [&]() { return exec_tensordot(p, a, b, c, true, slices, rtol, workspace, st, withfused, true); });
    // one round of the candidates; short contractions (a round under 20 ms) get two
    // more and keep each candidate's fastest, so that launch jitter does not decide
    std::vector<float> ms;
    ytn_status r = time_runs(st, runs, ms);
    if (r != YTN_OK) return r;
    float round_ms = 0.f;
    for (float x : ms) round_ms += x;
    for (int rep = 0; rep < 2 && round_ms < 20.f; rep++) {
      std::vector<float> more;
      if ((r = time_runs(st, runs, more)) != YTN_OK) return r;
      for (size_t i = 0; i < ms.size(); i++) ms[i] = std::min(ms[i], more[i]);
    }
    size_t k = 0;
    const float t64 = with64 ? ms[k++] : 0.f;
    const float tst = ms[k++];
    const float tfu = withfused ? ms[k++] : tst;
    const float tpi = withpipe ? ms[k++] : 0.f;
    const float tmx = withmix ? ms[k++] : 0.f;
    const float t128 = withfused ? tfu : tst;   // the 128-wide run of the variant tried with tails
    // the pipelined variant (128-wide tiles) is kept when it beats every other run
    const bool pipe_best = withpipe && tpi < std::min(tst, tfu) && (!withmix || tpi <= tmx);
    {
      std::lock_guard<std::mutex> lk(p->auto_mu);
      if (withfused && p->split_variant[slices] < 0) {
        p->split_variant[slices] = pipe_best ? 2 : tfu < tst ? 1 : 0;
        p->variant_ms[slices][0] = tst;
        p->variant_ms[slices][1] = tfu;
        p->variant_ms[slices][2] = tpi;
      }
      if (withmix) {
        p->tile_policy[slices] = !pipe_best && tmx < t128 ? 1 : 0;
        p->tile_ms[slices][0] = t128;
        p->tile_ms[slices][1] = tmx;
      }
      if (with64) {
        float best = std::min(tst, tfu);
        if (withpipe) best = std::min(best, tpi);
        if (withmix) best = std::min(best, tmx);
        p->auto_choice[slices] = best < t64 ? 1 : 0;
        p->auto_ms[slices][0] = t64;
        p->auto_ms[slices][1] = best;
      }
    }
    // C holds the last candidate's result
    fill_res(true, withmix ? (withfused ? 1 : 0) : withpipe ? 2 : withfused ? 1 : 0);
    if (res) res->narrow_tiles = withmix ? 1 : 0;
    return unstage();
  }
  if (prec == YTN_AUTO) split = choice == 1;
  // operands read straight from host memory go through the staged gathers, which
  // read every block linearly over the host link (the fused kernels read blocks in
  // runs, twice)
  const bool host_direct = (ha || hb) && !staged;
  const bool use_fused = split && p->sp_fused && variant >= 1 && !host_direct;
  // a stream being captured into a graph takes the fused variant unpipelined (the
  // pipeline's streams are shared by the context's calls)
  const bool use_pipe = use_fused && variant == 2 && !capturing;
  const bool use_mix = split && has_mix && tiles == 1 && !use_pipe;
  ytn_status r =
      exec_tensordot(p, a, b, c, split, split ? slices : 0, rtol, workspace, st, use_fused, use_mix, use_pipe);
  if (r != YTN_OK) return r;
  if ((r = unstage()) != YTN_OK) return r;
  fill_res(split, use_pipe ? 2 : use_fused ? 1 : 0);
  if (res) res->narrow_tiles = use_mix ? 1 : 0;
  return YTN_OK;
}

static ytn_status run_move(ytn_plan_t *p, Kind k, const double *a, double *out, ytn_stream stream,
                           const char *what) {
  if (!p) return fail(YTN_E_INVALID, "null plan");
  if (p->kind != k) return fail(YTN_E_INVALID, std::string("plan is not a ") + what + " plan");
  if (!p->dev) return fail(YTN_E_INVALID, "plan of a host-only context cannot run");
  if ((p->a_size && !a) || (p->out.size && !out)) return fail(YTN_E_INVALID, "null data buffer");
  DeviceGuard g(p->ctx->device);
  if (!g.ok()) return fail(YTN_E_CUDA, "cannot select device");
  {
    ytn_status vs;
    if ((vs = device_view(p->ctx, a, &a, "input")) != YTN_OK || (vs = device_view(p->ctx, out, &out, "output")) != YTN_OK)
      return vs;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  note_capture(p, st);
  cudaError_t e;
  const size_t elem_bytes = p->out.dtype == YTN_COMPLEX128 ? 16 : 8;
  if (p->zero_out && (e = cudaMemsetAsync(out, 0, (size_t)p->out.size * elem_bytes, st)) != cudaSuccess)
    return cuda_fail(e, "memset output");
  PhaseTimer t(p->ctx, YTN_PHASE_MOVE, st);
  if (k == Kind::Trace) {
    if ((e = launch_trace(p->d_tr_out, (int64_t)p->tr_out.size(), p->d_tr_contrib, a, out, st)) != cudaSuccess)
      return cuda_fail(e, "trace");
    return YTN_OK;
  }
  if ((e = copy_range(p, p->items_a_begin, p->items_a_end, a, out, st)) !=
      cudaSuccess)
    return cuda_fail(e, what);
  return YTN_OK;
}

ytn_status ytn_fuse(ytn_plan_t *p, const double *a, double *out, ytn_stream stream) {
  return run_move(p, Kind::Fuse, a, out, stream, "fuse");
}

ytn_status ytn_unfuse(ytn_plan_t *p, const double *a, double *out, ytn_stream stream) {
  return run_move(p, Kind::Unfuse, a, out, stream, "unfuse");
}

ytn_status ytn_trace(ytn_plan_t *p, const double *a, double *out, ytn_stream stream) {
  return run_move(p, Kind::Trace, a, out, stream, "trace");
}

ytn_status ytn_swap_gate(ytn_plan_t *p, const double *a, double *out, ytn_stream stream) {
  return run_move(p, Kind::Swap, a, out, stream, "swap-gate");
}

ytn_status ytn_conj(ytn_plan_t *p, const double *a, double *out, ytn_stream stream) {
  return run_move(p, Kind::Conj, a, out, stream, "conj");
}

ytn_status ytn_slice(ytn_plan_t *p, const double *a, double *out, ytn_stream stream) {
  return run_move(p, Kind::Slice, a, out, stream, "slice");
}

static ytn_status run_decomp(ytn_plan_t *p, Kind kind, const double *a, double *u, double *s, double *v,
                             void *workspace, size_t workspace_bytes, ytn_stream stream) {
  if (!p) return fail(YTN_E_INVALID, "null plan");
  if (p->kind != kind) return fail(YTN_E_INVALID, kind == Kind::Svd ? "plan is not an SVD plan" : "plan is not an eigh plan");
  if (!p->dev) return fail(YTN_E_INVALID, "plan of a host-only context cannot run");
  const bool has_v = p->outs.size() > 1;
  if ((p->a_size && !a) || (p->out.size && !u) || (p->outs[0].size && !s) || (has_v && p->outs[1].size && !v))
    return fail(YTN_E_INVALID, "null data buffer");
  const size_t need = align256((p->svd_ws_doubles + kSolverLanes * p->svd_lwork) * sizeof(double));
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255))
    return fail(YTN_E_WORKSPACE, "workspace missing, too small or not 256-byte aligned");
  DeviceGuard g(p->ctx->device);
  if (!g.ok()) return fail(YTN_E_CUDA, "cannot select device");
  {
    ytn_status vs;
    if ((vs = device_view(p->ctx, a, &a, "A")) != YTN_OK || (vs = device_view(p->ctx, u, &u, "U")) != YTN_OK ||
        (vs = device_view(p->ctx, s, &s, "S")) != YTN_OK || (vs = device_view(p->ctx, v, &v, "V")) != YTN_OK)
      return vs;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  double *ws = static_cast<double *>(workspace);
  cudaError_t e;
  if (p->svd_zero_m && (e = cudaMemsetAsync(ws, 0, p->svd_m_doubles * sizeof(double), st)) != cudaSuccess)
    return cuda_fail(e, "memset sector matrices");
  if ((e = copy_range(p, p->items_a_begin, p->items_a_end, a, ws, st)) !=
      cudaSuccess)
    return cuda_fail(e, "gather sector matrices");
  ytn_status r = svd_factor(p, ws, st);
  if (r != YTN_OK) return r;
  if (p->outs[0].size && (e = cudaMemsetAsync(s, 0, (size_t)p->outs[0].size * sizeof(double), st)) != cudaSuccess)
    return cuda_fail(e, "memset S");
  if ((e = copy_range(p, p->items_h_begin, p->items_h_end, ws, ws, st)) !=
      cudaSuccess)
    return cuda_fail(e, "conjugate a factor");
  if ((e = copy_range(p, p->items_b_begin, p->items_b_end, ws, u, st)) !=
          cudaSuccess ||
      (has_v &&
       (e = copy_range(p, p->items_c_begin, p->items_c_end, ws, v, st)) !=
           cudaSuccess) ||
      (e = copy_range(p, p->items_s_begin, p->items_s_end, ws, s, st)) !=
          cudaSuccess)
    return cuda_fail(e, "write the factors");
  return YTN_OK;
}

ytn_status ytn_svd(ytn_plan_t *p, const double *a, double *u, double *s, double *v, void *workspace,
                   size_t workspace_bytes, ytn_stream stream) {
  return run_decomp(p, Kind::Svd, a, u, s, v, workspace, workspace_bytes, stream);
}

ytn_status ytn_eigh(ytn_plan_t *p, const double *a, double *u, double *s, void *workspace, size_t workspace_bytes,
                    ytn_stream stream) {
  return run_decomp(p, Kind::Eigh, a, u, s, nullptr, workspace, workspace_bytes, stream);
}

ytn_status ytn_vdot(ytn_plan_t *p, const double *a, const double *b, double *out, void *workspace,
                    size_t workspace_bytes, ytn_stream stream) {
  if (!p) return fail(YTN_E_INVALID, "null plan");
  if (p->kind != Kind::Vdot) return fail(YTN_E_INVALID, "plan is not a scalar-product plan");
  if (!p->dev) return fail(YTN_E_INVALID, "plan of a host-only context cannot run");
  if ((p->a_size && !a) || (p->b_size && !b) || !out) return fail(YTN_E_INVALID, "null data buffer");
  const size_t need = align256(p->vd_chunks.size() * sizeof(double) * p->cw);
  if (need && (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255)))
    return fail(YTN_E_WORKSPACE, "workspace missing, too small or not 256-byte aligned");
  DeviceGuard g(p->ctx->device);
  if (!g.ok()) return fail(YTN_E_CUDA, "cannot select device");
  {
    ytn_status vs;
    if ((vs = device_view(p->ctx, a, &a, "A")) != YTN_OK || (vs = device_view(p->ctx, b, &b, "B")) != YTN_OK ||
        (vs = device_view(p->ctx, out, &out, "output")) != YTN_OK)
      return vs;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  note_capture(p, st);
  cudaError_t e;
  {
    PhaseTimer t(p->ctx, YTN_PHASE_REDUCE, st);
    e = launch_vdot(p->d_vd_chunks, (int64_t)p->vd_chunks.size(), p->d_vd_pieces, a, b,
                    static_cast<double *>(workspace), out, p->cw == 2, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "scalar product");
  return YTN_OK;
}

ytn_status ytn_ctx_set_gemm_sms(ytn_ctx *ctx, int nsms) {
  if (!ctx) return fail(YTN_E_INVALID, "null ctx");
  if (ctx->device < 0) return fail(YTN_E_INVALID, "host-only context");
  if (nsms < 0 || nsms > ctx->num_sms) return fail(YTN_E_INVALID, "SM count out of range");
  ctx->gemm_sms.store(nsms);
  return YTN_OK;
}

ytn_status ytn_profile_enable(ytn_ctx *ctx, int enable) {
  if (!ctx) return fail(YTN_E_INVALID, "null ctx");
  if (ctx->device < 0) return fail(YTN_E_INVALID, "host-only context");
  std::lock_guard<std::mutex> lk(ctx->prof_mu);
  if (enable && ctx->ev_pool.empty()) {
    DeviceGuard g(ctx->device);
    for (int i = 0; i < 8192; i++) {
      cudaEvent_t ev;
      cudaError_t e = cudaEventCreate(&ev);
      if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
      ctx->ev_pool.push_back(ev);
    }
  }
  ctx->prof = enable != 0;
  return YTN_OK;
}

ytn_status ytn_profile_read(ytn_ctx *ctx, ytn_profile *out) {
  if (!ctx || !out) return fail(YTN_E_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(ctx->prof_mu);
  if (ctx->device < 0) return YTN_OK;
  DeviceGuard g(ctx->device);
  for (auto &pe : ctx->pending) {
    cudaEvent_t e0 = static_cast<cudaEvent_t>(ctx->ev_pool[pe.second]);
    cudaEvent_t e1 = static_cast<cudaEvent_t>(ctx->ev_pool[pe.second + 1]);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
    if (pe.first >= 0 && pe.first < YTN_NPHASES) {
      out->calls[pe.first]++;
      out->ms[pe.first] += ms;
    }
  }
  out->dropped += ctx->dropped;
  ctx->pending.clear();
  ctx->ev_next = 0;
  ctx->dropped = 0;
  return YTN_OK;
}

ytn_status ytn_sync(ytn_ctx *ctx, ytn_stream stream, int64_t timeout_ms) {
  if (!ctx) return fail(YTN_E_INVALID, "null ctx");
  if (ctx->device < 0) return YTN_OK;
  DeviceGuard g(ctx->device);
  if (!g.ok()) return fail(YTN_E_CUDA, "cannot select device");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaStreamQuery(st);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return cuda_fail(e, "stream");
    if (timeout_ms >= 0 &&
        std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count() >
            timeout_ms)
      return fail(YTN_E_TIMEOUT, "stream did not finish within the timeout");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  int word[4] = {0, 0, 0, 0};
  cudaError_t e = cudaMemcpy(word, ctx->status_dev, sizeof(word), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read status word");
  if (word[0] != 0 || word[1] != 0) cudaMemset(ctx->status_dev, 0, sizeof(word));
  if (word[0] != 0)
    return fail(YTN_E_TIMEOUT, "a bounded device wait ran out (status " + std::to_string(word[0]) + ")");
  if (word[1] != 0)
    return fail(YTN_E_TOLERANCE,
                "a split-precision result is estimated above its rtol even after the FP64 recomputation "
                "(ytn_tensordot_report gives the estimate)");
  return YTN_OK;
}

ytn_status ytn_tensordot_report(const ytn_plan_t *p, const void *workspace, ytn_error_report *out,
                                ytn_stream stream) {
  if (!p || !out) return fail(YTN_E_INVALID, "null argument");
  if (p->kind != Kind::Tensordot) return fail(YTN_E_INVALID, "plan is not a tensordot plan");
  if (!p->dev) return fail(YTN_E_INVALID, "plan of a host-only context cannot run");
  std::memset(out, 0, sizeof(*out));
  if (p->sp_sectors.empty()) {   // nothing to multiply: exact
    out->within = 1;
    return YTN_OK;
  }
  if (!workspace) return fail(YTN_E_INVALID, "null workspace");
  DeviceGuard g(p->ctx->device);
  if (!g.ok()) return fail(YTN_E_CUDA, "cannot select device");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "stream");
  WsLayout w;
  workspace_layout(p, true, w);
  SplitRecord r;
  e = cudaMemcpy(&r, static_cast<const char *>(workspace) + w.rec, sizeof(r), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read the accuracy record");
  if (r.valid != 1) return fail(YTN_E_INVALID, "no split-precision call has completed in this workspace");
  out->err_est = r.err_est;
  out->split_err_est = r.split_err_est;
  out->max_sector_est = r.max_sector_est;
  out->fallback_flops = r.fallback_flops;
  out->rtol = r.rtol;
  out->nsectors = r.nsectors;
  out->nfallback = r.nfallback;
  out->within = r.within;
  out->slices = r.slices;
  return YTN_OK;
}

}  // extern "C"
