// Dense factorisation of the sector matrices of a block-diagonal SVD with the
// CUDA toolkit's dense solver (SVD by polar decomposition, one call per sector on
// the caller's stream). The paper leaves the SVD of the fused enlarged corner to its backend's
// linear algebra; this file only drives the library. Gathers and scatters around
// it are the planner's copy jobs (api.cu).
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <string>
#include <system_error>
#include <thread>
#include <vector>

#include "ytn_internal.hpp"

namespace ytn {

static const char *solver_error(cusolverStatus_t s) {
  switch (s) {
    case CUSOLVER_STATUS_NOT_INITIALIZED: return "solver not initialised";
    case CUSOLVER_STATUS_ALLOC_FAILED: return "solver allocation failed";
    case CUSOLVER_STATUS_INVALID_VALUE: return "solver: invalid value";
    case CUSOLVER_STATUS_EXECUTION_FAILED: return "solver execution failed";
    case CUSOLVER_STATUS_INTERNAL_ERROR: return "solver internal error";
    default: return "solver error";
  }
}

// Once per context: kSolverLanes solver handles, each with its parameters, its
// stream and an event. Then the largest device and host buffers of the plan's
// solver calls (polar-decomposition SVD, or the divide-and-conquer Hermitian
// eigensolver; the former measured 3-7 times faster than the Jacobi and QR SVDs).
ytn_status svd_prepare(ytn_plan_t *p) {
  ytn_ctx *ctx = p->ctx;
  std::lock_guard<std::mutex> lk(ctx->solver_mu);
  while ((int)ctx->solvers.size() < kSolverLanes) {
    cusolverDnHandle_t h = nullptr;
    cusolverDnParams_t prm = nullptr;
    cudaStream_t sm = nullptr;
    cudaEvent_t ev = nullptr;
    cusolverStatus_t s = cusolverDnCreate(&h);
    if (s == CUSOLVER_STATUS_SUCCESS) s = cusolverDnCreateParams(&prm);
    if (s != CUSOLVER_STATUS_SUCCESS) {
      if (h) cusolverDnDestroy(h);
      return fail(YTN_E_CUDA, std::string("solver set-up: ") + solver_error(s));
    }
    if (cudaStreamCreateWithFlags(&sm, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cusolverDnDestroyParams(prm);
      cusolverDnDestroy(h);
      if (sm) cudaStreamDestroy(sm);
      return fail(YTN_E_CUDA, "solver stream set-up failed");
    }
    ctx->solvers.push_back(h);
    ctx->solver_params.push_back(prm);
    ctx->solver_streams.push_back(sm);
    ctx->solver_events.push_back(ev);
  }
  auto h = static_cast<cusolverDnHandle_t>(ctx->solvers[0]);
  auto prm = static_cast<cusolverDnParams_t>(ctx->solver_params[0]);
  size_t dev_bytes = 0, host_bytes = 0;
  const cudaDataType T = p->out.dtype == YTN_COMPLEX128 ? CUDA_C_64F : CUDA_R_64F;
  for (const SvdSector &sv : p->svd_sec) {
    if (sv.k == 0) continue;
    const int64_t rows = std::max(sv.m, sv.n), cols = sv.k;
    size_t d = 0, hb = 0;
    cusolverStatus_t s =
        p->kind == Kind::Eigh
            ? cusolverDnXsyevd_bufferSize(h, prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, sv.m, T, nullptr,
                                          sv.m, CUDA_R_64F, nullptr, T, &d, &hb)
            : cusolverDnXgesvdp_bufferSize(h, prm, CUSOLVER_EIG_MODE_VECTOR, 1, rows, cols, T, nullptr, rows,
                                           CUDA_R_64F, nullptr, T, nullptr, rows, T, nullptr, cols, T, &d, &hb);
    if (s != CUSOLVER_STATUS_SUCCESS) return fail(YTN_E_CUDA, std::string("buffer size: ") + solver_error(s));
    dev_bytes = std::max(dev_bytes, d);
    host_bytes = std::max(host_bytes, hb);
  }
  p->svd_lwork = (dev_bytes + 255) / 256 * 256 / sizeof(double);
  p->svd_host_ws.assign(kSolverLanes, std::vector<char>(std::max<size_t>(host_bytes, 8), 0));
  return YTN_OK;
}

// X = M^T (n >= m) or X = M (trans): X = U_x S V_x^H; the factor with m rows is
// F_m, the one with n rows F_n (see SvdSector). Sectors go to the lanes largest
// first, each to the least loaded lane; a host thread per lane issues its calls
// (the solver waits for its host part), the lanes' streams start after the
// caller's stream and the caller's stream continues after all of them.
ytn_status svd_factor(ytn_plan_t *p, double *ws, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ytn_ctx *ctx = p->ctx;
  std::lock_guard<std::mutex> lk(ctx->solver_mu);
  if ((int)ctx->solvers.size() < kSolverLanes) return fail(YTN_E_INVALID, "SVD plan without a solver");
  int *info = reinterpret_cast<int *>(ws + p->svd_info_off);
  const bool cplx = p->out.dtype == YTN_COMPLEX128;
  const cudaDataType T = cplx ? CUDA_C_64F : CUDA_R_64F;
  const int64_t w = cplx ? 2 : 1;   // element offsets -> doubles
  std::vector<std::pair<double, size_t>> order;
  for (size_t i = 0; i < p->svd_sec.size(); i++)
    if (p->svd_sec[i].k > 0) order.push_back({(double)p->svd_sec[i].m * p->svd_sec[i].n * p->svd_sec[i].k, i});
  std::sort(order.begin(), order.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
  std::vector<std::vector<size_t>> lane(kSolverLanes);
  std::vector<double> load(kSolverLanes, 0.0);
  for (auto &o : order) {
    const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    lane[l].push_back(o.second);
    load[l] += o.first;
  }
  cudaEvent_t start = static_cast<cudaEvent_t>(ctx->solver_events[0]);
  if (cudaEventRecord(start, st) != cudaSuccess) return fail(YTN_E_CUDA, "record event");
  for (int l = 0; l < kSolverLanes; l++)
    if (cudaStreamWaitEvent(static_cast<cudaStream_t>(ctx->solver_streams[l]), start, 0) != cudaSuccess)
      return fail(YTN_E_CUDA, "stream wait");
  std::vector<cusolverStatus_t> result(kSolverLanes, CUSOLVER_STATUS_SUCCESS);
  auto work = [&](int l) {
    if (l > 0 && cudaSetDevice(ctx->device) != cudaSuccess) {   // a new thread starts on device 0
      result[l] = CUSOLVER_STATUS_EXECUTION_FAILED;
      return;
    }
    auto h = static_cast<cusolverDnHandle_t>(ctx->solvers[l]);
    auto prm = static_cast<cusolverDnParams_t>(ctx->solver_params[l]);
    cusolverStatus_t s = cusolverDnSetStream(h, static_cast<cudaStream_t>(ctx->solver_streams[l]));
    double *buf = ws + p->svd_ws_doubles + (size_t)l * p->svd_lwork;
    std::vector<char> &hbuf = p->svd_host_ws[l];
    for (size_t i : lane[l]) {
      if (s != CUSOLVER_STATUS_SUCCESS) break;
      const SvdSector &sv = p->svd_sec[i];
      const int64_t rows = std::max(sv.m, sv.n), cols = sv.k;
      double *ux = ws + w * (sv.trans ? sv.vp_off : sv.up_off);   // rows x k
      double *vx = ws + w * (sv.trans ? sv.up_off : sv.vp_off);   // cols x k
      double err_sigma = 0.0;
      if (p->kind == Kind::Eigh)   // M (column-major, Hermitian: its lower triangle) -> eigenvectors in place
        s = cusolverDnXsyevd(h, prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, sv.m, T, ws + w * sv.m_off,
                             sv.m, CUDA_R_64F, ws + sv.s_off, T, buf, p->svd_lwork * sizeof(double), hbuf.data(),
                             hbuf.size(), info + i);
      else
        s = cusolverDnXgesvdp(h, prm, CUSOLVER_EIG_MODE_VECTOR, 1, rows, cols, T, ws + w * sv.m_off, rows, CUDA_R_64F,
                              ws + sv.s_off, T, ux, rows, T, vx, cols, T, buf, p->svd_lwork * sizeof(double),
                              hbuf.data(), hbuf.size(), info + i, &err_sigma);
    }
    result[l] = s;
  };
  {
    // a lane whose thread cannot be started runs on the calling thread instead
    std::vector<std::thread> threads;
    std::vector<int> here{0};
    threads.reserve(kSolverLanes);
    here.reserve(kSolverLanes);
    for (int l = 1; l < kSolverLanes; l++) {
      if (lane[l].empty()) continue;
      try {
        threads.emplace_back(work, l);
      } catch (const std::system_error &) {
        here.push_back(l);
      }
    }
    for (int l : here) work(l);
    for (auto &t : threads) t.join();
  }
  for (int l = 0; l < kSolverLanes; l++) {
    auto ev = static_cast<cudaEvent_t>(ctx->solver_events[l]);
    if (cudaEventRecord(ev, static_cast<cudaStream_t>(ctx->solver_streams[l])) != cudaSuccess ||
        cudaStreamWaitEvent(st, ev, 0) != cudaSuccess)
      return fail(YTN_E_CUDA, "join the solver streams");
  }
  for (int l = 0; l < kSolverLanes; l++)
    if (result[l] != CUSOLVER_STATUS_SUCCESS)
      return fail(YTN_E_CUDA, std::string(p->kind == Kind::Eigh ? "eigensolver: " : "SVD: ") + solver_error(result[l]));
  return YTN_OK;
}

void svd_release(ytn_ctx *ctx) {
  for (void *x : ctx->solver_params) cusolverDnDestroyParams(static_cast<cusolverDnParams_t>(x));
  for (void *x : ctx->solvers) cusolverDnDestroy(static_cast<cusolverDnHandle_t>(x));
  for (void *x : ctx->solver_streams) cudaStreamDestroy(static_cast<cudaStream_t>(x));
  for (void *x : ctx->solver_events) cudaEventDestroy(static_cast<cudaEvent_t>(x));
  ctx->solvers.clear();
  ctx->solver_params.clear();
  ctx->solver_streams.clear();
  ctx->solver_events.clear();
}

}  // namespace ytn
