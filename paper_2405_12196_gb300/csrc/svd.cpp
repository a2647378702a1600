// Dense factorisation of the sector matrices of a block-diagonal SVD with the
// CUDA toolkit's dense solver (Jacobi SVD, one call per sector on the caller's
// stream). The paper leaves the SVD of the fused enlarged corner to its backend's
// linear algebra; this file only drives the library. Gathers and scatters around
// it are the planner's copy jobs (api.cu).
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <string>

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

// Once per context: the solver handle and the Jacobi parameters (sorted,
// descending singular values; default tolerance and sweeps). Then the largest
// solver buffer over the plan's sectors.
ytn_status svd_prepare(ytn_plan_t *p) {
  ytn_ctx *ctx = p->ctx;
  std::lock_guard<std::mutex> lk(ctx->solver_mu);
  if (!ctx->solver) {
    cusolverDnHandle_t h = nullptr;
    cusolverStatus_t s = cusolverDnCreate(&h);
    if (s != CUSOLVER_STATUS_SUCCESS) return fail(YTN_E_CUDA, std::string("create: ") + solver_error(s));
    gesvdjInfo_t prm = nullptr;
    s = cusolverDnCreateGesvdjInfo(&prm);
    if (s == CUSOLVER_STATUS_SUCCESS) s = cusolverDnXgesvdjSetSortEig(prm, 1);
    if (s != CUSOLVER_STATUS_SUCCESS) {
      cusolverDnDestroy(h);
      return fail(YTN_E_CUDA, std::string("parameters: ") + solver_error(s));
    }
    ctx->solver = h;
    ctx->svd_params = prm;
  }
  auto h = static_cast<cusolverDnHandle_t>(ctx->solver);
  auto prm = static_cast<gesvdjInfo_t>(ctx->svd_params);
  int lwork = 0;
  for (const SvdSector &sv : p->svd_sec) {
    if (sv.k == 0) continue;
    int lw = 0;
    // the sector matrix is factored as its column-major transpose, n x m
    cusolverStatus_t s = cusolverDnDgesvdj_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, 1, (int)sv.n, (int)sv.m, nullptr,
                                                      (int)sv.n, nullptr, nullptr, (int)sv.n, nullptr, (int)sv.m, &lw,
                                                      prm);
    if (s != CUSOLVER_STATUS_SUCCESS) return fail(YTN_E_CUDA, std::string("buffer size: ") + solver_error(s));
    lwork = std::max(lwork, lw);
  }
  p->svd_lwork = (size_t)lwork;
  return YTN_OK;
}

// M_c (row-major m x n) is, column-major, M^T (n x m) = U' S V'^T, so that
// M = V' S U'^T: V' (m x k) gives U's columns and U'^T gives V's rows.
ytn_status svd_factor(ytn_plan_t *p, double *ws, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ytn_ctx *ctx = p->ctx;
  std::lock_guard<std::mutex> lk(ctx->solver_mu);
  auto h = static_cast<cusolverDnHandle_t>(ctx->solver);
  auto prm = static_cast<gesvdjInfo_t>(ctx->svd_params);
  if (!h) return fail(YTN_E_INVALID, "SVD plan without a solver");
  cusolverStatus_t s = cusolverDnSetStream(h, st);
  if (s != CUSOLVER_STATUS_SUCCESS) return fail(YTN_E_CUDA, std::string("set stream: ") + solver_error(s));
  int *info = reinterpret_cast<int *>(ws + p->svd_info_off);
  double *work = ws + p->svd_ws_doubles;
  for (size_t i = 0; i < p->svd_sec.size(); i++) {
    const SvdSector &sv = p->svd_sec[i];
    if (sv.k == 0) continue;
    s = cusolverDnDgesvdj(h, CUSOLVER_EIG_MODE_VECTOR, 1, (int)sv.n, (int)sv.m, ws + sv.m_off, (int)sv.n,
                          ws + sv.s_off, ws + sv.up_off, (int)sv.n, ws + sv.vp_off, (int)sv.m, work,
                          (int)p->svd_lwork, info + i, prm);
    if (s != CUSOLVER_STATUS_SUCCESS) return fail(YTN_E_CUDA, std::string("Jacobi SVD: ") + solver_error(s));
  }
  return YTN_OK;
}

void svd_release(ytn_ctx *ctx) {
  if (ctx->svd_params) cusolverDnDestroyGesvdjInfo(static_cast<gesvdjInfo_t>(ctx->svd_params));
  if (ctx->solver) cusolverDnDestroy(static_cast<cusolverDnHandle_t>(ctx->solver));
  ctx->svd_params = nullptr;
  ctx->solver = nullptr;
}

}  // namespace ytn
