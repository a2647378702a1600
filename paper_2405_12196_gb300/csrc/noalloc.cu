// Allocation-free contraction entry point.
//
// Some callers cannot allocate device memory for a workspace: code embedded in a
// host application that reserves the whole device memory for its own pool up
// front, or code paths that must not call cudaMalloc because of its latency and
// implicit synchronisation. ytn_tensordot_noalloc runs the FP64 contraction path
// of ytn_tensordot with its workspace taken from a fixed scratch array that
// lives in this library's module for as long as the library is loaded (one copy
// on every GPU that loads it).
//
// The array's host-side name is not a device address: its device address is
// looked up once per device with cudaGetSymbolAddress, with that device current,
// on the first call that runs on that device.
#include <cuda_runtime.h>

#include <mutex>

#include "kernels.hpp"

namespace ytn {

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;   // 64 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {nullptr};

}  // namespace

}  // namespace ytn

using namespace ytn;

extern "C" ytn_status ytn_tensordot_noalloc(ytn_plan_t *plan, const double *a, const double *b, double *c,
                                            ytn_stream stream) {
  if (!plan) return fail(YTN_E_INVALID, "null plan");
  if (plan->kind != Kind::Tensordot) return fail(YTN_E_INVALID, "plan is not a tensordot plan");
  const int dev = plan->ctx ? plan->ctx->device : -1;
  if (dev < 0) return fail(YTN_E_INVALID, "plan of a host-only context cannot run");
  if (dev >= kMaxDevices)
    return fail(YTN_E_UNSUPPORTED, "ytn_tensordot_noalloc serves devices 0.." + std::to_string(kMaxDevices - 1));
  size_t need = 0;
  ytn_status st = ytn_workspace_size(plan, YTN_FP64, 0.0, &need);
  if (st != YTN_OK) return st;
  if (need > kNoAllocScratchBytes)
    return fail(YTN_E_WORKSPACE, "contraction needs " + std::to_string(need) +
                                     " bytes of workspace, more than the 64 MiB static scratch of "
                                     "ytn_tensordot_noalloc; use ytn_tensordot with a caller workspace");
  void *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      int prev = 0;
      cudaError_t e = cudaGetDevice(&prev);
      if (e != cudaSuccess) return fail(YTN_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
      if (prev != dev && (e = cudaSetDevice(dev)) != cudaSuccess)
        return fail(YTN_E_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      const cudaError_t er = prev != dev ? cudaSetDevice(prev) : cudaSuccess;
      if (e != cudaSuccess || !p)
        return fail(YTN_E_CUDA, std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
      if (er != cudaSuccess)
        return fail(YTN_E_CUDA, std::string("restoring the caller's device: ") + cudaGetErrorString(er));
      g_noalloc_ptr[dev] = p;
    }
    scratch = g_noalloc_ptr[dev];
  }
  return ytn_tensordot(plan, a, b, c, YTN_FP64, 0.0, scratch, kNoAllocScratchBytes, nullptr, stream);
}
