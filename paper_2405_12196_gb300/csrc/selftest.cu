// Self-test of the device failure path. Every device wait of the library is
// bounded: when the bound is reached, the kernel records a code in its
// context's status word and returns, and ytn_sync reports YTN_E_TIMEOUT. This
// launches a one-thread kernel that waits, with a bound of about two
// milliseconds, for a flag that nothing ever sets, so that a caller (or a test)
// can see that path work end to end without faulting or hanging the GPU.
#include <cuda_runtime.h>

#include "kernels.hpp"

namespace ytn {

namespace {

constexpr int kSelftestCode = 99;

__global__ void wait_for_nothing_kernel(const volatile int *flag, int *status, unsigned polls) {
  if (threadIdx.x != 0) return;
  for (unsigned i = 0; i < polls; i++) {
    if (*flag) return;
    __nanosleep(1000);
  }
  atomicCAS(status, 0, kSelftestCode);
}

}  // namespace

}  // namespace ytn

using namespace ytn;

extern "C" ytn_status ytn_selftest_timeout(ytn_ctx *ctx, ytn_stream stream) {
  if (!ctx) return fail(YTN_E_INVALID, "null ctx");
  if (ctx->device < 0) return fail(YTN_E_INVALID, "host-only context");
  int prev = 0;
  cudaError_t e = cudaGetDevice(&prev);
  if (e == cudaSuccess && prev != ctx->device) e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return fail(YTN_E_CUDA, std::string("select device: ") + cudaGetErrorString(e));
  // word 3 of the status area is never written by any kernel: it stays zero
  wait_for_nothing_kernel<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(ctx->status_dev + 3,
                                                                               ctx->status_dev, 2000u);
  e = cudaGetLastError();
  if (prev != ctx->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return fail(YTN_E_CUDA, std::string("self-test launch: ") + cudaGetErrorString(e));
  return YTN_OK;
}
