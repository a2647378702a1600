// Capture of a sequence of library calls into one CUDA graph (batching of
// many contractions: the host launches the whole chain once per replay).
// The graph keeps one reference to every plan whose tables its launches read.
#include <cuda_runtime.h>

#include <new>

#include "kernels.hpp"

struct ytn_graph_s {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<ytn_plan_t *> plans;
};

using namespace ytn;

static void end_capture_state(ytn_ctx *ctx, std::vector<ytn_plan_t *> &plans) {
  std::lock_guard<std::mutex> lk(ctx->cap_mu);
  plans.swap(ctx->cap_plans);
  ctx->cap_plans.clear();
  ctx->cap_stream = nullptr;
  ctx->capturing.store(false);
}

extern "C" {

ytn_status ytn_graph_begin(ytn_ctx *ctx, ytn_stream stream) {
  if (!ctx || ctx->device < 0) return fail(YTN_E_INVALID, "graph capture needs a device context");
  if (!stream) return fail(YTN_E_INVALID, "graph capture needs a created stream, not the default stream");
  {
    std::lock_guard<std::mutex> lk(ctx->cap_mu);
    if (ctx->capturing.load()) return fail(YTN_E_INVALID, "this context is already capturing a graph");
    ctx->cap_stream = stream;
    ctx->cap_plans.clear();
    ctx->capturing.store(true);
  }
  cudaError_t e = cudaStreamBeginCapture(reinterpret_cast<cudaStream_t>(stream), cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    std::vector<ytn_plan_t *> none;
    end_capture_state(ctx, none);
    return fail(YTN_E_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
  }
  return YTN_OK;
}

ytn_status ytn_graph_end(ytn_ctx *ctx, ytn_stream stream, ytn_graph_t **graph) {
  if (!ctx || !graph || !stream) return fail(YTN_E_INVALID, "null argument");
  *graph = nullptr;
  {
    std::lock_guard<std::mutex> lk(ctx->cap_mu);
    if (!ctx->capturing.load() || ctx->cap_stream != stream)
      return fail(YTN_E_INVALID, "this stream is not capturing for this context");
  }
  std::vector<ytn_plan_t *> plans;
  end_capture_state(ctx, plans);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(reinterpret_cast<cudaStream_t>(stream), &g);
  ytn_graph_t *out = e == cudaSuccess ? new (std::nothrow) ytn_graph_t : nullptr;
  if (out) {
    out->graph = g;
    out->plans.swap(plans);
    e = cudaGraphInstantiate(&out->exec, g, 0);
    if (e == cudaSuccess) {
      *graph = out;
      return YTN_OK;
    }
    plans.swap(out->plans);
    delete out;
  }
  if (g) cudaGraphDestroy(g);
  for (ytn_plan_t *p : plans) ytn_plan_release(p);
  if (e == cudaSuccess) return fail(YTN_E_NOMEM, "host allocation failed");
  return fail(YTN_E_CUDA, std::string("graph capture or instantiation: ") + cudaGetErrorString(e));
}

ytn_status ytn_graph_launch(ytn_graph_t *graph, ytn_stream stream) {
  if (!graph) return fail(YTN_E_INVALID, "null graph");
  cudaError_t e = cudaGraphLaunch(graph->exec, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail(YTN_E_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
  return YTN_OK;
}

void ytn_graph_destroy(ytn_graph_t *graph) {
  if (!graph) return;
  if (graph->exec) cudaGraphExecDestroy(graph->exec);
  if (graph->graph) cudaGraphDestroy(graph->graph);
  for (ytn_plan_t *p : graph->plans) ytn_plan_release(p);
  delete graph;
}

}  // extern "C"
