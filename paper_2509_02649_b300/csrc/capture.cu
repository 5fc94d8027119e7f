// Capture of library calls into one CUDA graph (fk_capture_begin / fk_capture_end /
// fk_graph_*): a fit's whole launch sequence (the additive model's 36 transforms,
// Gram assembly and dense solve, say) is recorded once and replayed with one graph
// launch, on the same buffers, for new data written into them.
//
// While a capture is active on a host thread, the library's calls on that thread:
//  * take scratch memory as graph allocation nodes (cudaMallocAsync on the capturing
//    stream, freed inside the graph);
//  * report device-side conditions into one flag word owned by the graph, zeroed at
//    the start of every replay and read by fk_graph_status;
//  * never synchronise: calls whose path needs a host round trip (conjugate gradients
//    other than the 2-D single-launch solver, the held-out loss, streaming sums,
//    per-call reports, autotuning) refuse with FK_EINVAL instead of being recorded;
//  * bracket the main spreading kernel with event record nodes, so that its time in
//    the last replay can be read (fk_graph_kernel_ms).
#include "fk_internal.cuh"

struct fk_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned* flags = nullptr;
  cudaStream_t last = nullptr;  // stream of the last launch (may be the legacy stream)
  bool launched = false;
  cudaEvent_t kstart = nullptr, kstop = nullptr;  // main spreading kernel, if recorded
  bool timed = false;
};

namespace fk {

namespace {
thread_local CaptureCtx* g_cap = nullptr;
}

CaptureCtx* capture_ctx() { return g_cap; }

fk_status capture_check(cudaStream_t st, bool capturable, bool wants_report, const char* what) {
  CaptureCtx* c = g_cap;
  if (!c) return FK_OK;
  if (st != c->st) return set_error(FK_EINVAL, "%s: capture is active on another stream", what);
  if (wants_report) return set_error(FK_EINVAL, "%s: a report synchronises, not capturable", what);
  if (!capturable) return set_error(FK_EINVAL, "%s needs a host round trip: not capturable", what);
  return FK_OK;
}

}  // namespace fk

using namespace fk;

extern "C" {

fk_status fk_capture_begin(void* stream) {
  clear_error();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (g_cap) return set_error(FK_EINVAL, "a capture is already active on this thread");
  if (!st) return set_error(FK_EINVAL, "capture needs a created stream (not the legacy default stream)");
  CaptureCtx* c = new CaptureCtx{};
  c->st = st;
  if (cudaMalloc(&c->flags, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return set_error(FK_ENOMEM, "capture flag word");
  }
  if (cudaEventCreate(&c->kstart) != cudaSuccess || cudaEventCreate(&c->kstop) != cudaSuccess) {
    cudaGetLastError();
    if (c->kstart) cudaEventDestroy(c->kstart);
    if (c->kstop) cudaEventDestroy(c->kstop);
    cudaFree(c->flags);
    delete c;
    return set_error(FK_ECUDA, "capture events");
  }
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->flags, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(st, &g);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    cudaEventDestroy(c->kstart);
    cudaEventDestroy(c->kstop);
    cudaFree(c->flags);
    delete c;
    return set_error(FK_ECUDA, "stream capture: %s", cudaGetErrorString(e));
  }
  g_cap = c;
  return FK_OK;
}

fk_status fk_capture_end(void* stream, fk_graph** out) {
  CaptureCtx* c = g_cap;
  if (!out) return set_error(FK_EINVAL, "null graph output");
  *out = nullptr;
  if (!c) return set_error(FK_EINVAL, "no capture is active on this thread");
  if (static_cast<cudaStream_t>(stream) != c->st) return set_error(FK_EINVAL, "capture is active on another stream");
  g_cap = nullptr;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->st, &g);
  const bool failed = c->failed;
  if (e != cudaSuccess || failed || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    cudaEventDestroy(c->kstart);
    cudaEventDestroy(c->kstop);
    cudaFree(c->flags);
    delete c;
    if (failed) return set_error(FK_EINVAL, "a captured call failed; the graph is discarded");
    return set_error(FK_ECUDA, "end of stream capture: %s", cudaGetErrorString(e));
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, g, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    cudaEventDestroy(c->kstart);
    cudaEventDestroy(c->kstop);
    cudaFree(c->flags);
    delete c;
    return set_error(FK_ECUDA, "graph instantiation: %s", cudaGetErrorString(e));
  }
  fk_graph* r = new fk_graph{};
  r->graph = g;
  r->exec = exec;
  r->flags = c->flags;
  r->kstart = c->kstart;
  r->kstop = c->kstop;
  r->timed = c->timed;
  delete c;
  *out = r;
  clear_error();
  return FK_OK;
}

fk_status fk_graph_launch(fk_graph* g, void* stream) {
  clear_error();
  if (!g) return set_error(FK_EINVAL, "null graph");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_CUDA(cudaGraphLaunch(g->exec, st));
  note_launch();
  g->last = st;
  g->launched = true;
  return FK_OK;
}

fk_status fk_graph_status(fk_graph* g) {
  clear_error();
  if (!g) return set_error(FK_EINVAL, "null graph");
  unsigned h = 0;
  if (g->launched) FK_CUDA(cudaStreamSynchronize(g->last));
  FK_CUDA(cudaMemcpy(&h, g->flags, sizeof(unsigned), cudaMemcpyDeviceToHost));
  return flags_status(h);
}

fk_status fk_graph_destroy(fk_graph* g) {
  clear_error();
  if (!g) return FK_OK;
  if (g->launched) cudaStreamSynchronize(g->last);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->flags) cudaFree(g->flags);
  if (g->kstart) cudaEventDestroy(g->kstart);
  if (g->kstop) cudaEventDestroy(g->kstop);
  delete g;
  return FK_OK;
}

fk_status fk_graph_kernel_ms(fk_graph* g, float* ms) {
  clear_error();
  if (!g || !ms) return set_error(FK_EINVAL, "null argument");
  if (!g->timed) return set_error(FK_EINVAL, "the captured calls ran no timed spreading kernel");
  if (!g->launched) return set_error(FK_EINVAL, "the graph has not been launched");
  FK_CUDA(cudaEventSynchronize(g->kstop));
  FK_CUDA(cudaEventElapsedTime(ms, g->kstart, g->kstop));
  return FK_OK;
}

}  // extern "C"
