// Batched passes: the products of several operators (meshes of uneven size), each with
// its own right-hand sides, captured once into one CUDA graph with an independent
// branch per operator and replayed with a single launch per pass.
//
// Creating a batch first runs every product once outside the capture, so that all
// work vectors exist and the tile widths of the tensor-core translations are tuned;
// the capture then holds only kernel launches.  The graph binds the given x and y
// buffers: a pass reads x and writes y of every member.
#include <string>
#include <vector>

#include "nesa_device.cuh"

struct nesa_batch {
  std::vector<nesa_ctx *> ctx;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  int64_t kernel_nodes = 0;
};

using namespace nesa;

static void batch_free(nesa_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->events) cudaEventDestroy(e);
  delete b;
}

extern "C" {

int nesa_build_batch(const nesa_mesh *meshes, int n, const double *k, const nesa_params *params, nesa_ctx **out) {
  if (!meshes || !k || !params || !out || n < 1 || n > 1024) return NESA_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) out[i] = nullptr;
  for (int i = 0; i < n; ++i) {
    const int st = nesa_build(&meshes[i], k[i], params, &out[i]);
    if (st != NESA_OK) {
      const std::string why = nesa_last_error();
      for (int j = 0; j < i; ++j) {
        nesa_destroy(out[j]);
        out[j] = nullptr;
      }
      set_last_error("nesa_build_batch: mesh " + std::to_string(i) + ": " + why);
      return st;
    }
  }
  return NESA_OK;
}

int nesa_batch_create(nesa_ctx *const *ctxs, int n, const nesa_c128 *const *x, nesa_c128 *const *y, const int *nrhs,
                      int parts, nesa_batch **out) {
  if (!out) return NESA_ERR_INVALID_ARG;
  *out = nullptr;
  if (!ctxs || !x || !y || !nrhs || n < 1 || n > 1024 || (parts & NESA_PART_ALL) == 0 ||
      (parts & ~(NESA_PART_ALL | NESA_PART_MIXED)) != 0)
    return NESA_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i] || !x[i] || !y[i] || nrhs[i] < 1 || nrhs[i] > 64) return NESA_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) {  // the branches of one context would share its work buffers
        set_last_error("nesa_batch_create: a context appears twice in the batch");
        return NESA_ERR_INVALID_ARG;
      }
    if (ctxs[i]->batch_refs > 0 && ctxs[i]->batch_nrhs != nrhs[i]) {
      set_last_error("nesa_batch_create: a member is in another batch with a different number of right-hand sides");
      return NESA_ERR_INVALID_ARG;
    }
  }
  nesa_batch *b = new nesa_batch();
  b->ctx.assign(ctxs, ctxs + n);
  cudaStream_t s0 = nullptr;
  bool capturing = false;
  std::vector<cudaStream_t> saved_stream(n);
  std::vector<bool> saved_prof(n);
  try {
    // eager run: work vectors, tuning
    for (int i = 0; i < n; ++i) {
      ensure_workspace(ctxs[i], nrhs[i]);
      launch_matvec(ctxs[i], (const cplx *)x[i], (cplx *)y[i], nrhs[i], parts);
      check_cuda(cudaStreamSynchronize(ctxs[i]->stream), "batch warm-up");
    }
    check_cuda(cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking), "stream");
    b->streams.push_back(s0);
    for (int i = 0; i < n; ++i) {
      cudaStream_t s;
      check_cuda(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream");
      b->streams.push_back(s);
    }
    for (int i = 0; i < n + 1; ++i) {
      cudaEvent_t e;
      check_cuda(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
      b->events.push_back(e);
    }
    check_cuda(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal), "begin capture");
    capturing = true;
    check_cuda(cudaEventRecord(b->events[0], s0), "fork");
    for (int i = 0; i < n; ++i) {
      nesa_ctx *c = ctxs[i];
      saved_stream[i] = c->stream;
      saved_prof[i] = c->profiling;
      c->stream = b->streams[i + 1];
      c->profiling = false;
      check_cuda(cudaStreamWaitEvent(c->stream, b->events[0], 0), "fork wait");
      launch_matvec(c, (const cplx *)x[i], (cplx *)y[i], nrhs[i], parts);
      check_cuda(cudaEventRecord(b->events[i + 1], c->stream), "join");
      check_cuda(cudaStreamWaitEvent(s0, b->events[i + 1], 0), "join wait");
      c->stream = saved_stream[i];
      c->profiling = saved_prof[i];
    }
    capturing = false;
    check_cuda(cudaStreamEndCapture(s0, &b->graph), "end capture");
    check_cuda(cudaGraphInstantiate(&b->exec, b->graph, 0), "instantiate");
    size_t nn = 0;
    check_cuda(cudaGraphGetNodes(b->graph, nullptr, &nn), "nodes");
    std::vector<cudaGraphNode_t> nodes(nn);
    check_cuda(cudaGraphGetNodes(b->graph, nodes.data(), &nn), "nodes");
    for (cudaGraphNode_t nd : nodes) {
      cudaGraphNodeType t;
      check_cuda(cudaGraphNodeGetType(nd, &t), "node type");
      if (t == cudaGraphNodeTypeKernel) b->kernel_nodes += 1;
    }
  } catch (const Error &e) {
    if (capturing) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(s0, &g);
      if (g) cudaGraphDestroy(g);
      // streams and profiling flags changed inside the capture go back
      for (int i = 0; i < n; ++i)
        for (size_t k = 1; k < b->streams.size(); ++k)
          if (ctxs[i]->stream == b->streams[k]) {
            ctxs[i]->stream = saved_stream[i];
            ctxs[i]->profiling = saved_prof[i];
          }
    }
    set_last_error(e.what);
    batch_free(b);
    return e.status;
  }
  for (int i = 0; i < n; ++i) {
    ctxs[i]->batch_refs += 1;
    ctxs[i]->batch_nrhs = nrhs[i];
  }
  *out = b;
  return NESA_OK;
}

int nesa_batch_launch(nesa_batch *b, void *stream) {
  if (!b || !b->exec) return NESA_ERR_INVALID_ARG;
  cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return NESA_ERR_CUDA;
  }
  return NESA_OK;
}

int nesa_batch_kernels(const nesa_batch *b, int64_t *kernel_nodes) {
  if (!b || !kernel_nodes) return NESA_ERR_INVALID_ARG;
  *kernel_nodes = b->kernel_nodes;
  return NESA_OK;
}

void nesa_batch_destroy(nesa_batch *b) {
  if (!b) return;
  if (b->exec)  // a batch that was created: its members are free to reallocate again
    for (nesa_ctx *c : b->ctx) c->batch_refs -= 1;
  batch_free(b);
}

int nesa_get_tuning(nesa_ctx *c, int32_t *tile_n, float *ms) {
  if (!c || !tile_n || !ms) return NESA_ERR_INVALID_ARG;
  tc_tuning(c, tile_n, ms);
  return NESA_OK;
}

}  // extern "C"
