// Batched key switching (Section IV-A batching, Section IV-C CUDA Graphs):
// a plan captures every item's pipeline into one CUDA graph; launching the
// plan replays the graph on the caller's stream with one host call.
#include <cstring>
#include <vector>

#include "../../include/fhe.h"
#include "ctx.h"
#include "internal.h"

struct fhe_plan {
  fhe_ctx *ctx = nullptr;
  std::vector<fhe_ks_item> items;
  int flags = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;
};

static int enqueue_items(fhe_ctx *c, const std::vector<fhe_ks_item> &items, cudaStream_t s) {
  for (const fhe_ks_item &it : items) {
    int rc;
    switch (it.op) {
      case FHE_OP_KS: rc = fhe_keyswitch(c, it.in, it.level, it.rot, it.out, s); break;
      case FHE_OP_ROTATE: rc = fhe_rotate(c, it.in, it.level, it.rot, it.out, s); break;
      case FHE_OP_RELIN: rc = fhe_hmult(c, it.in, it.in2, it.level, it.out, s); break;
      default: rc = fhe_fail(FHE_EINVAL, "fhe_batch: op %d", it.op);
    }
    if (rc != FHE_OK) return rc;
  }
  return FHE_OK;
}

extern "C" int fhe_batch_plan(fhe_ctx *c, const fhe_ks_item *items, int n, int flags, fhe_plan **out) {
  if (!c || !out || n < 0 || (n > 0 && !items)) return fhe_fail(FHE_EINVAL, "fhe_batch_plan: bad arguments");
  *out = nullptr;
  for (int i = 0; i < n; i++) {
    const fhe_ks_item &it = items[i];
    if (it.level < 1 || it.level > c->L) return fhe_fail(FHE_ELEVEL, "fhe_batch_plan: item %d level %d", i, it.level);
    if (!it.in || !it.out || (it.op == FHE_OP_RELIN && !it.in2))
      return fhe_fail(FHE_EINVAL, "fhe_batch_plan: item %d has a null buffer", i);
    if (it.op == FHE_OP_RELIN && !c->relin_key) return fhe_fail(FHE_ENOKEY, "fhe_batch_plan: no relinearisation key");
    if ((it.op == FHE_OP_ROTATE && fhe_galois_elt(it.rot, c->N) != 1u) || it.op == FHE_OP_KS)
      if (!c->find_key(it.rot)) return fhe_fail(FHE_ENOKEY, "fhe_batch_plan: item %d has no key", i);
  }
  fhe_plan *p = new fhe_plan();
  p->ctx = c;
  p->items.assign(items, items + n);
  p->flags = flags;
  if (flags & FHE_PLAN_GRAPH) {
    cudaSetDevice(c->device);
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
      delete p;
      return fhe_fail(FHE_ECUDA, "fhe_batch_plan: stream");
    }
    // the capture must not race with work already queued on this context
    if (c->have_last) cudaStreamSynchronize(c->last_stream);
    fhe::Tracer *saved_tracer = c->tabs.tracer;
    c->tabs.tracer = nullptr;  // no trace events inside a captured graph
    c->capturing = true;
    int rc = FHE_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      rc = fhe_fail(FHE_ECUDA, "fhe_batch_plan: begin capture");
    if (rc == FHE_OK) rc = enqueue_items(c, p->items, cs);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    c->capturing = false;
    c->tabs.tracer = saved_tracer;
    if (rc == FHE_OK && e != cudaSuccess) rc = fhe_fail(FHE_ECUDA, "fhe_batch_plan: end capture: %s", cudaGetErrorString(e));
    if (rc == FHE_OK && cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess)
      rc = fhe_fail(FHE_ECUDA, "fhe_batch_plan: instantiate");
    cudaStreamDestroy(cs);
    if (rc != FHE_OK) {
      if (g) cudaGraphDestroy(g);
      delete p;
      return rc;
    }
    p->graph = g;
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(g, nodes.data(), &nn);
    for (auto nd : nodes) {
      cudaGraphNodeType t;
      cudaGraphNodeGetType(nd, &t);
      p->kernels += t == cudaGraphNodeTypeKernel;
    }
  } else {
    const long long before = fhe::kernel_launches();
    (void)before;
    p->kernels = -1;
  }
  *out = p;
  return FHE_OK;
}

extern "C" int fhe_batch_launch(fhe_plan *p, fhe_stream stream) {
  if (!p) return fhe_fail(FHE_EINVAL, "fhe_batch_launch: null plan");
  fhe_ctx *c = p->ctx;
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (p->exec) {
    c->order_stream(s);
    cudaError_t e = cudaGraphLaunch(p->exec, s);
    if (e != cudaSuccess) return fhe_fail(FHE_ECUDA, "fhe_batch_launch: %s", cudaGetErrorString(e));
    return FHE_OK;
  }
  const long long before = fhe::kernel_launches();
  int rc = enqueue_items(c, p->items, s);
  p->kernels = (int)(fhe::kernel_launches() - before);
  return rc;
}

extern "C" int fhe_plan_destroy(fhe_plan *p) {
  if (!p) return fhe_fail(FHE_EINVAL, "fhe_plan_destroy: null");
  cudaSetDevice(p->ctx->device);
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  delete p;
  return FHE_OK;
}

extern "C" int fhe_plan_kernel_count(const fhe_plan *p) { return p ? p->kernels : -1; }
