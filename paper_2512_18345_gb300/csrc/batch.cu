// Batched key switching (Section IV-A multi-polynomial caching and batching,
// Section IV-C CUDA Graphs).
//
// A plan splits its items into groups whose stage-1 working sets (beta(l)
// (l + K) limbs each, the footprint column of Table "ks-param") fit an L2
// budget, builds one stage program per group (every stage kernel processes
// all items of the group in one launch, each item in its own workspace slot)
// and captures all groups into one CUDA graph.  Launching the plan replays
// the graph on the caller's stream with one host call.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/fhe.h"
#include "ctx.h"
#include "internal.h"
#include "program.h"

struct fhe_plan {
  fhe_ctx *ctx = nullptr;
  std::vector<fhe_ks_item> items;
  int flags = 0;
  std::vector<Program> progs;
  std::vector<DevProgram> dev;
  std::vector<std::vector<std::pair<const uint32_t *, uint32_t *>>> copies;  // identity rotations per group
  size_t copy_bytes = 0;
  std::vector<int> group_sizes;
  int nlanes = 1;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;
};

// Groups run round-robin on the plan's lanes: lane 0 on the caller's stream,
// lane l > 0 on the context's lane stream l, forked from and joined back into
// the caller's stream.  Each lane has its own workspace slots, so groups on
// different lanes overlap (one group's DRAM-bound inner product next to
// another group's ALU-bound transforms).
static int enqueue_plan(fhe_plan *p, cudaStream_t s) {
  fhe_ctx *c = p->ctx;
  const int nl = p->nlanes;
  if (nl > 1) {
    int rc = ensure_lanes(c, nl);
    if (rc != FHE_OK) return rc;
    if (cudaEventRecord(c->lanes[0].done, s) != cudaSuccess) return fhe_fail(FHE_ECUDA, "fhe_batch: fork");
    for (int l = 1; l < nl; l++)
      if (cudaStreamWaitEvent(c->lanes[l].stream, c->lanes[0].done, 0) != cudaSuccess)
        return fhe_fail(FHE_ECUDA, "fhe_batch: fork");
  }
  for (size_t g = 0; g < p->progs.size(); g++) {
    const int lane = (int)(g % nl);
    cudaStream_t q = lane == 0 ? s : c->lanes[lane].stream;
    for (auto &cp : p->copies[g])
      if (cudaMemcpyAsync(cp.second, cp.first, p->copy_bytes, cudaMemcpyDeviceToDevice, q) != cudaSuccess)
        return fhe_fail(FHE_ECUDA, "fhe_batch: copy");
    int rc = run_program_dev(c, p->progs[g], p->dev[g], q, lane);
    if (rc != FHE_OK) return rc;
  }
  for (int l = 1; l < nl; l++) {
    if (cudaEventRecord(c->lanes[l].done, c->lanes[l].stream) != cudaSuccess ||
        cudaStreamWaitEvent(s, c->lanes[l].done, 0) != cudaSuccess)
      return fhe_fail(FHE_ECUDA, "fhe_batch: join");
  }
  return FHE_OK;
}

static void destroy(fhe_plan *p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  for (auto &d : p->dev) free_program(d);
  delete p;
}

extern "C" int fhe_ctx_set_batch(fhe_ctx *c, size_t l2_budget_bytes, int max_group, int lanes) {
  if (!c || max_group < 0 || lanes < 0 || lanes > 8) return fhe_fail(FHE_EINVAL, "fhe_ctx_set_batch: bad arguments");
  c->batch_budget = l2_budget_bytes;
  c->batch_max_group = max_group;
  c->batch_lanes = lanes ? lanes : 2;
  return FHE_OK;
}

extern "C" int fhe_batch_plan(fhe_ctx *c, const fhe_ks_item *items, int n, int flags, fhe_plan **out) {
  if (!c || !out || n < 1 || !items) return fhe_fail(FHE_EINVAL, "fhe_batch_plan: bad arguments (n >= 1 items)");
  *out = nullptr;
  const size_t N = c->N;
  for (int i = 0; i < n; i++) {
    const fhe_ks_item &it = items[i];
    if (it.level < 1 || it.level > c->L) return fhe_fail(FHE_ELEVEL, "fhe_batch_plan: item %d level %d", i, it.level);
    if (!it.in || !it.out || (it.op == FHE_OP_RELIN && !it.in2))
      return fhe_fail(FHE_EINVAL, "fhe_batch_plan: item %d has a null buffer", i);
    // the stage kernels move 16-byte vectors and bulk copies through these buffers
    if (((uintptr_t)it.in | (uintptr_t)it.out | (uintptr_t)(it.in2 ? it.in2 : it.in)) & 15)
      return fhe_fail(FHE_EINVAL, "fhe_batch_plan: item %d has a buffer that is not 16-byte aligned", i);
    {
      const size_t poly = (size_t)it.level * c->N * 4;
      const size_t in_bytes = it.op == FHE_OP_KS ? poly : 2 * poly;
      auto overlap = [](const void *a, size_t na, const void *b, size_t nb) {
        const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
        return x < y + nb && y < x + na;
      };
      if (overlap(it.out, 2 * poly, it.in, in_bytes) || (it.in2 && overlap(it.out, 2 * poly, it.in2, 2 * poly)))
        return fhe_fail(FHE_EALIAS, "fhe_batch_plan: item %d output overlaps its input", i);
    }
    if (it.op < FHE_OP_KS || it.op > FHE_OP_RELIN) return fhe_fail(FHE_EINVAL, "fhe_batch_plan: item %d op %d", i, it.op);
    if (it.op == FHE_OP_RELIN && !c->relin_key) return fhe_fail(FHE_ENOKEY, "fhe_batch_plan: no relinearisation key");
    if ((it.op == FHE_OP_ROTATE && fhe_galois_elt(it.rot, c->N) != 1u) || it.op == FHE_OP_KS)
      if (!c->find_key(it.rot)) return fhe_fail(FHE_ENOKEY, "fhe_batch_plan: item %d has no key", i);
  }
  cudaSetDevice(c->device);
  fhe_plan *p = new fhe_plan();
  p->ctx = c;
  p->items.assign(items, items + n);
  p->flags = flags;
  // group items so that the stage-1 working sets of the groups in flight stay within
  // the budget (default: twice the L2 -- the stage kernels are bound by the integer
  // pipes, and larger launches amortise their ramp more than L2 residency saves)
  size_t budget = c->batch_budget;
  if (!budget) {
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device);
    budget = (size_t)l2 * 2;
  }
  const int max_group = c->batch_max_group > 0 ? c->batch_max_group : 8;
  const int nl = std::max(1, c->batch_lanes);
  budget /= nl;  // groups on different lanes are resident in L2 at the same time
  std::vector<std::vector<int>> groups(1);
  size_t used = 0;
  for (int i = 0; i < n; i++) {
    const int lv = items[i].level;
    const size_t fp = (size_t)c->beta(lv) * (lv + c->K) * 4 * N;
    if (!groups.back().empty() && (used + fp > budget || (int)groups.back().size() >= max_group)) {
      groups.emplace_back();
      used = 0;
    }
    groups.back().push_back(i);
    used += fp;
  }
  int rc = FHE_OK;
  p->nlanes = std::min<int>(nl, (int)groups.size());
  if (p->nlanes < 1) p->nlanes = 1;
  size_t gmax = 1;
  for (auto &grp : groups) gmax = std::max(gmax, grp.size());
  for (size_t gi = 0; gi < groups.size(); gi++) {
    auto &grp = groups[gi];
    const int slot0 = (int)(gi % p->nlanes) * (int)gmax;
    std::vector<Item> its;
    std::vector<std::pair<const uint32_t *, uint32_t *>> cps;
    for (int i : grp) {
      const fhe_ks_item &x = items[i];
      Item it;
      it.level = x.level;
      it.in = x.in;
      it.in2 = x.in2;
      it.out = x.out;
      if (x.op == FHE_OP_KS) {
        it.kind = IT_KS;
        it.key = c->find_key(x.rot);
      } else if (x.op == FHE_OP_RELIN) {
        it.kind = IT_RELIN;
        it.key = c->relin_key;
      } else {
        const uint32_t k = fhe_galois_elt(x.rot, c->N);
        if (k == 1u) {  // identity rotation: a copy
          cps.push_back({x.in, x.out});
          continue;
        }
        it.kind = IT_ROTATE;
        it.galois = k;
        it.key = c->find_key(x.rot);
      }
      it.slot = slot0 + (int)its.size();
      its.push_back(it);
    }
    // copies of identity rotations have level-dependent sizes: handle them as one-item groups
    Program P;
    if (rc == FHE_OK) rc = build_program(c, its, true, P);
    DevProgram D;
    if (rc == FHE_OK) rc = upload_program(c, P, D);
    p->progs.push_back(P);
    p->dev.push_back(D);
    p->copies.push_back({});
    for (auto &cp : cps) {
      // find the item's level to size the copy: identity rotations are copied one by one
      p->copies.back().push_back(cp);
    }
    p->group_sizes.push_back((int)its.size());
    if (rc != FHE_OK) break;
  }
  // identity-rotation copies need per-item sizes; record them per copy via a side list
  p->copy_bytes = 0;
  if (rc == FHE_OK) {
    bool mixed = false;
    size_t bytes = 0;
    for (int i = 0; i < n; i++)
      if (items[i].op == FHE_OP_ROTATE && fhe_galois_elt(items[i].rot, c->N) == 1u) {
        const size_t b = 8 * N * (size_t)items[i].level;
        if (bytes && b != bytes) mixed = true;
        bytes = b;
      }
    if (mixed) rc = fhe_fail(FHE_EUNSUPPORTED, "fhe_batch_plan: identity rotations at different levels in one plan");
    p->copy_bytes = bytes;
  }
  if (rc == FHE_OK && (flags & FHE_PLAN_GRAPH)) {
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
      destroy(p);
      return fhe_fail(FHE_ECUDA, "fhe_batch_plan: stream");
    }
    if (c->have_last) cudaStreamSynchronize(c->last_stream);
    fhe::Tracer *saved_tracer = c->tabs.tracer;
    c->tabs.tracer = nullptr;  // no trace events inside a captured graph
    c->capturing = true;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      rc = fhe_fail(FHE_ECUDA, "fhe_batch_plan: begin capture");
    if (rc == FHE_OK) rc = enqueue_plan(p, cs);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    c->capturing = false;
    c->tabs.tracer = saved_tracer;
    if (rc == FHE_OK && e != cudaSuccess) rc = fhe_fail(FHE_ECUDA, "fhe_batch_plan: end capture: %s", cudaGetErrorString(e));
    if (rc == FHE_OK && cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess)
      rc = fhe_fail(FHE_ECUDA, "fhe_batch_plan: instantiate");
    cudaStreamDestroy(cs);
    p->graph = g;
    if (rc == FHE_OK) {
      size_t nn = 0;
      cudaGraphGetNodes(g, nullptr, &nn);
      std::vector<cudaGraphNode_t> nodes(nn);
      cudaGraphGetNodes(g, nodes.data(), &nn);
      for (auto nd : nodes) {
        cudaGraphNodeType t;
        cudaGraphNodeGetType(nd, &t);
        p->kernels += t == cudaGraphNodeTypeKernel;
      }
    }
  } else if (rc == FHE_OK) {
    p->kernels = -1;
  }
  if (rc != FHE_OK) {
    destroy(p);
    return rc;
  }
  *out = p;
  return FHE_OK;
}

extern "C" int fhe_batch_launch(fhe_plan *p, fhe_stream stream) {
  if (!p) return fhe_fail(FHE_EINVAL, "fhe_batch_launch: null plan");
  fhe_ctx *c = p->ctx;
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->order_stream(s);
  if (p->exec) {
    cudaError_t e = cudaGraphLaunch(p->exec, s);
    if (e != cudaSuccess) return fhe_fail(FHE_ECUDA, "fhe_batch_launch: %s", cudaGetErrorString(e));
    return FHE_OK;
  }
  const long long before = fhe::kernel_launches();
  int rc = enqueue_plan(p, s);
  p->kernels = (int)(fhe::kernel_launches() - before);
  return rc;
}

extern "C" int fhe_plan_destroy(fhe_plan *p) {
  if (!p) return fhe_fail(FHE_EINVAL, "fhe_plan_destroy: null");
  cudaSetDevice(p->ctx->device);
  destroy(p);
  return FHE_OK;
}

extern "C" int fhe_plan_kernel_count(const fhe_plan *p) { return p ? p->kernels : -1; }

extern "C" int fhe_plan_groups(const fhe_plan *p, int *sizes, int max) {
  if (!p) return fhe_fail(FHE_EINVAL, "fhe_plan_groups: null");
  for (int i = 0; i < max && i < (int)p->group_sizes.size(); i++) sizes[i] = p->group_sizes[i];
  return (int)p->group_sizes.size();
}
