// Key-switching pipelines (Section IV, Fig. "keysw") and the CKKS operations
// built on them, enqueued on the caller's stream.
//
// Stage 1 (ModUp): INTT of the input limbs, scaled by N^-1 (D_j/q_t)^-1 (the
//   BConv pre-factor folded into the INTT output), base conversion of every
//   digit to the limbs it lacks, NTT of the converted limbs.  For a rotation
//   the automorphism is a gather in the INTT's loads.
// Stage 2 (inner product): one element-wise kernel per run of extended limbs,
//   both key halves at once.
// Stage 3 (ModDown): INTT of the special limbs (scaled by the BConv
//   pre-factor), BConv to the ciphertext limbs, NTT whose last pass also
//   subtracts from the inner product, multiplies by P^-1 and adds the
//   pass-through polynomial (Section III-D: NTT(a1) + a2 + ... is fusable).
// The plain pipeline runs every step (gather, scaling, combine) as its own
// kernel on one stream.
#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/fhe.h"
#include "ctx.h"
#include "elementwise.cuh"
#include "internal.h"
#include "program.h"

using namespace fhe;

#define LAUNCH_OR_FAIL(call)                                                                          \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) return fhe_fail(FHE_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));      \
  } while (0)

static Seg mkseg(const uint32_t *src, uint32_t *dst, int n, int prime) {
  Seg s;
  memset(&s, 0, sizeof s);
  s.src = src;
  s.dst = dst;
  s.n = n;
  s.prime = prime;
  s.src_stride = 1;
  s.src_prime = -1;

  return s;
}

struct SegBuilder {
  SegList l;
  SegBuilder() {
    memset(&l, 0, sizeof l);
    l.ks[0].galois_own = l.ks[0].galois_ext = l.ks[0].galois_add = 1;
  }
  void add(const Seg &s) {
    if (s.n <= 0) return;
    l.seg[l.nseg++] = s;
    l.total += s.n;
  }
};

static bool overlaps(const void *a, size_t abytes, const void *b, size_t bbytes) {
  const char *x = (const char *)a, *y = (const char *)b;
  return x < y + bbytes && y < x + abytes;
}

// run a program of at most kMaxInlineItems items with by-value launch arguments
static int run_items(fhe_ctx *c, const std::vector<Item> &items, cudaStream_t s) {
  Program P;
  int rc = build_program(c, items, c->fused != 0, P);
  if (rc != FHE_OK) return rc;
  return run_program_inline(c, P, s);
}

// Run items in consecutive chunks, each as large as by-value launch arguments allow.
// Items other than IT_MODUP get workspace slots first_slot, first_slot + 1, ... within
// their chunk; an IT_MODUP item keeps its own slot.
int run_items_chunked(fhe_ctx *c, const std::vector<Item> &items, int first_slot, cudaStream_t s) {
  size_t i = 0;
  while (i < items.size()) {
    std::vector<Item> chunk;
    Program best;
    int nslot = 0;
    size_t j = i;
    while (j < items.size()) {
      Item it = items[j];
      // an extended-basis inner product needs no workspace of its own: it reads its ModUp's slot
      const bool own_slot = it.kind != IT_MODUP && it.kind != IT_IPX;
      if (it.kind == IT_IPX) it.slot = it.ext_slot;
      if (own_slot) it.slot = first_slot + nslot;
      chunk.push_back(it);
      Program Q;
      const int rc = build_program(c, chunk, c->fused != 0, Q);
      if (rc != FHE_OK) return rc;
      if (!program_fits_inline(Q)) {
        chunk.pop_back();
        break;
      }
      best = std::move(Q);
      if (own_slot) nslot++;
      j++;
    }
    if (chunk.empty()) return fhe_fail(FHE_EINVAL, "internal: one item does not fit the launch arguments");
    const int rc = run_program_inline(c, best, s);
    if (rc != FHE_OK) return rc;
    i = j;
  }
  return FHE_OK;
}

static int check_level(const fhe_ctx *c, int level, const char *fn) {
  if (level < 1 || level > c->L) return fhe_fail(FHE_ELEVEL, "%s: level %d outside [1, %d]", fn, level, c->L);
  return FHE_OK;
}

static int check_ptr(const void *p, const char *fn, const char *name) {
  if (!p) return fhe_fail(FHE_EINVAL, "%s: %s is null", fn, name);
  if ((uintptr_t)p & 15) return fhe_fail(FHE_EINVAL, "%s: %s is not 16-byte aligned", fn, name);
  return FHE_OK;
}

#define CHECK(x)            \
  do {                      \
    int rc_ = (x);          \
    if (rc_ != FHE_OK) return rc_; \
  } while (0)

extern "C" int fhe_keyswitch(fhe_ctx *c, const uint32_t *d, int level, int32_t key_id, uint32_t *out,
                             fhe_stream stream) {
  if (!c) return fhe_fail(FHE_EINVAL, "fhe_keyswitch: null ctx");
  CHECK(check_level(c, level, "fhe_keyswitch"));
  CHECK(check_ptr(d, "fhe_keyswitch", "d"));
  CHECK(check_ptr(out, "fhe_keyswitch", "out"));
  const size_t poly = (size_t)level * c->N * 4;
  if (overlaps(d, poly, out, 2 * poly)) return fhe_fail(FHE_EALIAS, "fhe_keyswitch: out overlaps d");
  const uint32_t *key = c->find_key(key_id);
  if (!key) return fhe_fail(FHE_ENOKEY, "fhe_keyswitch: no key for id %d", key_id);
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->order_stream(s);
  Item it;
  it.kind = IT_KS;
  it.level = level;
  it.in = d;
  it.out = out;
  it.key = key;
  return run_items(c, {it}, s);
}

extern "C" int fhe_rotate(fhe_ctx *c, const uint32_t *ct, int level, int32_t rot, uint32_t *out, fhe_stream stream) {
  if (!c) return fhe_fail(FHE_EINVAL, "fhe_rotate: null ctx");
  CHECK(check_level(c, level, "fhe_rotate"));
  CHECK(check_ptr(ct, "fhe_rotate", "ct"));
  CHECK(check_ptr(out, "fhe_rotate", "out"));
  const size_t poly = (size_t)level * c->N;
  if (overlaps(ct, 8 * poly, out, 8 * poly)) return fhe_fail(FHE_EALIAS, "fhe_rotate: out overlaps ct");
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t k = fhe_galois_elt(rot, c->N);
  if (k == 1u) {
    c->order_stream(s);
    if (cudaMemcpyAsync(out, ct, 8 * poly, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return fhe_fail(FHE_ECUDA, "fhe_rotate: copy");
    return FHE_OK;
  }
  const uint32_t *key = c->find_key(rot);
  if (!key) return fhe_fail(FHE_ENOKEY, "fhe_rotate: no rotation key for %d", rot);
  c->order_stream(s);
  Item it;
  it.kind = IT_ROTATE;
  it.level = level;
  it.galois = k;
  it.in = ct;
  it.out = out;
  it.key = key;
  return run_items(c, {it}, s);
}

extern "C" int fhe_hmult(fhe_ctx *c, const uint32_t *a, const uint32_t *b, int level, uint32_t *out,
                         fhe_stream stream) {
  if (!c) return fhe_fail(FHE_EINVAL, "fhe_hmult: null ctx");
  CHECK(check_level(c, level, "fhe_hmult"));
  CHECK(check_ptr(a, "fhe_hmult", "a"));
  CHECK(check_ptr(b, "fhe_hmult", "b"));
  CHECK(check_ptr(out, "fhe_hmult", "out"));
  if (!c->relin_key) return fhe_fail(FHE_ENOKEY, "fhe_hmult: relinearisation key not set");
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->order_stream(s);
  Item it;
  it.kind = IT_RELIN;
  it.level = level;
  it.in = a;
  it.in2 = b;
  it.out = out;
  it.key = c->relin_key;
  return run_items(c, {it}, s);
}

extern "C" int fhe_rescale(fhe_ctx *c, const uint32_t *ct, int level, uint32_t *out, fhe_stream stream) {
  if (!c) return fhe_fail(FHE_EINVAL, "fhe_rescale: null ctx");
  if (level < 2 || level > c->L) return fhe_fail(FHE_ELEVEL, "fhe_rescale: level %d outside [2, %d]", level, c->L);
  CHECK(check_ptr(ct, "fhe_rescale", "ct"));
  CHECK(check_ptr(out, "fhe_rescale", "out"));
  const size_t N = c->N, poly = (size_t)level * N;
  if (overlaps(ct, 8 * poly, out, 8 * (poly - N))) return fhe_fail(FHE_EALIAS, "fhe_rescale: out overlaps ct");
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->order_stream(s);
  uint32_t *V = c->slots[0].V;
  SegBuilder f1, f2, g1, g2;
  for (int cc = 0; cc < 2; cc++) {
    f1.add(mkseg(ct + cc * poly + (size_t)(level - 1) * N, V + cc * N, 1, level - 1));
    f2.add(mkseg(V + cc * N, V + cc * N, 1, level - 1));
  }
  LAUNCH_OR_FAIL(launch_ntt(c->tabs, false, PRO_PLAIN, EPI_SCALE, f1.l, f2.l, s));
  for (int cc = 0; cc < 2; cc++) {
    uint32_t *o = out + (size_t)cc * (level - 1) * N;
    Seg a = mkseg(V + cc * N, o, level - 1, 0);
    a.src_stride = 0;
    a.src_prime = level - 1;
    g1.add(a);
    Seg b = mkseg(o, o, level - 1, 0);
    b.src2 = ct + cc * poly;
    b.scale = c->d_rs_qinv + (size_t)(level - 1) * c->L;
    g2.add(b);
  }
  LAUNCH_OR_FAIL(launch_ntt(c->tabs, true, PRO_REDUCE, EPI_RESCALE, g1.l, g2.l, s));
  return FHE_OK;
}

extern "C" int fhe_rotate_hoisted(fhe_ctx *c, const uint32_t *ct, int level, const int32_t *rots, int n,
                                  uint32_t *const *outs, fhe_stream stream) {
  if (!c) return fhe_fail(FHE_EINVAL, "fhe_rotate_hoisted: null ctx");
  CHECK(check_level(c, level, "fhe_rotate_hoisted"));
  CHECK(check_ptr(ct, "fhe_rotate_hoisted", "ct"));
  if (n < 0 || (n > 0 && (!rots || !outs))) return fhe_fail(FHE_EINVAL, "fhe_rotate_hoisted: bad rotation list");
  const size_t poly = (size_t)level * c->N;
  std::vector<const uint32_t *> keys(n);
  for (int r = 0; r < n; r++) {
    CHECK(check_ptr(outs[r], "fhe_rotate_hoisted", "outs[i]"));
    if (overlaps(ct, 8 * poly, outs[r], 8 * poly)) return fhe_fail(FHE_EALIAS, "fhe_rotate_hoisted: output overlaps ct");
    if (fhe_galois_elt(rots[r], c->N) != 1u) {
      keys[r] = c->find_key(rots[r]);
      if (!keys[r]) return fhe_fail(FHE_ENOKEY, "fhe_rotate_hoisted: no rotation key for %d", rots[r]);
    }
  }
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->order_stream(s);
  // one shared ModUp of c1 (slot 0), then the rotations' ModDowns batched
  // as many at a time as fit the by-value launch arguments, each with its own slot
  std::vector<Item> todo;
  for (int r = 0; r < n; r++) {
    const uint32_t k = fhe_galois_elt(rots[r], c->N);
    if (k == 1u) {
      if (cudaMemcpyAsync(outs[r], ct, 8 * poly, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return fhe_fail(FHE_ECUDA, "fhe_rotate_hoisted: copy");
      continue;
    }
    Item it;
    it.kind = IT_MODDOWN;
    it.level = level;
    it.galois = k;
    it.in = ct;
    it.out = outs[r];
    it.key = keys[r];
    it.ext_slot = 0;
    todo.push_back(it);
  }
  if (todo.empty()) return FHE_OK;
  Item up;
  up.kind = IT_MODUP;
  up.level = level;
  up.in = ct + poly;
  up.slot = 0;
  todo.insert(todo.begin(), up);
  CHECK(run_items_chunked(c, todo, 1, s));
  return FHE_OK;
}

static int elementwise2(fhe_ctx *c, int op, const uint32_t *a, const uint32_t *b, int npoly, int level,
                        uint32_t *out, bool b_per_poly, cudaStream_t s) {
  const size_t poly = (size_t)level * c->N;
  SegBuilder sb;
  for (int p = 0; p < npoly; p++) {
    Seg x = mkseg(a + p * poly, out + p * poly, level, 0);
    x.src2 = b_per_poly ? b + p * poly : b;
    sb.add(x);
  }
  c->order_stream(s);
  LAUNCH_OR_FAIL(launch_ew(c->tabs, op, sb.l, s));
  return FHE_OK;
}

extern "C" int fhe_pmult(fhe_ctx *c, const uint32_t *ct, const uint32_t *pt, int level, uint32_t *out,
                         fhe_stream stream) {
  if (!c) return fhe_fail(FHE_EINVAL, "fhe_pmult: null ctx");
  CHECK(check_level(c, level, "fhe_pmult"));
  CHECK(check_ptr(ct, "fhe_pmult", "ct"));
  CHECK(check_ptr(pt, "fhe_pmult", "pt"));
  CHECK(check_ptr(out, "fhe_pmult", "out"));
  cudaSetDevice(c->device);
  return elementwise2(c, EW_MUL, ct, pt, 2, level, out, false, (cudaStream_t)stream);
}

extern "C" int fhe_add(fhe_ctx *c, const uint32_t *a, const uint32_t *b, int npoly, int level, uint32_t *out,
                       fhe_stream stream) {
  if (!c) return fhe_fail(FHE_EINVAL, "fhe_add: null ctx");
  CHECK(check_level(c, level, "fhe_add"));
  if (npoly < 1 || npoly > 8) return fhe_fail(FHE_EINVAL, "fhe_add: npoly %d outside [1, 8]", npoly);
  CHECK(check_ptr(a, "fhe_add", "a"));
  CHECK(check_ptr(b, "fhe_add", "b"));
  CHECK(check_ptr(out, "fhe_add", "out"));
  cudaSetDevice(c->device);
  return elementwise2(c, EW_ADD, a, b, npoly, level, out, true, (cudaStream_t)stream);
}

// ------------------------------------------------------------------ stage-level entry points

static int transform(fhe_ctx *c, uint32_t *a, const int *idx, int n, bool fwd, fhe_stream stream, const char *fn) {
  if (!c) return fhe_fail(FHE_EINVAL, "%s: null ctx", fn);
  CHECK(check_ptr(a, fn, "a"));
  if (n < 0 || (n > 0 && !idx)) return fhe_fail(FHE_EINVAL, "%s: bad prime list", fn);
  for (int i = 0; i < n; i++)
    if (idx[i] < 0 || idx[i] >= c->L + c->K) return fhe_fail(FHE_EINVAL, "%s: prime index %d out of range", fn, idx[i]);
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->order_stream(s);
  const size_t N = c->N;
  int i = 0;
  while (i < n) {
    SegBuilder sb;
    while (i < n && sb.l.nseg < kMaxSeg) {
      int j = i + 1;
      while (j < n && idx[j] == idx[j - 1] + 1) j++;
      sb.add(mkseg(a + (size_t)i * N, a + (size_t)i * N, j - i, idx[i]));
      i = j;
    }
    LAUNCH_OR_FAIL(launch_ntt(c->tabs, fwd, PRO_PLAIN, fwd ? EPI_PLAIN : EPI_SCALE, sb.l, sb.l, s));
  }
  return FHE_OK;
}

extern "C" int fhe_ntt(fhe_ctx *c, uint32_t *a, const int *idx, int n, fhe_stream stream) {
  return transform(c, a, idx, n, true, stream, "fhe_ntt");
}
extern "C" int fhe_intt(fhe_ctx *c, uint32_t *a, const int *idx, int n, fhe_stream stream) {
  return transform(c, a, idx, n, false, stream, "fhe_intt");
}

extern "C" int fhe_modup(fhe_ctx *c, const uint32_t *d, int level, uint32_t *ext, fhe_stream stream) {
  if (!c) return fhe_fail(FHE_EINVAL, "fhe_modup: null ctx");
  CHECK(check_level(c, level, "fhe_modup"));
  CHECK(check_ptr(d, "fhe_modup", "d"));
  CHECK(check_ptr(ext, "fhe_modup", "ext"));
  const size_t N = c->N;
  const int n_ext = level + c->K, beta = c->beta(level);
  if (overlaps(d, 4 * N * level, ext, 4 * N * (size_t)beta * n_ext)) return fhe_fail(FHE_EALIAS, "fhe_modup: ext overlaps d");
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->order_stream(s);
  Item it;
  it.kind = IT_MODUP;
  it.level = level;
  it.in = d;
  it.slot = 0;
  CHECK(run_items(c, {it}, s));
  if (cudaMemcpyAsync(ext, c->slots[0].EXT, 4 * N * (size_t)beta * n_ext, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return fhe_fail(FHE_ECUDA, "fhe_modup: copy");
  for (int j = 0; j < beta; j++) {
    const int lo = j * c->alpha, hi = std::min((j + 1) * c->alpha, level);
    if (cudaMemcpyAsync(ext + ((size_t)j * n_ext + lo) * N, d + (size_t)lo * N, 4 * N * (hi - lo),
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return fhe_fail(FHE_ECUDA, "fhe_modup: copy");
  }
  return FHE_OK;
}

extern "C" int fhe_moddown(fhe_ctx *c, const uint32_t *u, int level, uint32_t *out, fhe_stream stream) {
  if (!c) return fhe_fail(FHE_EINVAL, "fhe_moddown: null ctx");
  CHECK(check_level(c, level, "fhe_moddown"));
  CHECK(check_ptr(u, "fhe_moddown", "u"));
  CHECK(check_ptr(out, "fhe_moddown", "out"));
  const size_t N = c->N;
  const int K = c->K, L = c->L;
  if (overlaps(u, 4 * N * (level + K), out, 4 * N * level)) return fhe_fail(FHE_EALIAS, "fhe_moddown: out overlaps u");
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->order_stream(s);
  uint32_t *UC = c->slots[0].UC, *R = c->slots[0].R;
  SegBuilder first, second, nr, cb;
  first.add(mkseg(u + (size_t)level * N, UC, K, L));
  Seg b = mkseg(UC, UC, K, L);
  b.scale = c->d_md_scale;
  second.add(b);
  LAUNCH_OR_FAIL(launch_ntt(c->tabs, false, PRO_PLAIN, EPI_SCALE, first.l, second.l, s));
  BconvArgs ba;
  memset(&ba, 0, sizeof ba);
  BconvGroup &g = ba.g[ba.ngroups++];
  g.in = UC;
  g.out = R;
  g.T = c->d_mdT;
  g.omap = c->d_mdmap;
  g.n_in = K;
  g.n_out = level;
  g.Btc = c->d_md_Btc;
  g.npad = tc_npad(level);
  if (c->bconv_mode == FHE_BCONV_TC)
    LAUNCH_OR_FAIL(launch_bconv_tc(c->tabs, ba, K, level, s, c->tabs.tc_k));
  else
    LAUNCH_OR_FAIL(launch_bconv(c->tabs, ba, K, level, s));
  nr.add(mkseg(R, R, level, 0));
  LAUNCH_OR_FAIL(launch_ntt(c->tabs, true, PRO_PLAIN, EPI_PLAIN, nr.l, nr.l, s));
  Seg x = mkseg(u, out, level, 0);
  x.src2 = R;
  cb.add(x);
  cb.l.ks[0].pinv = c->d_pinv;
  cb.l.ks[0].level = level;
  LAUNCH_OR_FAIL(launch_ew(c->tabs, EW_COMBINE, cb.l, s));
  return FHE_OK;
}

// The tables of one fhe_bconv combination (input primes, output primes, kernel): the
// pre-factors (Qstar/q_j)^-1 mod q_j, T[o][j] = (Qstar/q_j) mod p_o, the output map and, for
// the tensor-core kernel, its byte-digit table.  The first call with a combination builds them,
// allocates one device block and copies them with cudaMemcpyAsync on `s` (from pageable host
// memory, so that first call may wait while the runtime stages it); later calls find them in
// the context and allocate, copy and wait for nothing.
// The context also keeps the pre-multiplied input ([16][N] words, allocated once).  Calls on a
// context are ordered on the GPU (order_stream), so one copy of each serves every call.  A
// context keeps at most kMaxBconvPrep combinations; a new one beyond that waits for the
// context's earlier work and releases the cached tables first.
static constexpr size_t kMaxBconvPrep = 64;

static int bconv_prepare(fhe_ctx *c, const int *in_idx, int n_in, const int *out_idx, int n_out, bool tc, int kt,
                         cudaStream_t s, fhe_ctx::BconvPrep *out) {
  const size_t N = c->N;
  if (!c->bconv_y) {
    const size_t bytes = 16 * N * sizeof(uint32_t);
    const int rc = c->reserve(bytes, "fhe_bconv scratch");
    if (rc != FHE_OK) return rc;
    if (cudaMalloc(&c->bconv_y, bytes) != cudaSuccess) return fhe_fail(FHE_ENOMEM, "fhe_bconv: scratch");
    c->grown_bytes += bytes;
  }
  std::vector<int> key;
  key.reserve(n_in + n_out + 3);
  key.push_back(tc ? kt : 0);
  key.push_back(n_in);
  key.insert(key.end(), in_idx, in_idx + n_in);
  key.insert(key.end(), out_idx, out_idx + n_out);
  auto it = c->bconv_prep.find(key);
  c->order_stream(s);
  if (it != c->bconv_prep.end()) {
    *out = it->second;
    return FHE_OK;
  }
  if (c->bconv_prep.size() >= kMaxBconvPrep) {
    // the cached tables may still be read by enqueued work: wait for it before freeing them
    if (cudaStreamSynchronize(s) != cudaSuccess) return fhe_fail(FHE_ECUDA, "fhe_bconv: sync before releasing tables");
    for (auto &kv : c->bconv_prep) cudaFree(kv.second.block);
    c->bconv_prep.clear();
  }
  const std::vector<uint32_t> &pr = c->primes;
  std::vector<uint2> pre(n_in);
  for (int j = 0; j < n_in; j++) {
    const uint32_t q = pr[in_idx[j]];
    uint32_t prod = 1;
    for (int k = 0; k < n_in; k++)
      if (k != j) prod = h_mulmod_pub(prod, pr[in_idx[k]] % q, q);
    const uint32_t w = h_invmod_pub(prod, q);
    pre[j] = make_uint2(w, (uint32_t)(((uint64_t)w << 32) / q));
  }
  std::vector<uint32_t> T((size_t)n_out * n_in);
  std::vector<int2> om(n_out);
  std::vector<uint32_t> pout(n_out);
  for (int o = 0; o < n_out; o++) {
    const uint32_t p = pr[out_idx[o]];
    for (int j = 0; j < n_in; j++) {
      uint32_t prod = 1;
      for (int k = 0; k < n_in; k++)
        if (k != j) prod = h_mulmod_pub(prod, pr[in_idx[k]] % p, p);
      T[(size_t)o * n_in + j] = prod;
    }
    om[o] = make_int2(o, out_idx[o]);
    pout[o] = p;
  }
  const std::vector<uint16_t> Btc = tc ? bconv_tc_table(T, n_in, pout, kt) : std::vector<uint16_t>(8, 0);
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t oT = 0, oM = up(4 * T.size()), oP = oM + up(8 * om.size()), oB = oP + up(8 * pre.size());
  const size_t bytes = oB + up(2 * Btc.size());
  const int rc = c->reserve(bytes, "fhe_bconv tables");
  if (rc != FHE_OK) return rc;
  fhe_ctx::BconvPrep p;
  if (cudaMalloc(&p.block, bytes) != cudaSuccess) return fhe_fail(FHE_ENOMEM, "fhe_bconv: tables");
  c->grown_bytes += bytes;
  char *b = static_cast<char *>(p.block);
  p.T = reinterpret_cast<uint32_t *>(b + oT);
  p.om = reinterpret_cast<int2 *>(b + oM);
  p.pre = reinterpret_cast<uint2 *>(b + oP);
  p.Btc = reinterpret_cast<uint16_t *>(b + oB);
  if (cudaMemcpyAsync(p.T, T.data(), 4 * T.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(p.om, om.data(), 8 * om.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(p.pre, pre.data(), 8 * pre.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(p.Btc, Btc.data(), 2 * Btc.size(), cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaFree(p.block);
    c->grown_bytes -= bytes;
    return fhe_fail(FHE_ECUDA, "fhe_bconv: table copy");
  }
  c->bconv_prep.emplace(std::move(key), p);
  *out = p;
  return FHE_OK;
}

extern "C" int fhe_bconv(fhe_ctx *c, const uint32_t *in, const int *in_idx, int n_in, uint32_t *out,
                         const int *out_idx, int n_out, fhe_stream stream) {
  if (!c) return fhe_fail(FHE_EINVAL, "fhe_bconv: null ctx");
  CHECK(check_ptr(in, "fhe_bconv", "in"));
  CHECK(check_ptr(out, "fhe_bconv", "out"));
  if (n_in < 1 || n_in > 16 || n_out < 1 || n_out > 64 || !in_idx || !out_idx)
    return fhe_fail(FHE_EINVAL, "fhe_bconv: n_in=%d (1..16), n_out=%d (1..64)", n_in, n_out);
  const int NP = c->L + c->K;
  for (int i = 0; i < n_in; i++)
    if (in_idx[i] < 0 || in_idx[i] >= NP) return fhe_fail(FHE_EINVAL, "fhe_bconv: in prime index");
  for (int i = 0; i < n_out; i++)
    if (out_idx[i] < 0 || out_idx[i] >= NP) return fhe_fail(FHE_EINVAL, "fhe_bconv: out prime index");
  const size_t N = c->N;
  if (overlaps(in, 4 * N * n_in, out, 4 * N * n_out)) return fhe_fail(FHE_EALIAS, "fhe_bconv: out overlaps in");
  const bool tc = c->bconv_mode == FHE_BCONV_TC;
  if (tc && n_in > kTcMaxIn12)
    return fhe_fail(FHE_EUNSUPPORTED, "fhe_bconv: tensor-core base conversion takes at most %d inputs", kTcMaxIn12);
  const int kt = tc_k_for(n_in);
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  fhe_ctx::BconvPrep prep;
  const int rc0 = bconv_prepare(c, in_idx, n_in, out_idx, n_out, tc, kt, s, &prep);
  if (rc0 != FHE_OK) return rc0;
  // pre-multiply limb by limb (each limb its own prime: one segment per limb)
  uint32_t *y = c->bconv_y;
  for (int j0 = 0; j0 < n_in; j0 += kMaxSeg) {
    SegBuilder sb;
    for (int j = j0; j < std::min(n_in, j0 + kMaxSeg); j++) {
      Seg x = mkseg(in + (size_t)j * N, y + (size_t)j * N, 1, in_idx[j]);
      x.scale = prep.pre + j;
      sb.add(x);
    }
    if (launch_ew(c->tabs, EW_SCALE, sb.l, s) != cudaSuccess) return fhe_fail(FHE_ECUDA, "fhe_bconv: scale");
  }
  BconvArgs ba;
  memset(&ba, 0, sizeof ba);
  BconvGroup &g = ba.g[ba.ngroups++];
  g.in = y;
  g.out = out;
  g.T = prep.T;
  g.omap = prep.om;
  g.n_in = n_in;
  g.n_out = n_out;
  g.Btc = prep.Btc;
  g.npad = tc_npad(n_out);
  const cudaError_t e = tc ? launch_bconv_tc(c->tabs, ba, n_in, n_out, s, kt) : launch_bconv(c->tabs, ba, n_in, n_out, s);
  if (e != cudaSuccess) return fhe_fail(FHE_ECUDA, "fhe_bconv: %s", cudaGetErrorString(e));
  return FHE_OK;
}
