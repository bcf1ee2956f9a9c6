// Baby-step / giant-step plaintext matrix-vector product (the linear-transform
// shape of bootstrapping that relies on hoisted key switching, Section V-C:
// hoisting shares one ModUp across the rotations of one ciphertext):
//   out = sum_{g < G} rot_{B g}( sum_{b < B} diag[g B + b] (.) rot_b(ct) ).
// The B baby rotations are hoisted (one ModUp of c1, then per rotation the
// automorphism on the extended digits, inner product and ModDown); the
// diagonal multiply-accumulate reads every baby rotation once and every
// diagonal once (the diagonals stream from HBM: G B l limbs); the G - 1 giant
// rotations are ordinary rotations, run as one batched stage program per four.
#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/fhe.h"
#include "ctx.h"
#include "elementwise.cuh"
#include "internal.h"
#include "program.h"

using namespace fhe;

namespace fhe {

constexpr int kMaxBaby = 32, kMaxGiant = 16;
struct DiagArgs {
  const uint32_t *babies[kMaxBaby];  // [2][level][N] each
  const uint32_t *diags;             // [giant * nb][level][N]
  uint32_t *out;                     // [giant][2][level][N]
  int nb, giant, level;
};

// out_g[c][i][n] = sum_b diag[g nb + b][i][n] babies[b][c][i][n] mod q_i; one thread per
// coefficient of one limb, each baby value read once, accumulators reduced every three
// products (a reduced value plus three 62-bit products stays below 2^64).
__global__ void __launch_bounds__(256) k_diagmac(const __grid_constant__ DiagArgs a, const PrimeC *pc, int logn) {
  const size_t N = (size_t)1 << logn;
  const int per_limb = (int)(N / 256);
  const int i = blockIdx.x / per_limb;
  const size_t n = (size_t)(blockIdx.x % per_limb) * 256 + threadIdx.x;
  const PrimeC P = pc[i];
  const size_t poly = (size_t)a.level * N;
  uint64_t acc[2][kMaxGiant];
#pragma unroll
  for (int g = 0; g < kMaxGiant; g++) acc[0][g] = acc[1][g] = 0;
  for (int b = 0; b < a.nb; b++) {
    const uint32_t x0 = __ldg(a.babies[b] + (size_t)i * N + n);
    const uint32_t x1 = __ldg(a.babies[b] + poly + (size_t)i * N + n);
#pragma unroll
    for (int g = 0; g < kMaxGiant; g++) {
      if (g < a.giant) {
        const uint32_t d = __ldg(a.diags + ((size_t)(g * a.nb + b) * a.level + i) * N + n);
        acc[0][g] += (uint64_t)d * x0;
        acc[1][g] += (uint64_t)d * x1;
      }
    }
    if (b % 3 == 2) {
#pragma unroll
      for (int g = 0; g < kMaxGiant; g++)
        if (g < a.giant) {
          acc[0][g] = reduce_u64(acc[0][g], P);
          acc[1][g] = reduce_u64(acc[1][g], P);
        }
    }
  }
#pragma unroll
  for (int g = 0; g < kMaxGiant; g++)
    if (g < a.giant)
      for (int c = 0; c < 2; c++) a.out[((size_t)g * 2 + c) * poly + (size_t)i * N + n] = reduce_u64(acc[c][g], P);
}

}  // namespace fhe

static int ensure_lt_scratch(fhe_ctx *c, size_t words) {
  if (c->lt_words >= words) return FHE_OK;
  if (c->lt_scratch) cudaFree(c->lt_scratch);
  c->lt_scratch = nullptr;
  c->lt_words = 0;
  if (cudaMalloc(&c->lt_scratch, words * sizeof(uint32_t)) != cudaSuccess)
    return fhe_fail(FHE_ENOMEM, "fhe_linear_transform: %zu bytes of scratch", words * 4);
  c->lt_words = words;
  return FHE_OK;
}

extern "C" int fhe_linear_transform(fhe_ctx *c, const uint32_t *ct, int level, const uint32_t *diags, int baby,
                                    int giant, uint32_t *out, fhe_stream stream) {
  if (!c) return fhe_fail(FHE_EINVAL, "fhe_linear_transform: null ctx");
  if (level < 1 || level > c->L) return fhe_fail(FHE_ELEVEL, "fhe_linear_transform: level %d", level);
  if (!ct || !diags || !out || (((uintptr_t)ct | (uintptr_t)diags | (uintptr_t)out) & 15))
    return fhe_fail(FHE_EINVAL, "fhe_linear_transform: null or misaligned buffer");
  if (baby < 1 || baby > kMaxBaby || giant < 1 || giant > kMaxGiant)
    return fhe_fail(FHE_EINVAL, "fhe_linear_transform: baby %d (1..%d), giant %d (1..%d)", baby, kMaxBaby, giant,
                    kMaxGiant);
  for (int r = 1; r < baby; r++)
    if (fhe_galois_elt(r, c->N) != 1u && !c->find_key(r))
      return fhe_fail(FHE_ENOKEY, "fhe_linear_transform: no rotation key for baby step %d", r);
  for (int g = 1; g < giant; g++)
    if (fhe_galois_elt(baby * g, c->N) != 1u && !c->find_key(baby * g))
      return fhe_fail(FHE_ENOKEY, "fhe_linear_transform: no rotation key for giant step %d", baby * g);
  const size_t N = c->N, poly = (size_t)level * N, ct_words = 2 * poly;
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  // scratch: baby rotations, inner sums, giant rotations
  int rc = ensure_lt_scratch(c, ct_words * ((size_t)baby + 2 * giant));
  if (rc != FHE_OK) return rc;
  uint32_t *babies = c->lt_scratch, *inner = babies + baby * ct_words, *grot = inner + giant * ct_words;
  std::vector<int32_t> rots(baby);
  std::vector<uint32_t *> bo(baby);
  for (int b = 0; b < baby; b++) {
    rots[b] = b;
    bo[b] = babies + b * ct_words;
  }
  rc = fhe_rotate_hoisted(c, ct, level, rots.data(), baby, bo.data(), stream);
  if (rc != FHE_OK) return rc;
  DiagArgs da;
  memset(&da, 0, sizeof da);
  for (int b = 0; b < baby; b++) da.babies[b] = bo[b];
  da.diags = diags;
  da.out = inner;
  da.nb = baby;
  da.giant = giant;
  da.level = level;
  {
    TraceScope ts(c->tabs, "diag_mac", s);
    k_diagmac<<<(unsigned)(level * (N / 256)), 256, 0, s>>>(da, c->d_pc, c->logn);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return fhe_fail(FHE_ECUDA, "fhe_linear_transform: diagonal kernel");
  }
  // giant rotations, as many per batched stage program as the launch arguments hold
  std::vector<Item> its;
  for (int g = 1; g < giant; g++) {
    const uint32_t k = fhe_galois_elt(baby * g, c->N);
    if (k == 1u) {
      if (cudaMemcpyAsync(grot + g * ct_words, inner + g * ct_words, 4 * ct_words, cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess)
        return fhe_fail(FHE_ECUDA, "fhe_linear_transform: copy");
      continue;
    }
    Item it;
    it.kind = IT_ROTATE;
    it.level = level;
    it.galois = k;
    it.in = inner + g * ct_words;
    it.out = grot + g * ct_words;
    it.key = c->find_key(baby * g);
    its.push_back(it);
  }
  rc = run_items_chunked(c, its, 0, s);
  if (rc != FHE_OK) return rc;
  // out = inner_0 + sum_g rot_{B g}(inner_g)
  if (cudaMemcpyAsync(out, inner, 4 * ct_words, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return fhe_fail(FHE_ECUDA, "fhe_linear_transform: copy");
  for (int g = 1; g < giant; g++) {
    rc = fhe_add(c, out, grot + g * ct_words, 2, level, out, stream);
    if (rc != FHE_OK) return rc;
  }
  return FHE_OK;
}
