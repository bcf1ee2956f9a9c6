// Baby-step / giant-step plaintext matrix-vector product (the linear-transform
// shape of bootstrapping that relies on hoisted key switching, Section V-C:
// hoisting shares one ModUp across the rotations of one ciphertext):
//   out = sum_{g < G} rot_{B g}( sum_{b < B} diag[g B + b] (.) rot_b(ct) ).
// The B baby rotations are hoisted (one ModUp of c1, then per rotation the
// automorphism on the extended digits, inner product and ModDown); the
// diagonal multiply-accumulate reads every baby rotation once and every
// diagonal once (the diagonals stream from HBM: G B l limbs); the G - 1 giant
// rotations are ordinary rotations, run as batched stage programs; one pass sums
// the giant-step outputs.
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
// coefficient of one limb and group of kGsub giant steps (blockIdx.y; the groups re-read
// the baby values from L2); two baby steps' loads are issued before their
// multiply-accumulates, and the accumulators are reduced after every second baby step
// (a reduced value plus two 62-bit products stays below 2^64).
constexpr int kGsub = 4;
__global__ void __launch_bounds__(256) k_diagmac(const __grid_constant__ DiagArgs a, const PrimeC *pc, int logn) {
  const size_t N = (size_t)1 << logn;
  const int per_limb = (int)(N / 256);
  const int i = blockIdx.x / per_limb;
  const size_t n = (size_t)(blockIdx.x % per_limb) * 256 + threadIdx.x;
  const int g0 = blockIdx.y * kGsub, ng = min(kGsub, a.giant - g0);
  const PrimeC P = pc[i];
  const size_t poly = (size_t)a.level * N;
  const uint32_t *dbase = a.diags + (size_t)i * N + n;
  uint64_t acc[2][kGsub];
#pragma unroll
  for (int g = 0; g < kGsub; g++) acc[0][g] = acc[1][g] = 0;
  for (int b = 0; b < a.nb; b += 2) {
    const bool two = b + 1 < a.nb;
    uint32_t x[2][2], d[2][kGsub];
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int bb = two ? b + h : b;
      x[h][0] = __ldg(a.babies[bb] + (size_t)i * N + n);
      x[h][1] = __ldg(a.babies[bb] + poly + (size_t)i * N + n);
#pragma unroll
      for (int g = 0; g < kGsub; g++)
        d[h][g] = g < ng ? __ldg(dbase + (size_t)((g0 + g) * a.nb + bb) * poly) : 0u;
    }
#pragma unroll
    for (int h = 0; h < 2; h++) {
      if (h == 1 && !two) break;
#pragma unroll
      for (int g = 0; g < kGsub; g++) {
        acc[0][g] += (uint64_t)d[h][g] * x[h][0];
        acc[1][g] += (uint64_t)d[h][g] * x[h][1];
      }
    }
#pragma unroll
    for (int g = 0; g < kGsub; g++) {
      acc[0][g] = reduce_u64(acc[0][g], P);
      acc[1][g] = reduce_u64(acc[1][g], P);
    }
  }
#pragma unroll
  for (int g = 0; g < kGsub; g++)
    if (g < ng)
#pragma unroll
      for (int c = 0; c < 2; c++) a.out[((size_t)(g0 + g) * 2 + c) * poly + (size_t)i * N + n] = (uint32_t)acc[c][g];
}

// out[c][i][n] = sum_{g < count} in_g[c][i][n] mod q_i (the giant-step outputs), one thread
// per coefficient of one limb of both polynomials
struct SumArgs {
  const uint32_t *in[kMaxGiant];  // [2][level][N] each
  uint32_t *out;
  int count, level;
};
__global__ void __launch_bounds__(256) k_sum(const __grid_constant__ SumArgs a, const PrimeC *pc, int logn) {
  const size_t N = (size_t)1 << logn;
  const int per_limb = (int)(N / 256);
  const int i = blockIdx.x / per_limb;
  const size_t n = (size_t)(blockIdx.x % per_limb) * 256 + threadIdx.x;
  const uint32_t q = pc[i].q;
  const size_t poly = (size_t)a.level * N;
#pragma unroll
  for (int c = 0; c < 2; c++) {
    uint32_t acc = 0;
    for (int g = 0; g < a.count; g++) acc = add_mod(acc, __ldg(a.in[g] + c * poly + (size_t)i * N + n), q);
    a.out[c * poly + (size_t)i * N + n] = acc;
  }
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
    const dim3 grid((unsigned)(level * (N / 256)), (unsigned)((giant + kGsub - 1) / kGsub));
    k_diagmac<<<grid, 256, 0, s>>>(da, c->d_pc, c->logn);
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
  // out = inner_0 + sum_g rot_{B g}(inner_g), in one pass
  SumArgs sa;
  memset(&sa, 0, sizeof sa);
  sa.in[0] = inner;
  for (int g = 1; g < giant; g++) sa.in[g] = grot + g * ct_words;
  sa.count = giant;
  sa.out = out;
  sa.level = level;
  {
    TraceScope ts(c->tabs, "lt_sum", s);
    k_sum<<<(unsigned)(level * (N / 256)), 256, 0, s>>>(sa, c->d_pc, c->logn);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return fhe_fail(FHE_ECUDA, "fhe_linear_transform: sum kernel");
  }
  return FHE_OK;
}
