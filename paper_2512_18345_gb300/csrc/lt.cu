// Baby-step / giant-step plaintext matrix-vector product (the linear-transform
// shape of bootstrapping that relies on hoisted key switching, Section V-C:
// hoisting shares one ModUp across the rotations of one ciphertext):
//   out = sum_{g < G} rot_{B g}( sum_{b < B} diag[g B + b] (.) rot_b(ct) ).
// The B baby rotations are hoisted (one ModUp of c1, then per rotation the
// automorphism on the extended digits, inner product and ModDown); the
// diagonal multiply-accumulate reads every baby rotation once and every
// diagonal once (the diagonals stream from HBM: G B l limbs); the G - 1 giant
// rotations are ordinary rotations, run as batched stage programs; one pass sums
// the giant-step outputs (fhe_linear_transform).
//
// fhe_linear_transform_dh is the double-hoisted form used by the CoeffToSlot /
// SlotToCoeff levels of bootstrapping: sparse diagonals chosen per (giant, baby)
// pair, baby rotations kept in the extended basis Q_l u P, ModDown hoisted over
// both step kinds (see the function's comment below).
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
  const uint32_t *babies[kMaxBaby];  // [2][nlimb][N] each
  const uint32_t *diags;             // [n_diag][nlimb][N]
  uint32_t *out;                     // [giant][2][nlimb][N]
  int nb, giant, nlimb, level, L;    // limb i < level is modulo q_i, limb i >= level modulo p_{i - level}
  int16_t didx[kMaxGiant * kMaxBaby];  // [giant][nb]: index into diags, -1 where the pair has no diagonal
  uint32_t gmask[kMaxGiant];           // bit b of gmask[g]: didx[g][b] >= 0
};

static void diag_masks(DiagArgs &da) {
  for (int g = 0; g < da.giant; g++) {
    da.gmask[g] = 0;
    for (int b = 0; b < da.nb; b++)
      if (da.didx[g * da.nb + b] >= 0) da.gmask[g] |= 1u << b;
  }
}

__device__ __forceinline__ int limb_prime(int i, int level, int L) { return i < level ? i : L + (i - level); }

// out_g[c][i][n] = sum_b diag[didx[g][b]][i][n] babies[b][c][i][n] mod (prime of limb i).
// A unit is kDiagChunk coefficients of one limb for one group of kGsub giant steps; the
// units of one chunk's groups are adjacent, so the later groups find the baby rows in L2.
// Per (unit, baby step with a diagonal in the group) a producer warp (one lane) copies the
// baby rotation's two rows and the group's diagonal rows (4 KB each) into a ring of
// shared-memory stages with cp.async.bulk, completing on the stage's full mbarrier, and
// refills a stage as soon as every consumer thread has released it.  The consumers wait on
// the full barriers themselves (bounded; a warp gives up as a whole) and multiply-accumulate
// from shared memory into 64-bit accumulators; every third step folds them (fold34), and the
// end of a unit reduces them.
constexpr int kGsub = 4;
constexpr int kDiagChunk = 1024, kDiagThreads = 256, kDiagEpt = kDiagChunk / kDiagThreads;
constexpr int kDiagRows = 2 + kGsub;  // stage rows: baby c0, baby c1, one diagonal per giant step
static_assert(kDiagEpt == 4, "diagonal kernel: one 16-byte access per row and thread");

// One CTA per SM (the 8 consumer warps' accumulators take about 100 registers a thread, and
// a second CTA would put 5 warps on one SM sub-partition: more than its register file holds),
// so the ring takes most of the shared memory: 8 stages, 192 KB in flight per SM.
constexpr int kDiagStageBytes = kDiagRows * kDiagChunk * 4 + 16;  // rows, two mbarriers
constexpr int kDiagStages = 8;
static_assert(kDiagStages * kDiagStageBytes <= 227 * 1024, "diagonal kernel: stages exceed shared memory");

// a = hi 2^34 + lo  ->  hi r34 + lo with r34 = 2^34 mod q: the same residue, below 2^61 + 2^34
// for any 64-bit a (hi < 2^30, r34 < 2^31), so three more products below 2^62 still fit
__device__ __forceinline__ uint64_t fold34(uint64_t a, uint32_t r34) {
  return (uint64_t)(uint32_t)(a >> 34) * r34 + (a & ((1ull << 34) - 1));
}

__global__ void __launch_bounds__(kDiagThreads + 32, 1) k_diag_bulk(const __grid_constant__ DiagArgs a, const PrimeC *pc,
                                                                   int logn, unsigned int *status) {
  constexpr int stages = kDiagStages;
  extern __shared__ __align__(128) uint8_t smem[];
  constexpr int E = kDiagEpt;
  const int tid = threadIdx.x;
  const size_t N = (size_t)1 << logn, poly = (size_t)a.nlimb * N;
  const int chunks = (int)(N / kDiagChunk), groups = (a.giant + kGsub - 1) / kGsub;
  const int total = a.nlimb * chunks * groups;
  const size_t stage_words = (size_t)kDiagRows * kDiagChunk;
  uint32_t *buf = reinterpret_cast<uint32_t *>(smem);
  // per stage: `bar` completes when the stage's copies have landed, `ebar` when every
  // consumer thread is done with it
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + (size_t)stages * stage_words * 4);
  uint64_t *ebar = bar + stages;
  if (tid == 0)
    for (int st = 0; st < stages; st++) {
      mbar_init(&bar[st], 1);
      mbar_init(&ebar[st], kDiagThreads);
    }
  __syncthreads();
  // the baby steps of group grp that meet a diagonal
  auto group_mask = [&](int grp, uint32_t (&gm)[kGsub]) {
    uint32_t any = 0;
#pragma unroll
    for (int g = 0; g < kGsub; g++) {
      gm[g] = grp * kGsub + g < a.giant ? a.gmask[grp * kGsub + g] : 0u;
      any |= gm[g];
    }
    return any;
  };

  if (tid >= kDiagThreads) {  // the producer
    if (tid != kDiagThreads) return;
    const uint64_t once = l2_evict_first_policy();  // diagonals are read exactly once
    int k = 0;
    for (int u = blockIdx.x; u < total; u += gridDim.x) {
      const int grp = u % groups, ch = (u / groups) % chunks, i = u / (groups * chunks);
      const size_t off = (size_t)i * N + (size_t)ch * kDiagChunk;
      uint32_t gm[kGsub];
      for (uint32_t live = group_mask(grp, gm); live; live &= live - 1) {
        const int b = __ffs(live) - 1;
        const int st = k % stages;
        // the consumers released this stage's previous step (bounded: if they gave up, so do we)
        if (k >= stages && !mbar_wait_bounded(&ebar[st], (uint32_t)(k / stages - 1) & 1u)) return;
        fence_proxy_async_smem();
        uint32_t rows = 2;
#pragma unroll
        for (int g = 0; g < kGsub; g++) rows += (gm[g] >> b) & 1u;
        mbar_arrive_expect_tx(&bar[st], rows * kDiagChunk * 4u);
        uint32_t *dst = buf + (size_t)st * stage_words;
        bulk_g2s(dst, a.babies[b] + off, kDiagChunk * 4u, &bar[st]);
        bulk_g2s(dst + kDiagChunk, a.babies[b] + poly + off, kDiagChunk * 4u, &bar[st]);
#pragma unroll
        for (int g = 0; g < kGsub; g++)
          if ((gm[g] >> b) & 1u)
            bulk_g2s_hint(dst + (size_t)(2 + g) * kDiagChunk,
                          a.diags + (size_t)a.didx[(grp * kGsub + g) * a.nb + b] * poly + off, kDiagChunk * 4u,
                          &bar[st], once);
        k++;
      }
    }
    return;
  }

  const int lane = tid & 31;
  bool ok = true;
  int k = 0;
  for (int u = blockIdx.x; ok && u < total; u += gridDim.x) {
    const int grp = u % groups, ch = (u / groups) % chunks, i = u / (groups * chunks);
    const PrimeC P = pc[limb_prime(i, a.level, a.L)];
    const uint32_t r34 = P.r34;
    uint32_t gm[kGsub];
    uint32_t live = group_mask(grp, gm);
    uint64_t acc[2][kGsub][E];
#pragma unroll
    for (int g = 0; g < kGsub; g++)
#pragma unroll
      for (int e = 0; e < E; e++) acc[0][g][e] = acc[1][g][e] = 0;
    int since = 0;  // products added to each accumulator since the last fold
    for (; live; live &= live - 1) {
      const int b = __ffs(live) - 1;
      const int st = k % stages;
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bar[st], (uint32_t)(k / stages) & 1u))) {
        ok = false;
        break;
      }
      const uint32_t *src = buf + (size_t)st * stage_words + tid * E;
      uint32_t x0[E], x1[E];
      ld_words<E>(src, x0);
      ld_words<E>(src + kDiagChunk, x1);
#pragma unroll
      for (int g = 0; g < kGsub; g++)
        if ((gm[g] >> b) & 1u) {
          uint32_t d[E];
          ld_words<E>(src + (size_t)(2 + g) * kDiagChunk, d);
#pragma unroll
          for (int e = 0; e < E; e++) {
            acc[0][g][e] += (uint64_t)d[e] * x0[e];
            acc[1][g][e] += (uint64_t)d[e] * x1[e];
          }
        }
      mbar_arrive(&ebar[st]);  // this thread is done with stage st
      k++;
      if (++since == 3) {
        since = 0;
#pragma unroll
        for (int g = 0; g < kGsub; g++)
#pragma unroll
          for (int e = 0; e < E; e++) {
            acc[0][g][e] = fold34(acc[0][g][e], r34);
            acc[1][g][e] = fold34(acc[1][g][e], r34);
          }
      }
    }
    if (!ok) break;
    const int g0 = grp * kGsub, ng = min(kGsub, a.giant - g0);
    const size_t o = (size_t)i * N + (size_t)ch * kDiagChunk + tid * E;
#pragma unroll
    for (int g = 0; g < kGsub; g++)
      if (g < ng)
#pragma unroll
        for (int c = 0; c < 2; c++) {
          uint32_t r[E];
#pragma unroll
          for (int e = 0; e < E; e++) r[e] = reduce_u64(acc[c][g][e], P);
          st_words<E>(a.out + ((size_t)(g0 + g) * 2 + c) * poly + o, r);
        }
  }
  if (!ok && lane == 0) {
    // an expired wait: report it, then wait (bounded) for this CTA's copies that may still be
    // in flight (the producer runs at most `stages` steps beyond the last one released)
    atomicOr(status, 4u);
    int issued = 0;  // steps of this CTA
    for (int u = blockIdx.x; u < total; u += gridDim.x) {
      uint32_t gm[kGsub];
      issued += __popc(group_mask(u % groups, gm));
    }
    for (int k2 = k; k2 < min(issued, k + stages); k2++)
      mbar_wait_bounded(&bar[k2 % stages], (uint32_t)(k2 / stages) & 1u);
  }
}


static cudaError_t launch_diag(fhe_ctx *c, const DiagArgs &da, cudaStream_t s) {
  static PerDeviceOnce configured;
  const cudaError_t e = configured.run([] {
    return cudaFuncSetAttribute(k_diag_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kDiagStages * kDiagStageBytes);
  });
  if (e != cudaSuccess) return e;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const int units = da.nlimb * (int)(c->N / kDiagChunk) * ((da.giant + kGsub - 1) / kGsub);
  const unsigned grid = (unsigned)std::min(units, std::max(1, sms));  // persistent: one CTA per SM
  k_diag_bulk<<<grid, kDiagThreads + 32, kDiagStages * kDiagStageBytes, s>>>(da, c->d_pc, c->logn, c->tabs.status);
  note_launch();
  return cudaGetLastError();
}

// The identity baby step of a double-hoisted transform, in the extended basis:
// out[c] = P ct[c] on the q-limbs and 0 on the special limbs (ModDown of it returns ct exactly).
__global__ void __launch_bounds__(256) k_lift(const uint32_t *ct, uint32_t *out, const uint2 *pmod, const PrimeC *pc,
                                              int level, int nlimb, int logn) {
  const size_t N = (size_t)1 << logn;
  const int per_limb = (int)(N / 1024);  // four consecutive coefficients per thread
  const int i = blockIdx.x / per_limb;
  const size_t n = (size_t)(blockIdx.x % per_limb) * 1024 + threadIdx.x * 4;
#pragma unroll
  for (int c = 0; c < 2; c++) {
    uint4 v = make_uint4(0, 0, 0, 0);
    if (i < level) {
      const uint4 x = __ldg(reinterpret_cast<const uint4 *>(ct + ((size_t)c * level + i) * N + n));
      const uint2 pm = pmod[i];
      const uint32_t q = pc[i].q;
      v = make_uint4(shoup(x.x, pm, q), shoup(x.y, pm, q), shoup(x.z, pm, q), shoup(x.w, pm, q));
    }
    *reinterpret_cast<uint4 *>(out + ((size_t)c * nlimb + i) * N + n) = v;
  }
}

// Giant-step accumulation of a double-hoisted transform, in the extended basis:
//   out_0 = sum_g sigma_g(inner_g,0) + v_g,0,   out_1 = sum_g v_g,1,
// where v_g is the extended-basis key switch of sigma_g applied to ModDown(inner_g,1); a giant
// step without rotation (v_g null) adds inner_g itself.
struct GsumArgs {
  const uint32_t *inner[kMaxGiant];  // [2][nlimb][N]
  const uint32_t *v[kMaxGiant];      // [2][nlimb][N] or null
  uint32_t galois[kMaxGiant];
  uint32_t *out;                     // [2][nlimb][N]
  int count, nlimb, level, L;
};
// Four consecutive coefficients per thread: 16-byte loads and stores for every operand but
// the sigma-gathered c0 halves.
constexpr int kGsumEpt = 4;
__global__ void __launch_bounds__(256) k_gsum(const __grid_constant__ GsumArgs a, const PrimeC *pc, int logn) {
  const size_t N = (size_t)1 << logn;
  const int per_limb = (int)(N / (256 * kGsumEpt));
  const int i = blockIdx.x / per_limb;
  const uint32_t n = (uint32_t)((blockIdx.x % per_limb) * (256 * kGsumEpt) + threadIdx.x * kGsumEpt);
  const uint32_t q = pc[limb_prime(i, a.level, a.L)].q;
  const size_t poly = (size_t)a.nlimb * N, off = (size_t)i * N;
  uint32_t a0[kGsumEpt] = {}, a1[kGsumEpt] = {};
  auto add4 = [&](uint32_t (&acc)[kGsumEpt], const uint32_t *p) {
    const uint4 w = __ldg(reinterpret_cast<const uint4 *>(p));
    acc[0] = add_mod(acc[0], w.x, q);
    acc[1] = add_mod(acc[1], w.y, q);
    acc[2] = add_mod(acc[2], w.z, q);
    acc[3] = add_mod(acc[3], w.w, q);
  };
  for (int g = 0; g < a.count; g++) {
    const uint32_t *in = a.inner[g] + off;
    if (!a.v[g]) {
      add4(a0, in + n);
      add4(a1, in + poly + n);
    } else {
#pragma unroll
      for (int e = 0; e < kGsumEpt; e++) a0[e] = add_mod(a0[e], __ldg(in + galois_src(n + e, a.galois[g], logn)), q);
      add4(a0, a.v[g] + off + n);
      add4(a1, a.v[g] + poly + off + n);
    }
  }
  *reinterpret_cast<uint4 *>(a.out + off + n) = make_uint4(a0[0], a0[1], a0[2], a0[3]);
  *reinterpret_cast<uint4 *>(a.out + poly + off + n) = make_uint4(a1[0], a1[1], a1[2], a1[3]);
}

// out[c][i][n] = sum_{g < count} in_g[c][i][n] mod q_i (the giant-step outputs), one thread
// per four consecutive coefficients of one limb of both polynomials (16-byte accesses)
struct SumArgs {
  const uint32_t *in[kMaxGiant];  // [2][level][N] each
  uint32_t *out;
  int count, level;
};
__global__ void __launch_bounds__(256) k_sum(const __grid_constant__ SumArgs a, const PrimeC *pc, int logn) {
  const size_t N = (size_t)1 << logn;
  const int per_limb = (int)(N / 1024);
  const int i = blockIdx.x / per_limb;
  const size_t n = (size_t)(blockIdx.x % per_limb) * 1024 + threadIdx.x * 4;
  const uint32_t q = pc[i].q;
  const size_t poly = (size_t)a.level * N;
#pragma unroll
  for (int c = 0; c < 2; c++) {
    uint32_t acc[4] = {0, 0, 0, 0};
    for (int g = 0; g < a.count; g++) {
      const uint4 w = __ldg(reinterpret_cast<const uint4 *>(a.in[g] + c * poly + (size_t)i * N + n));
      acc[0] = add_mod(acc[0], w.x, q);
      acc[1] = add_mod(acc[1], w.y, q);
      acc[2] = add_mod(acc[2], w.z, q);
      acc[3] = add_mod(acc[3], w.w, q);
    }
    *reinterpret_cast<uint4 *>(a.out + c * poly + (size_t)i * N + n) = make_uint4(acc[0], acc[1], acc[2], acc[3]);
  }
}

}  // namespace fhe

static bool ranges_overlap(const void *a, size_t abytes, const void *b, size_t bbytes) {
  const char *x = (const char *)a, *y = (const char *)b;
  return x < y + bbytes && y < x + abytes;
}

#define LT_CHECK(x)                \
  do {                             \
    const int rc_ = (x);           \
    if (rc_ != FHE_OK) return rc_; \
  } while (0)

static int ensure_lt_scratch(fhe_ctx *c, size_t words) {
  if (c->lt_words >= words) return FHE_OK;
  const size_t old_bytes = c->lt_words * sizeof(uint32_t);
  // the old buffer is released first, so only the difference counts against the limit
  const int rc = c->reserve(words * sizeof(uint32_t) - old_bytes, "linear-transform scratch");
  if (rc != FHE_OK) return rc;
  if (c->lt_scratch) cudaFree(c->lt_scratch);
  c->grown_bytes -= old_bytes;
  c->lt_scratch = nullptr;
  c->lt_words = 0;
  if (cudaMalloc(&c->lt_scratch, words * sizeof(uint32_t)) != cudaSuccess)
    return fhe_fail(FHE_ENOMEM, "fhe_linear_transform: %zu bytes of scratch", words * 4);
  c->lt_words = words;
  c->grown_bytes += words * sizeof(uint32_t);
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
  da.nlimb = level;
  da.level = level;
  da.L = c->L;
  for (int k = 0; k < baby * giant; k++) da.didx[k] = (int16_t)k;
  diag_masks(da);
  {
    TraceScope ts(c->tabs, "diag_mac", s);
    if (launch_diag(c, da, s) != cudaSuccess) return fhe_fail(FHE_ECUDA, "fhe_linear_transform: diagonal kernel");
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
    k_sum<<<(unsigned)(level * (N / 1024)), 256, 0, s>>>(sa, c->d_pc, c->logn);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return fhe_fail(FHE_ECUDA, "fhe_linear_transform: sum kernel");
  }
  return FHE_OK;
}

// Double-hoisted baby-step / giant-step transform (the hoisting of the
// linear-transform literature the paper cites in Section V-C, with ModDown
// hoisted as well as ModUp):
//   out = sum_g rot_{giant[g]}( sum_b pt[idx[g][b]] (.) rot_{baby[b]}(ct) ).
// (1) one ModUp of c1; every baby rotation's inner product stays in the
//     extended basis Q_l u P, with P sigma_b(c0) folded onto its q-limbs
//     (IT_IPX); a baby step without rotation is P ct (k_lift);
// (2) the inner sums are formed in the extended basis (k_diag_bulk over l + K limbs);
// (3) per rotating giant step, the c1 half of its inner sum goes down to Q_l
//     (IT_MDX), is decomposed again (IT_MODUP) and key-switched with sigma_g on the
//     extended digits (IT_IPX), again without ModDown;
// (4) k_gsum adds sigma_g of the c0 halves and the key-switch outputs;
// (5) one ModDown of both halves (IT_MDX).
extern "C" int fhe_linear_transform_dh(fhe_ctx *c, const uint32_t *ct, int level, const int32_t *baby, int n_baby,
                                       const int32_t *giant, int n_giant, const uint32_t *diags, int n_diag,
                                       const int32_t *idx, uint32_t *out, fhe_stream stream) {
  const char *fn = "fhe_linear_transform_dh";
  if (!c) return fhe_fail(FHE_EINVAL, "%s: null ctx", fn);
  if (level < 1 || level > c->L) return fhe_fail(FHE_ELEVEL, "%s: level %d", fn, level);
  if (!ct || !diags || !out || (((uintptr_t)ct | (uintptr_t)diags | (uintptr_t)out) & 15))
    return fhe_fail(FHE_EINVAL, "%s: null or misaligned buffer", fn);
  if (!baby || !giant || !idx) return fhe_fail(FHE_EINVAL, "%s: null rotation or index list", fn);
  if (n_baby < 1 || n_baby > kMaxBaby || n_giant < 1 || n_giant > kMaxGiant)
    return fhe_fail(FHE_EINVAL, "%s: n_baby %d (1..%d), n_giant %d (1..%d)", fn, n_baby, kMaxBaby, n_giant, kMaxGiant);
  if (n_diag < 1 || n_diag > 32767) return fhe_fail(FHE_EINVAL, "%s: n_diag %d outside [1, 32767]", fn, n_diag);
  for (int k = 0; k < n_baby * n_giant; k++)
    if (idx[k] < -1 || idx[k] >= n_diag) return fhe_fail(FHE_EINVAL, "%s: idx[%d] = %d outside [-1, %d)", fn, k, idx[k], n_diag);
  const int K = c->K, n_ext = level + K;
  const size_t N = c->N, poly = (size_t)level * N, xpoly = (size_t)n_ext * N;
  if (ranges_overlap(out, 2 * poly * 4, ct, 2 * poly * 4) || ranges_overlap(out, 2 * poly * 4, diags, (size_t)n_diag * xpoly * 4))
    return fhe_fail(FHE_EALIAS, "%s: output overlaps an input", fn);
  std::vector<uint32_t> gb(n_baby), gg(n_giant);
  std::vector<const uint32_t *> kb(n_baby, nullptr), kg(n_giant, nullptr);
  for (int b = 0; b < n_baby; b++) {
    gb[b] = fhe_galois_elt(baby[b], c->N);
    if (gb[b] != 1u && !(kb[b] = c->find_key(baby[b])))
      return fhe_fail(FHE_ENOKEY, "%s: no rotation key for baby step %d", fn, baby[b]);
  }
  for (int g = 0; g < n_giant; g++) {
    gg[g] = fhe_galois_elt(giant[g], c->N);
    if (gg[g] != 1u && !(kg[g] = c->find_key(giant[g])))
      return fhe_fail(FHE_ENOKEY, "%s: no rotation key for giant step %d", fn, giant[g]);
  }
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->order_stream(s);
  // scratch: baby rotations, inner sums and giant key switches (extended basis, two
  // halves each), the giant steps' c1 halves in Q_l, the accumulator
  const size_t xct = 2 * xpoly;
  int rc = ensure_lt_scratch(c, xct * ((size_t)n_baby + 2 * n_giant + 1) + poly * n_giant);
  if (rc != FHE_OK) return rc;
  uint32_t *bab = c->lt_scratch, *inner = bab + n_baby * xct, *v = inner + n_giant * xct, *acc = v + n_giant * xct,
           *c1d = acc + xct;
  const unsigned grid_x = (unsigned)(n_ext * (N / 256));

  // (1) baby steps
  std::vector<Item> its;
  for (int b = 0; b < n_baby; b++) {
    if (gb[b] == 1u) {
      TraceScope ts(c->tabs, "lt_lift", s);
      k_lift<<<grid_x / 4, 256, 0, s>>>(ct, bab + b * xct, c->d_pmod, c->d_pc, level, n_ext, c->logn);
      note_launch();
      if (cudaGetLastError() != cudaSuccess) return fhe_fail(FHE_ECUDA, "%s: lift kernel", fn);
      continue;
    }
    Item it;
    it.kind = IT_IPX;
    it.level = level;
    it.galois = gb[b];
    it.in = ct + poly;
    it.in2 = ct;
    it.out = bab + b * xct;
    it.key = kb[b];
    it.ext_slot = 0;
    its.push_back(it);
  }
  if (!its.empty()) {
    Item up;
    up.kind = IT_MODUP;
    up.level = level;
    up.in = ct + poly;
    up.slot = 0;
    its.insert(its.begin(), up);
    LT_CHECK(run_items_chunked(c, its, 1, s));
  }

  // (2) inner sums in the extended basis
  DiagArgs da;
  memset(&da, 0, sizeof da);
  for (int b = 0; b < n_baby; b++) da.babies[b] = bab + b * xct;
  da.diags = diags;
  da.out = inner;
  da.nb = n_baby;
  da.giant = n_giant;
  da.nlimb = n_ext;
  da.level = level;
  da.L = c->L;
  for (int k = 0; k < n_baby * n_giant; k++) da.didx[k] = (int16_t)idx[k];
  diag_masks(da);
  {
    TraceScope ts(c->tabs, "diag_mac", s);
    if (launch_diag(c, da, s) != cudaSuccess) return fhe_fail(FHE_ECUDA, "%s: diagonal kernel", fn);
  }

  // (3) rotating giant steps: ModDown of the c1 halves, then ModUp + extended-basis key switch
  std::vector<int> rg;
  for (int g = 0; g < n_giant; g++)
    if (gg[g] != 1u) rg.push_back(g);
  if (!rg.empty()) {
    std::vector<Item> md;
    for (int g : rg) {
      Item it;
      it.kind = IT_MDX;
      it.level = level;
      it.npoly = 1;
      it.in = inner + g * xct + xpoly;
      it.out = c1d + g * poly;
      md.push_back(it);
    }
    LT_CHECK(run_items_chunked(c, md, 1, s));
    std::vector<Item> ks;
    const int ng = (int)rg.size();
    for (int j = 0; j < ng; j++) {
      Item up;
      up.kind = IT_MODUP;
      up.level = level;
      up.in = c1d + rg[j] * poly;
      up.slot = 1 + j;
      ks.push_back(up);
    }
    for (int j = 0; j < ng; j++) {
      const int g = rg[j];
      Item it;
      it.kind = IT_IPX;
      it.level = level;
      it.galois = gg[g];
      it.in = c1d + g * poly;
      it.out = v + g * xct;
      it.key = kg[g];
      it.ext_slot = 1 + j;
      ks.push_back(it);
    }
    LT_CHECK(run_items_chunked(c, ks, 1 + ng, s));
  }

  // (4) giant-step accumulation, (5) one ModDown of both halves
  GsumArgs ga;
  memset(&ga, 0, sizeof ga);
  for (int g = 0; g < n_giant; g++) {
    ga.inner[g] = inner + g * xct;
    ga.v[g] = gg[g] != 1u ? v + g * xct : nullptr;
    ga.galois[g] = gg[g];
  }
  ga.out = acc;
  ga.count = n_giant;
  ga.nlimb = n_ext;
  ga.level = level;
  ga.L = c->L;
  {
    TraceScope ts(c->tabs, "lt_gsum", s);
    k_gsum<<<grid_x / kGsumEpt, 256, 0, s>>>(ga, c->d_pc, c->logn);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return fhe_fail(FHE_ECUDA, "%s: giant-step sum kernel", fn);
  }
  Item fin;
  fin.kind = IT_MDX;
  fin.level = level;
  fin.npoly = 2;
  fin.in = acc;
  fin.out = out;
  std::vector<Item> f{fin};
  LT_CHECK(run_items_chunked(c, f, 1, s));
  return FHE_OK;
}
