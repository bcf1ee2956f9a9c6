// Element-wise kernels of the plain (per-kernel) pipeline: automorphism
// gather, scaling, key inner product, ModDown combine, HMult tensor product,
// addition and plaintext multiplication (Section II-B "The rest": element-wise
// parallel operations over L x N).  Four elements per thread; contiguous
// reads and writes are 128-bit.
#pragma once
#include "async.cuh"
#include "common.cuh"
#include "ntt.cuh"

namespace fhe {

constexpr int kEwThreads = 256;

enum : int {
  EW_GATHER = 0,   // dst = src[sigma(j)]               (galois = seg.galois)
  EW_SCALE = 1,    // dst = src * scale[l]
  EW_IP = 2,       // (k_ip) both halves of the key inner product
  EW_COMBINE = 3,  // dst = (src - src2) P^-1  (src = u, src2 = NTT(r))
  EW_ADD = 4,      // dst = src + src2
  EW_MUL = 5,      // dst = src * src2
  EW_COPY = 6,     // dst = src
  EW_TENSOR = 7,   // HMult tensor: src = a, src2 = b ([2][n][N] each), dst = (d0, d1, d2) [3][n][N]
};

template <int OP>
__global__ void __launch_bounds__(kEwThreads) k_ew(const __grid_constant__ SegList sl, const PrimeC *pc, int logn) {
  const size_t N = (size_t)1 << logn;
  const int blocks_per_limb = (int)(N / (4 * kEwThreads));
  const int v = blockIdx.x / blocks_per_limb;
  const uint32_t j0 = (uint32_t)((blockIdx.x % blocks_per_limb) * 4 * kEwThreads + threadIdx.x * 4);
  int within;
  const Seg &sg = seg_at(sl, seg_find(sl, v, within));
  const KsArgs &ks = item_ks(sl, sg);
  const int prime = sg.prime + within;
  const PrimeC P = pc[prime];
  const uint32_t q = P.q;
  const uint32_t *src = sg.src ? sg.src + (size_t)within * sg.src_stride * N : nullptr;
  const uint32_t *src2 = sg.src2 ? sg.src2 + (size_t)within * N : nullptr;
  uint32_t *dst = sg.dst + (size_t)within * N;
  uint32_t o[4];
  if (OP == EW_TENSOR) {  // the segment covers one ciphertext's limbs; n = level is the poly stride
    const size_t poly = (size_t)sg.n * N, off = (size_t)within * N + j0;
    const uint4 A0 = __ldg(reinterpret_cast<const uint4 *>(sg.src + off));
    const uint4 A1 = __ldg(reinterpret_cast<const uint4 *>(sg.src + poly + off));
    const uint4 B0 = __ldg(reinterpret_cast<const uint4 *>(sg.src2 + off));
    const uint4 B1 = __ldg(reinterpret_cast<const uint4 *>(sg.src2 + poly + off));
    const uint32_t a0[4] = {A0.x, A0.y, A0.z, A0.w}, a1[4] = {A1.x, A1.y, A1.z, A1.w};
    const uint32_t b0[4] = {B0.x, B0.y, B0.z, B0.w}, b1[4] = {B1.x, B1.y, B1.z, B1.w};
    uint32_t d0[4], d1[4], d2[4];
#pragma unroll
    for (int x = 0; x < 4; x++) {
      d0[x] = mul_mod(a0[x], b0[x], P);
      d1[x] = reduce_u64((uint64_t)a0[x] * b1[x] + (uint64_t)a1[x] * b0[x], P);  // < 2^63
      d2[x] = mul_mod(a1[x], b1[x], P);
    }
    uint32_t *d = sg.dst + off;
    *reinterpret_cast<uint4 *>(d) = make_uint4(d0[0], d0[1], d0[2], d0[3]);
    *reinterpret_cast<uint4 *>(d + poly) = make_uint4(d1[0], d1[1], d1[2], d1[3]);
    *reinterpret_cast<uint4 *>(d + 2 * poly) = make_uint4(d2[0], d2[1], d2[2], d2[3]);
    return;
  }
  if (OP == EW_GATHER) {
#pragma unroll
    for (int e = 0; e < 4; e++) o[e] = __ldg(src + galois_src(j0 + e, sg.galois, logn));
  } else {
    const uint4 a = __ldg(reinterpret_cast<const uint4 *>(src + j0));
    const uint32_t av[4] = {a.x, a.y, a.z, a.w};
    uint32_t bv[4] = {0, 0, 0, 0};
    if (OP == EW_COMBINE || OP == EW_ADD || OP == EW_MUL) {
      const uint4 b = __ldg(reinterpret_cast<const uint4 *>(src2 + j0));
      bv[0] = b.x; bv[1] = b.y; bv[2] = b.z; bv[3] = b.w;
    }
    uint2 sc = make_uint2(0, 0);
    if (OP == EW_SCALE) sc = sg.scale[within];
    if (OP == EW_COMBINE) sc = ks.pinv[prime];
#pragma unroll
    for (int e = 0; e < 4; e++) {
      if (OP == EW_SCALE) o[e] = shoup(av[e], sc.x, sc.y, q);
      else if (OP == EW_ADD) o[e] = add_mod(av[e], bv[e], q);
      else if (OP == EW_MUL) o[e] = mul_mod(av[e], bv[e], P);
      else if (OP == EW_COPY) o[e] = av[e];
      else  // EW_COMBINE (u carries P times the pass-through term)
        o[e] = shoup(av[e] + q - bv[e], sc.x, sc.y, q);
    }
  }
  *reinterpret_cast<uint4 *>(dst + j0) = make_uint4(o[0], o[1], o[2], o[3]);
}

// Stage 2: the key inner product for a run of extended limbs, both halves at
// once (each ModUp value is read once):
//   u_c[t][n] = sum_{j < beta} E_j[t][n] key[j][c][row(t)][n] mod prime(t),
// E_j[t] = own[t] (read through sigma_{galois_own}) when t is one of digit j's
// q-limbs, else ext[j][t] (read through sigma_{galois_ext}).  seg.dst points
// at u_0[t0]; u_1 sits n_ext limbs further.  beta <= 4, so the four 62-bit
// products of a sum fit one 64-bit accumulator.
template <bool GOWN, bool GEXT>
__global__ void __launch_bounds__(kEwThreads) k_ip(const __grid_constant__ SegList sl, const PrimeC *pc, int logn) {
  const size_t N = (size_t)1 << logn;
  const int blocks_per_limb = (int)(N / (4 * kEwThreads));
  const int v = blockIdx.x / blocks_per_limb;
  const uint32_t j0 = (uint32_t)((blockIdx.x % blocks_per_limb) * 4 * kEwThreads + threadIdx.x * 4);
  int within;
  const Seg &sg = seg_at(sl, seg_find(sl, v, within));
  const KsArgs &ks = item_ks(sl, sg);
  const int t = sg.t0 + within, row = sg.key_row0 + within;
  const PrimeC P = pc[sg.prime + within];
  const size_t kstride = (size_t)2 * (ks.L + ks.K) * N;
  // issue every digit's loads before any arithmetic (memory-level parallelism)
  uint4 ev[4], kv0[4], kv1[4];
#pragma unroll
  for (int jd = 0; jd < 4; jd++) {
    if (jd < ks.beta) {
      const bool own = t < ks.level && t >= jd * ks.alpha && t < (jd + 1) * ks.alpha;
      const uint32_t *p = own ? ks.own + (size_t)t * N : ks.ext + ((size_t)jd * ks.n_ext + t) * N;
      if ((own && GOWN) || (!own && GEXT)) {
        const uint32_t g = own ? ks.galois_own : ks.galois_ext;
        ev[jd] = make_uint4(__ldg(p + galois_src(j0, g, logn)), __ldg(p + galois_src(j0 + 1, g, logn)),
                            __ldg(p + galois_src(j0 + 2, g, logn)), __ldg(p + galois_src(j0 + 3, g, logn)));
      } else {
        ev[jd] = __ldg(reinterpret_cast<const uint4 *>(p + j0));
      }
      const uint32_t *kp = ks.key + jd * kstride + (size_t)row * N + j0;
      kv0[jd] = __ldg(reinterpret_cast<const uint4 *>(kp));
      kv1[jd] = __ldg(reinterpret_cast<const uint4 *>(kp + (size_t)(ks.L + ks.K) * N));
    } else {
      ev[jd] = kv0[jd] = kv1[jd] = make_uint4(0, 0, 0, 0);
    }
  }
  uint64_t a0[4] = {0, 0, 0, 0}, a1[4] = {0, 0, 0, 0};
#pragma unroll
  for (int jd = 0; jd < 4; jd++) {
    const uint32_t e4[4] = {ev[jd].x, ev[jd].y, ev[jd].z, ev[jd].w};
    const uint32_t k0[4] = {kv0[jd].x, kv0[jd].y, kv0[jd].z, kv0[jd].w};
    const uint32_t k1[4] = {kv1[jd].x, kv1[jd].y, kv1[jd].z, kv1[jd].w};
#pragma unroll
    for (int i = 0; i < 4; i++) {
      a0[i] += (uint64_t)e4[i] * k0[i];
      a1[i] += (uint64_t)e4[i] * k1[i];
    }
  }
  uint32_t r0[4], r1[4];
#pragma unroll
  for (int i = 0; i < 4; i++) {
    r0[i] = reduce_u64(a0[i], P);
    r1[i] = reduce_u64(a1[i], P);
  }
  if (ks.addp && t < ks.level) {  // pass-through term: u_c += P * addp_c (c = 0; c = 1 for HMult)
    const uint2 pm = ks.pmod[t];
    const uint32_t *ap = ks.addp + (size_t)t * N;
#pragma unroll
    for (int i = 0; i < 4; i++) {
      const uint32_t ja = ks.galois_add == 1u ? j0 + i : galois_src(j0 + i, ks.galois_add, logn);
      r0[i] = add_mod(r0[i], shoup(__ldg(ap + ja), pm.x, pm.y, P.q), P.q);
      if (ks.add_c1) r1[i] = add_mod(r1[i], shoup(__ldg(ap + (size_t)ks.level * N + ja), pm.x, pm.y, P.q), P.q);
    }
  }
  uint32_t *d0 = sg.dst + (size_t)within * N + j0, *d1 = d0 + (size_t)ks.n_ext * N;
  *reinterpret_cast<uint4 *>(d0) = make_uint4(r0[0], r0[1], r0[2], r0[3]);
  *reinterpret_cast<uint4 *>(d1) = make_uint4(r1[0], r1[1], r1[2], r1[3]);
}

// Stage 2 as a persistent streaming kernel (the ext limbs are read in order).
// A unit is kIpChunk coefficients of one extended limb.  A producer warp (one
// lane) streams each unit's operands -- per digit the ModUp value (ext, or the
// own limb when it is not read through an automorphism) and both key halves,
// 4 KB each -- into a ring of shared-memory stages with cp.async.bulk,
// completing on the stage's full mbarrier, after writing the unit's descriptor
// (output, prime, digit count) next to the stage; it refills a stage as soon as
// the consumers release it, up to `stages` units ahead.  Every one of the
// kIpThreads consumers waits on the barriers itself (bounded; a warp gives up
// as a whole) and releases a stage by its own arrival.  The own digit of a
// rotation (sigma_{galois_own} applied on the fly) is gathered with plain
// loads one unit ahead.
constexpr int kIpChunk = 1024;  // coefficients per unit
constexpr int kIpThreads = 256;
constexpr int kIpEpt = kIpChunk / kIpThreads;  // coefficients per thread and unit (2 or 4)
static_assert(kIpEpt == 2 || kIpEpt == 4, "inner product: 2 or 4 coefficients per thread");

// E consecutive words <-> registers (one 8- or 16-byte access)
template <int E>
__device__ __forceinline__ void ld_words(const uint32_t *p, uint32_t (&v)[E]) {
  if constexpr (E == 4) {
    const uint4 t = *reinterpret_cast<const uint4 *>(p);
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
  } else {
    const uint2 t = *reinterpret_cast<const uint2 *>(p);
    v[0] = t.x, v[1] = t.y;
  }
}
template <int E>
__device__ __forceinline__ void ldg_words(const uint32_t *p, uint32_t (&v)[E]) {
  if constexpr (E == 4) {
    const uint4 t = __ldg(reinterpret_cast<const uint4 *>(p));
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
  } else {
    const uint2 t = __ldg(reinterpret_cast<const uint2 *>(p));
    v[0] = t.x, v[1] = t.y;
  }
}
template <int E>
__device__ __forceinline__ void st_words(uint32_t *p, const uint32_t (&v)[E]) {
  if constexpr (E == 4)
    *reinterpret_cast<uint4 *>(p) = make_uint4(v[0], v[1], v[2], v[3]);
  else
    *reinterpret_cast<uint2 *>(p) = make_uint2(v[0], v[1]);
}

struct IpUnit {            // one unit, as the consumers need it
  uint32_t *d0;            // u_0 at this unit's first coefficient; u_1 = d0 + d1_off
  const uint32_t *gsrc;    // own limb read through the automorphism (nullptr: none)
  const uint32_t *esrc[4]; // GEXT: every digit's limb, read through its automorphism
  uint32_t egal[4];        // GEXT: that automorphism's Galois element
  const uint32_t *add0;    // pass-through limb added (times P) to u_0, or nullptr; add1 = add0 + add1_off
  PrimeC P;
  uint2 pm;                // P mod the unit's prime (Shoup pair)
  uint32_t d1_off, galois, j0, galois_add, add1_off;
  int beta, gjd, add1;
};

// GEXT (hoisted rotations: the ModUp digits themselves are read through the
// automorphism): only the key chunks stream through the stages; every digit's values
// are gathered with plain loads one unit ahead (the shared digits stay in L2).
template <bool GOWN, bool GEXT>
__global__ void __launch_bounds__(kIpThreads + 32, 2) k_ip_bulk(const __grid_constant__ SegList sl, const PrimeC *pc,
                                                           int logn, unsigned int *status, int beta_max, int stages) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int tid = threadIdx.x;
  const size_t N = (size_t)1 << logn;
  const int chunks = (int)(N / kIpChunk);
  const int total = sl.total * chunks;
  // stage rows per digit: the ModUp value (unless gathered) and both key halves
  constexpr int RPD = GEXT ? 2 : 3, KR = GEXT ? 0 : 1;  // rows per digit, first key row
  const size_t stage_words = (size_t)RPD * beta_max * kIpChunk;
  uint32_t *buf = reinterpret_cast<uint32_t *>(smem);
  // per stage: `bar` completes when the stage's copies have landed, `dbar` when its
  // descriptor is written, `ebar` when the consumers are done with it (then it is refilled)
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + (size_t)stages * stage_words * 4);
  uint64_t *dbar = bar + stages, *ebar = dbar + stages;
  IpUnit *desc = reinterpret_cast<IpUnit *>(ebar + stages);

  // keys are read exactly once: evict them first, so that ModUp outputs (and the digits shared
  // by hoisted rotations) stay in L2
  const uint64_t key_policy = l2_evict_first_policy();
  // the producer: describe unit u and stream its operands into stage st
  auto issue = [&](int u, int st) {
    int within;
    const Seg &sg = seg_at(sl, seg_find(sl, u / chunks, within));
    const KsArgs &ks = item_ks(sl, sg);
    const int t = sg.t0 + within, row = sg.key_row0 + within;
    const size_t c0 = (size_t)(u % chunks) * kIpChunk;
    IpUnit d;
    d.d0 = sg.dst + (size_t)within * N + c0;
    d.d1_off = (uint32_t)((size_t)ks.n_ext * N);
    d.P = pc[sg.prime + within];
    d.beta = ks.beta;
    d.gjd = (GOWN && !GEXT && t < ks.level) ? t / ks.alpha : -1;
    d.gsrc = d.gjd >= 0 ? ks.own + (size_t)t * N : nullptr;
    if (GEXT)
      for (int jd = 0; jd < 4; jd++) {
        const bool own = t < ks.level && t >= jd * ks.alpha && t < (jd + 1) * ks.alpha;
        d.esrc[jd] = jd >= ks.beta ? nullptr : own ? ks.own + (size_t)t * N : ks.ext + ((size_t)jd * ks.n_ext + t) * N;
        d.egal[jd] = own ? ks.galois_own : ks.galois_ext;
      }
    d.galois = ks.galois_own;
    d.j0 = (uint32_t)c0;
    const bool add = ks.addp && t < ks.level;
    d.add0 = add ? ks.addp + (size_t)t * N : nullptr;
    d.add1 = add && ks.add_c1;
    d.add1_off = (uint32_t)((size_t)ks.level * N);
    d.galois_add = ks.galois_add;
    d.pm = add ? ks.pmod[t] : make_uint2(0, 0);
    desc[st] = d;
    mbar_arrive(&dbar[st]);  // the descriptor is readable (release)
    const size_t kstride = (size_t)2 * (ks.L + ks.K) * N, half = (size_t)(ks.L + ks.K) * N;
    const uint32_t copies = GEXT ? 2u * (uint32_t)ks.beta : 3u * (uint32_t)ks.beta - (d.gjd >= 0 ? 1u : 0u);
    mbar_arrive_expect_tx(&bar[st], copies * kIpChunk * 4u);
    uint32_t *dst = buf + (size_t)st * stage_words;
    for (int jd = 0; jd < ks.beta; jd++) {
      if (!GEXT && jd != d.gjd) {
        const bool own = t < ks.level && t >= jd * ks.alpha && t < (jd + 1) * ks.alpha;
        const uint32_t *e = own ? ks.own + (size_t)t * N : ks.ext + ((size_t)jd * ks.n_ext + t) * N;
        bulk_g2s(dst + (size_t)(RPD * jd) * kIpChunk, e + c0, kIpChunk * 4u, &bar[st]);
      }
      const uint32_t *kp = ks.key + jd * kstride + (size_t)row * N + c0;
      bulk_g2s_hint(dst + (size_t)(RPD * jd + KR) * kIpChunk, kp, kIpChunk * 4u, &bar[st], key_policy);
      bulk_g2s_hint(dst + (size_t)(RPD * jd + KR + 1) * kIpChunk, kp + half, kIpChunk * 4u, &bar[st], key_policy);
    }
  };
  // Warp specialisation: warps 0..7 reduce units, warp 8 (one lane) produces them.  The
  // producer runs ahead of the consumers by up to `stages` units, so its dependent reads
  // of the launch descriptors stay off the consumers' path.
  if (tid == 0) {
    for (int st = 0; st < stages; st++) {
      mbar_init(&bar[st], 1);
      mbar_init(&dbar[st], 1);
      mbar_init(&ebar[st], kIpThreads);
    }
  }
  __syncthreads();
  if (tid >= kIpThreads) {
    if (tid != kIpThreads) return;
    for (int k = 0;; k++) {
      const int u = (int)blockIdx.x + k * (int)gridDim.x;
      if (u >= total) break;
      const int st = k % stages;
      // the consumers released this stage's previous unit (bounded: if they gave up, so do we)
      if (k >= stages && !mbar_wait_bounded(&ebar[st], (uint32_t)(k / stages - 1) & 1u)) break;
      fence_proxy_async_smem();
      issue(u, st);
    }
    return;
  }

  // the gathered own values of a unit are loaded one unit ahead (after the wait
  // that orders the unit's descriptor), so their latency overlaps a unit's work
  constexpr int E = kIpEpt;
  auto gather = [&](const IpUnit &d, uint32_t (&v)[E]) {
    const uint32_t j = d.j0 + tid * E;
#pragma unroll
    for (int e = 0; e < E; e++) v[e] = __ldg(d.gsrc + galois_src(j + e, d.galois, logn));
  };
  // pass-through values of a unit (read through sigma_{galois_add}), also one unit ahead
  auto pass = [&](const IpUnit &d, uint32_t (&p0)[E], uint32_t (&p1)[E]) {
    const uint32_t j = d.j0 + tid * E;
    if (d.galois_add == 1u) {
      ldg_words<E>(d.add0 + j, p0);
      if (d.add1) ldg_words<E>(d.add0 + d.add1_off + j, p1);
    } else {
#pragma unroll
      for (int e = 0; e < E; e++) p0[e] = __ldg(d.add0 + galois_src(j + e, d.galois_add, logn));
    }
  };
  // GEXT: every digit's values of a unit, one unit ahead
  constexpr int XD = GEXT ? 4 : 1;
  auto gather_all = [&](const IpUnit &d, uint32_t (&v)[XD][E]) {
    const uint32_t j = d.j0 + tid * E;
#pragma unroll
    for (int jd = 0; jd < XD; jd++)
      if (jd < d.beta)
#pragma unroll
        for (int e = 0; e < E; e++) v[jd][e] = __ldg(d.esrc[jd] + galois_src(j + e, d.egal[jd], logn));
  };
  // every consumer thread waits on the barriers itself (bounded; a warp gives up as a whole)
  uint32_t gnext[E] = {}, pnext0[E] = {}, pnext1[E] = {}, xnext[XD][E] = {};
  bool ok = true;
  if ((int)blockIdx.x < total) {
    ok = __all_sync(0xffffffffu, mbar_wait_bounded(&dbar[0], 0u));
    if (ok) {
      if (GOWN && desc[0].gjd >= 0) gather(desc[0], gnext);
      if (GEXT) gather_all(desc[0], xnext);
      if (desc[0].add0) pass(desc[0], pnext0, pnext1);
    }
  }
  int k = 0;
  for (int u = blockIdx.x; ok && u < total; u += gridDim.x, k++) {
    const int st = k % stages;
    uint32_t gv[E], pv0[E], pv1[E], xv[XD][E];
#pragma unroll
    for (int e = 0; e < E; e++) gv[e] = gnext[e], pv0[e] = pnext0[e], pv1[e] = pnext1[e];
#pragma unroll
    for (int jd = 0; jd < XD; jd++)
#pragma unroll
      for (int e = 0; e < E; e++) xv[jd][e] = xnext[jd][e];
    const bool has_next = u + (int)gridDim.x < total;
    bool w = mbar_wait_bounded(&bar[st], (uint32_t)(k / stages) & 1u);
    if (w && has_next) w = mbar_wait_bounded(&dbar[(k + 1) % stages], (uint32_t)((k + 1) / stages) & 1u);
    ok = __all_sync(0xffffffffu, w);
    if (!ok) break;
    const IpUnit d = desc[st];
    if (has_next) {  // the next unit's descriptor (its readiness was waited for above)
      const IpUnit dn = desc[(k + 1) % stages];
      if (GOWN && dn.gjd >= 0) gather(dn, gnext);
      if (GEXT) gather_all(dn, xnext);
      if (dn.add0) pass(dn, pnext0, pnext1);
    }
    const uint32_t *src = buf + (size_t)st * stage_words + tid * E;
    uint64_t a0[E] = {}, a1[E] = {};
#pragma unroll
    for (int jd = 0; jd < 4; jd++) {
      if (jd < d.beta) {
        uint32_t ev[E], k0[E], k1[E];
        if (GEXT) {
#pragma unroll
          for (int e = 0; e < E; e++) ev[e] = xv[jd < XD ? jd : 0][e];
        } else if (jd == d.gjd) {
#pragma unroll
          for (int e = 0; e < E; e++) ev[e] = gv[e];
        } else {
          ld_words<E>(src + (size_t)(RPD * jd) * kIpChunk, ev);
        }
        ld_words<E>(src + (size_t)(RPD * jd + KR) * kIpChunk, k0);
        ld_words<E>(src + (size_t)(RPD * jd + KR + 1) * kIpChunk, k1);
#pragma unroll
        for (int i = 0; i < E; i++) {
          a0[i] += (uint64_t)ev[i] * k0[i];
          a1[i] += (uint64_t)ev[i] * k1[i];
        }
      }
    }
    uint32_t r0[E], r1[E];
#pragma unroll
    for (int i = 0; i < E; i++) {
      r0[i] = reduce_u64(a0[i], d.P);
      r1[i] = reduce_u64(a1[i], d.P);
    }
    if (d.add0) {  // pass-through term: u_c += P * addp_c
      const uint32_t q = d.P.q;
#pragma unroll
      for (int i = 0; i < E; i++) {
        r0[i] = add_mod(r0[i], shoup(pv0[i], d.pm.x, d.pm.y, q), q);
        if (d.add1) r1[i] = add_mod(r1[i], shoup(pv1[i], d.pm.x, d.pm.y, q), q);
      }
    }
    uint32_t *d0 = d.d0 + tid * E;
    st_words<E>(d0, r0);
    st_words<E>(d0 + d.d1_off, r1);
    mbar_arrive(&ebar[st]);  // this thread is done with stage st and its descriptor
  }
  if (!ok && (tid & 31) == 0) {
    // an expired wait: report it, then wait (bounded) for this CTA's copies that may still
    // be in flight (the producer issues at most `stages` units beyond the last one
    // released) so that none lands after the CTA has left the SM
    atomicOr(status, 2u);
    const int issued = (total - 1 - (int)blockIdx.x) / (int)gridDim.x + 1;  // units of this CTA
    for (int k2 = k; k2 < min(issued, k + stages); k2++)
      mbar_wait_bounded(&bar[k2 % stages], (uint32_t)(k2 / stages) & 1u);
  }
}
}  // namespace fhe
