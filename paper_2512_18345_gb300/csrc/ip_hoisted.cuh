// Hoisted key inner product with the digits staged block by block (the
// hoisted rotations of Section V-C: sigma_k applied to the ModUp digits,
// u_c = sum_j sigma(ModUp_j) * key_j[c], plus P sigma(c0) on the q-limbs).
//
// In bit-reversed NTT order the automorphism maps every aligned block of 32
// coefficients onto one aligned block of 32: for a destination block B the
// low (logN - 5) bits of brv(j) k + (k - 1)/2 do not depend on the offset
// within B, so the source block is fixed and only the offset inside it is
// permuted.  The producer warp therefore copies, for each unit (1024
// coefficients of one extended limb), the 32 source blocks of every digit and
// of the pass-through polynomial into the unit's stage (16-byte cp.async
// pieces, four whole blocks per warp instruction; one 128-byte bulk copy per
// block ran at less than half the speed: the copy engine's per-copy cost
// dominates at that size), beside the unit's key chunks (4 KB bulk copies); a
// consumer thread forms
// its coefficients' within-block offsets once and reads every digit's value
// from shared memory.  The arithmetic (64-bit accumulation of at most four
// products, one reduction per half, the pass-through Shoup product) is the
// streaming inner product's, so results are bit-identical to it.
//
// Stage layout (32-bit words): beta_max digit rows and one pass-through row of
// 32 blocks at a stride of kIhSlot words (padding spreads a warp's reads over
// the banks), then 2 beta_max key rows of kIpChunk words (b_j, a_j per digit).
#pragma once
#include "async.cuh"
#include "elementwise.cuh"
#include "ntt_bulk.cuh"  // cp.async helpers

namespace fhe {

constexpr int kIhSlot = 36;               // words per staged 32-coefficient block
constexpr int kIhRow = 32 * kIhSlot;      // one staged row of 1024 coefficients

struct IhUnit {
  uint32_t *d0;              // u_0 at this unit's first coefficient; u_1 = d0 + d1_off
  const uint32_t *src[5];    // digit limbs (beta of them), then the pass-through limb (or null)
  uint32_t gal[5];           // the Galois element each of those rows is read through
  PrimeC P;
  uint2 pm;                  // P mod the unit's prime (Shoup pair)
  uint32_t d1_off, j0;
  int beta;
};

__host__ __device__ constexpr int ip_hoisted_stage_words(int beta_max) {
  return (beta_max + 1) * kIhRow + 2 * beta_max * kIpChunk;
}

__global__ void __launch_bounds__(kIpThreads + 32, 2)
    k_ip_hoisted(const __grid_constant__ SegList sl, const PrimeC *pc, int logn, unsigned int *status, int beta_max,
                 int stages) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int tid = threadIdx.x;
  const size_t N = (size_t)1 << logn;
  const int chunks = (int)(N / kIpChunk);
  const int total = sl.total * chunks;
  const size_t stage_words = (size_t)ip_hoisted_stage_words(beta_max);
  uint32_t *buf = reinterpret_cast<uint32_t *>(smem);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + (size_t)stages * stage_words * 4);  // full (+ descriptor)
  uint64_t *ebar = bar + stages;                                                         // empty
  IhUnit *desc = reinterpret_cast<IhUnit *>(ebar + stages);
  if (tid == 0)
    for (int st = 0; st < stages; st++) {
      mbar_init(&bar[st], 33);  // 32 producer lanes' copy completions + the descriptor and key bytes
      mbar_init(&ebar[st], kIpThreads);
    }
  __syncthreads();

  // each CTA takes a contiguous range of units, so that consecutive units mostly share their
  // limb and the producer re-reads the launch descriptors only when the limb changes
  const int u0 = (int)(((long long)blockIdx.x * total) / gridDim.x);
  const int u1 = (int)(((long long)(blockIdx.x + 1) * total) / gridDim.x);
  const int nunits = u1 - u0;

  if (tid >= kIpThreads) {  // ------------------------------------------------ producer warp
    const int lane = tid - kIpThreads;
    const uint64_t key_policy = l2_evict_first_policy();
    IhUnit lim;             // the current limb's descriptor (j0 = 0, d0 at the limb's start)
    const uint32_t *kp = nullptr;  // this lane's key row at coefficient 0 (lanes < 2 beta)
    int cur_v = -1;
    bool ok = true;
    for (int k = 0; k < nunits; k++) {
      const int u = u0 + k, v = u / chunks, st = k % stages;
      const size_t c0 = (size_t)(u % chunks) * kIpChunk;
      if (v != cur_v) {  // a new limb: read its arguments (before the stage wait, which hides them)
        int within;
        const Seg &sg = seg_at(sl, seg_find(sl, v, within));
        const KsArgs &ks = item_ks(sl, sg);
        const int t = sg.t0 + within, row = sg.key_row0 + within;
        const bool add = ks.addp && t < ks.level;
        lim.d0 = sg.dst + (size_t)within * N;
        lim.d1_off = (uint32_t)((size_t)ks.n_ext * N);
        lim.P = pc[sg.prime + within];
        lim.beta = ks.beta;
        for (int jd = 0; jd < 4; jd++) {
          const bool own = t < ks.level && t >= jd * ks.alpha && t < (jd + 1) * ks.alpha;
          lim.src[jd] = jd >= ks.beta ? nullptr : own ? ks.own + (size_t)t * N : ks.ext + ((size_t)jd * ks.n_ext + t) * N;
          lim.gal[jd] = own ? ks.galois_own : ks.galois_ext;
        }
        lim.src[4] = add ? ks.addp + (size_t)t * N : nullptr;
        lim.gal[4] = ks.galois_add;
        lim.pm = add ? ks.pmod[t] : make_uint2(0, 0);
        const size_t kstride = (size_t)2 * (ks.L + ks.K) * N, half = (size_t)(ks.L + ks.K) * N;
        kp = lane < 2 * ks.beta ? ks.key + (lane >> 1) * kstride + (lane & 1) * half + (size_t)row * N : nullptr;
        cur_v = v;
      }
      if (k >= stages) {  // the consumers released this stage's previous unit (bounded)
        bool w = true;
        if (lane == 0) w = mbar_wait_bounded(&ebar[st], (uint32_t)(k / stages - 1) & 1u);
        ok = __shfl_sync(0xffffffffu, w ? 1 : 0, 0) != 0;
        if (!ok) break;
      }
      fence_proxy_async_smem();
      if (lane == 0) {
        IhUnit d = lim;
        d.d0 = lim.d0 + c0;
        d.j0 = (uint32_t)c0;
        desc[st] = d;
        // lane 0's arrival: the descriptor (release) and the key chunks' bytes
        mbar_arrive_expect_tx(&bar[st], 2u * (uint32_t)lim.beta * kIpChunk * 4u);
      }
      __syncwarp();
      uint32_t *dst = buf + (size_t)st * stage_words;
      const uint32_t sbase = smem_addr(dst);
      // Every staged row: lane b forms the source block of destination block b, and the warp
      // copies the row in 16-byte pieces, eight per lane, each warp instruction covering four
      // whole 128-byte blocks (lane l: block 4 i + l / 8, piece l % 8).
      const uint32_t jb = (uint32_t)c0 + 32u * (uint32_t)lane;
      const uint32_t sb0 = galois_src(jb, lim.gal[0], logn) >> 5;
      const int part = lane & 7;
#pragma unroll
      for (int r = 0; r < 5; r++) {
        const uint32_t *srow = r < 4 ? (r < lim.beta ? lim.src[r] : nullptr) : lim.src[4];
        if (!srow) continue;  // uniform over the warp
        const uint32_t sbl = lim.gal[r] == lim.gal[0] ? sb0 : galois_src(jb, lim.gal[r], logn) >> 5;
        const int slot_row = r < 4 ? r : beta_max;  // the pass-through row follows beta_max digit rows
        const uint32_t rbase = sbase + (uint32_t)(slot_row * kIhRow) * 4u;
#pragma unroll
        for (int i = 0; i < 8; i++) {
          const int b = 4 * i + (lane >> 3);
          const uint32_t sbb = __shfl_sync(0xffffffffu, sbl, b);
          cp_async16(rbase + (uint32_t)(b * kIhSlot + 4 * part) * 4u, srow + ((size_t)sbb << 5) + 4 * part);
        }
      }
      cp_async_arrive_noinc(&bar[st]);  // one arrival per lane once its pieces have landed
      if (kp)  // key chunks: b_j and a_j of digit lane / 2
        bulk_g2s_hint(dst + (size_t)(beta_max + 1) * kIhRow + (size_t)lane * kIpChunk, kp + c0, kIpChunk * 4u,
                      &bar[st], key_policy);
    }
    cp_async_wait_all();  // no copy of this warp is still in flight when it leaves
    return;
  }

  // ---------------------------------------------------------------- consumer warps
  constexpr int E = kIpEpt;
  bool ok = true;
  int k = 0;
  for (; k < nunits; k++) {
    const int st = k % stages;
    ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar[st], (uint32_t)(k / stages) & 1u));
    if (!ok) break;
    const IhUnit d = desc[st];
    const uint32_t *sb = buf + (size_t)st * stage_words;
    const uint32_t j = d.j0 + tid * E;
    const int base = (tid * E >> 5) * kIhSlot;  // this thread's block slot (its E coefficients share a block)
    // within-block source offsets, formed once for the Galois element the rows share (a row
    // read through another element -- an own digit or the pass-through of a mixed batch --
    // forms its own)
    const uint32_t g0 = d.gal[0];
    int off[E];
#pragma unroll
    for (int e = 0; e < E; e++) off[e] = base + (int)(galois_src(j + e, g0, logn) & 31u);
    auto offsets = [&](uint32_t g, int (&o)[E]) {
#pragma unroll
      for (int e = 0; e < E; e++) o[e] = g == g0 ? off[e] : base + (int)(galois_src(j + e, g, logn) & 31u);
    };
    const uint32_t *keys = sb + (size_t)(beta_max + 1) * kIhRow + tid * E;
    uint64_t a0[E] = {}, a1[E] = {};
#pragma unroll
    for (int jd = 0; jd < 4; jd++) {
      if (jd < d.beta) {
        const uint32_t *rowp = sb + (size_t)jd * kIhRow;
        int o[E];
        offsets(d.gal[jd], o);
        uint32_t k0[E], k1[E];
        ld_words<E>(keys + (size_t)(2 * jd) * kIpChunk, k0);
        ld_words<E>(keys + (size_t)(2 * jd + 1) * kIpChunk, k1);
#pragma unroll
        for (int e = 0; e < E; e++) {
          const uint32_t ev = rowp[o[e]];
          a0[e] += (uint64_t)ev * k0[e];
          a1[e] += (uint64_t)ev * k1[e];
        }
      }
    }
    uint32_t r0[E], r1[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
      r0[e] = reduce_u64(a0[e], d.P);
      r1[e] = reduce_u64(a1[e], d.P);
    }
    if (d.src[4]) {  // pass-through term: u_0 += P * sigma(c0)
      const uint32_t *prow = sb + (size_t)beta_max * kIhRow;
      const uint32_t q = d.P.q;
      int o[E];
      offsets(d.gal[4], o);
#pragma unroll
      for (int e = 0; e < E; e++) r0[e] = add_mod(r0[e], shoup(prow[o[e]], d.pm.x, d.pm.y, q), q);
    }
    mbar_arrive(&ebar[st]);  // this thread is done with stage st
    st_words<E>(d.d0 + tid * E, r0);
    st_words<E>(d.d0 + d.d1_off + tid * E, r1);
  }
  if (!ok && (tid & 31) == 0) {
    // an expired wait: report it, then wait (bounded) for this CTA's copies that may still be
    // in flight (at most `stages` units beyond the last one consumed)
    atomicOr(status, 2u);
    for (int k2 = k; k2 < min(nunits, k + stages); k2++)
      mbar_wait_bounded(&bar[k2 % stages], (uint32_t)(k2 / stages) & 1u);
  }
}

}  // namespace fhe
