// Hoisted key inner product with the digits staged block by block (the
// hoisted rotations of Section V-C: sigma_k applied to the ModUp digits,
// u_c = sum_j sigma(ModUp_j) * key_j[c], plus P sigma(c0) on the q-limbs).
//
// In bit-reversed NTT order the automorphism maps every aligned block of 32
// coefficients onto one aligned block of 32: for a destination block B the
// low (logN - 5) bits of brv(j) k + (k - 1)/2 do not depend on the offset
// within B, so the source block is fixed and only the offset inside it is
// permuted.  So a permuted block can be copied whole (128 contiguous bytes)
// and permuted in shared memory.
//
// Every warp is its own pipeline, with no producer warp and no barrier between
// warps: a warp unit is 128 coefficients (4 blocks) of one extended limb; for
// the unit D - 1 ahead of the one it reduces, a warp copies each digit's 4
// source blocks, the pass-through polynomial's and the unit's key chunks into
// its own ring of D stages with 16-byte cp.async pieces (lane l: block l / 8,
// piece l % 8, so that one warp instruction moves 4 whole lines), and waits
// for them with cp.async.wait_group.  A single producer warp per CTA issuing
// every copy, or 128-byte bulk copies per block, both ran slower: the copy
// issue, not the memory, was the limit.
//
// Lane l reduces coefficient l of each of the unit's 4 blocks: a warp's 32
// reads of a staged block are a permutation of its 32 words (32 distinct
// banks), and its key reads and output stores are whole 128-byte lines.  The
// arithmetic (64-bit accumulation of at most four products in digit order, one
// reduction per half, the pass-through Shoup product) is the streaming inner
// product's, so results are bit-identical to it.
//
// Stage layout (32-bit words, per warp): beta_max digit rows and the
// pass-through row of 128 words each (4 blocks of 32), then 2 beta_max key
// rows of 128 words (b_j, a_j of digit j).
#pragma once
#include "async.cuh"
#include "elementwise.cuh"

namespace fhe {

constexpr int kIhMaxWarps = 16;                   // warps per CTA at most (the register file's share)
constexpr int kIhUnit = 128;                      // coefficients per warp unit
constexpr int kIhRun = 8;                         // consecutive units a warp takes at a time
__host__ __device__ constexpr int ip_hoisted_stage_words(int beta_max) { return kIhUnit * (3 * beta_max + 1); }

__device__ __forceinline__ void cp_async16_hint(uint32_t dst_smem, const void *src, uint64_t policy) {
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(dst_smem), "l"(src), "l"(policy)
               : "memory");
}
__device__ __forceinline__ void cp_async_plain16(uint32_t dst_smem, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst_smem), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// One extended limb's arguments, as a warp needs them to stage and to reduce its units.
struct IhLimb {
  const uint32_t *src[5];  // digit limbs (beta of them), then the pass-through limb (or null)
  uint32_t gal[5];         // the Galois element each of those rows is read through
  const uint32_t *key;     // key half b of digit 0 at this limb's row; digit j half c at + j kstride + c khalf
  size_t kstride, khalf;
  uint32_t *d0;            // u_0 at this limb's coefficient 0; u_1 = d0 + d1_off
  size_t d1_off;
  PrimeC P;
  uint2 pm;                // P mod the limb's prime (Shoup pair)
  int beta;
  bool mixed;              // some row in use is read through another element than gal[0]
};

// limb v of the launch: in the list's limb-major order when it has one (hoisted sets run as
// single operations, whose lists are passed by value)
__device__ __forceinline__ int ih_find(const SegList &sl, int v, int &within) {
  if (sl.lm_groups) {
    for (int g = 0; g < sl.lm_groups; g++) {
      const int m = sl.lm_count[g], size = m * sl.seg[sl.lm_first[g]].n;
      if (v < size || g == sl.lm_groups - 1) {
        within = v / m;
        return sl.lm_first[g] + v % m;
      }
      v -= size;
    }
  }
  return seg_find(sl, v, within);
}

__device__ __forceinline__ void ih_limb(const SegList &sl, const PrimeC *pc, int v, size_t N, IhLimb &o) {
  int within;
  const Seg &sg = seg_at(sl, ih_find(sl, v, within));
  const KsArgs &ks = item_ks(sl, sg);
  const int t = sg.t0 + within, row = sg.key_row0 + within;
  const bool add = ks.addp && t < ks.level;
#pragma unroll
  for (int jd = 0; jd < 4; jd++) {
    const bool own = t < ks.level && t >= jd * ks.alpha && t < (jd + 1) * ks.alpha;
    o.src[jd] = jd >= ks.beta ? nullptr : own ? ks.own + (size_t)t * N : ks.ext + ((size_t)jd * ks.n_ext + t) * N;
    o.gal[jd] = own ? ks.galois_own : ks.galois_ext;
  }
  o.src[4] = add ? ks.addp + (size_t)t * N : nullptr;
  o.gal[4] = ks.galois_add;
  o.khalf = (size_t)(ks.L + ks.K) * N;
  o.kstride = 2 * o.khalf;
  o.key = ks.key + (size_t)row * N;
  o.d0 = sg.dst + (size_t)within * N;
  o.d1_off = (size_t)ks.n_ext * N;
  o.P = pc[sg.prime + within];
  o.pm = add ? ks.pmod[t] : make_uint2(0, 0);
  o.beta = ks.beta;
  o.mixed = false;
#pragma unroll
  for (int r = 1; r < 5; r++) o.mixed |= o.src[r] && o.gal[r] != o.gal[0];
}

// D: stages per warp (units in flight while one is reduced, plus one).  The warps sweep the
// launch's units together, in runs of kIhRun consecutive units dealt out round-robin: with
// the limbs listed by extended-basis index (every rotation of a hoisted set beside the others
// at the same limb), the digits in use at any time are a few limbs', which stay in L2 while
// every rotation reads them, and a warp's limb (and its arguments) change once per run.
template <int D>
__global__ void __launch_bounds__(kIhMaxWarps * 32, 1)
    k_ip_hoisted(const __grid_constant__ SegList sl, const PrimeC *pc, int logn, int beta_max) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int warp = threadIdx.x >> 5, l = threadIdx.x & 31;
  const size_t N = (size_t)1 << logn;
  const int lpl = logn - 7;  // log2 of the units per limb (kIhUnit = 2^7)
  const int total = sl.total << lpl;
  const int sw = ip_hoisted_stage_words(beta_max);
  const int KR = (beta_max + 1) * kIhUnit;  // first key row of a stage
  uint32_t *ring = reinterpret_cast<uint32_t *>(smem) + (size_t)warp * D * sw;
  const uint32_t ring_s = smem_addr(ring);
  const int wpc = (int)(blockDim.x >> 5);
  const int gw = (int)blockIdx.x * wpc + warp, nw = (int)gridDim.x * wpc;
  // unit k of this warp: run k / kIhRun of the warp's, unit k % kIhRun of the run
  auto unit = [&](int k) { return ((k / kIhRun) * nw + gw) * kIhRun + (k % kIhRun); };
  const int runs = (total + kIhRun - 1) / kIhRun;
  const int my_runs = gw < runs ? (runs - gw + nw - 1) / nw : 0;
  const int n = my_runs ? (my_runs - 1) * kIhRun + min(kIhRun, total - (gw + (my_runs - 1) * nw) * kIhRun) : 0;
  // keys are read exactly once: evict them first, so that the digits, shared by every rotation
  // of the hoisted set, stay in L2
  const uint64_t key_policy = l2_evict_first_policy();
  const int eb = l >> 3, part = l & 7;               // staging: this lane's block and 16-byte piece
  const uint32_t pw = (uint32_t)(eb * 32 + 4 * part);  // that piece's word within a staged row

  IhLimb is, cs;  // the limbs of the unit being staged and of the unit being reduced
  int is_v = -1, cs_v = -1;
  // stage unit k of this warp's range (nothing past its end), as one cp.async group
  auto stage = [&](int k) {
    if (k < n) {
      const int g = unit(k), v = g >> lpl;
      const uint32_t c0 = (uint32_t)(g & ((1 << lpl) - 1)) * kIhUnit;
      if (v != is_v) {
        ih_limb(sl, pc, v, N, is);
        is_v = v;
      }
      const uint32_t dbase = ring_s + (uint32_t)((k % D) * sw) * 4u;
      const uint32_t jb = c0 + 32u * (uint32_t)eb;  // first coefficient of this lane's block
      const uint32_t sb0 = galois_src(jb, is.gal[0], logn) >> 5;
#pragma unroll
      for (int r = 0; r < 5; r++) {
        const uint32_t *srow = is.src[r];
        if (!srow) continue;
        uint32_t sb = sb0;
        if (is.mixed) sb = galois_src(jb, is.gal[r], logn) >> 5;  // uniform over the warp
        const int slot = r < 4 ? r : beta_max;  // the pass-through row follows beta_max digit rows
        cp_async_plain16(dbase + (uint32_t)(slot * kIhUnit + pw) * 4u, srow + ((size_t)sb << 5) + 4 * part);
      }
      const uint32_t *kp = is.key + c0 + pw;
#pragma unroll
      for (int r = 0; r < 4; r++)
        if (r < is.beta) {
          const uint32_t *kr = kp + (size_t)r * is.kstride;
          cp_async16_hint(dbase + (uint32_t)(KR + 2 * r * kIhUnit + pw) * 4u, kr, key_policy);
          cp_async16_hint(dbase + (uint32_t)(KR + (2 * r + 1) * kIhUnit + pw) * 4u, kr + is.khalf, key_policy);
        }
    }
    cp_async_commit();  // (an empty group past the end keeps the group count uniform)
  };

#pragma unroll
  for (int k = 0; k < D - 1; k++) stage(k);
  for (int k = 0; k < n; k++) {
    stage(k + D - 1);
    cp_async_wait_group<D - 1>();  // this lane's pieces of unit k have landed ...
    __syncwarp();                  // ... and every lane's
    const int g = unit(k), v = g >> lpl;
    const uint32_t c0 = (uint32_t)(g & ((1 << lpl) - 1)) * kIhUnit;
    if (v != cs_v) {
      ih_limb(sl, pc, v, N, cs);
      cs_v = v;
    }
    const uint32_t *st = ring + (size_t)(k % D) * sw;
    // this lane's coefficients c0 + 32 e + l: their staged words, formed once for the Galois
    // element the digits share (a row read through another element forms its own)
    const uint32_t ga = cs.gal[0];
    int off[4];
#pragma unroll
    for (int e = 0; e < 4; e++) off[e] = e * 32 + (int)(galois_src(c0 + 32u * e + l, ga, logn) & 31u);
    auto offsets = [&](uint32_t gx, int (&o)[4]) {
#pragma unroll
      for (int e = 0; e < 4; e++) o[e] = off[e];
      if (cs.mixed)  // uniform over the warp
#pragma unroll
        for (int e = 0; e < 4; e++) o[e] = e * 32 + (int)(galois_src(c0 + 32u * e + l, gx, logn) & 31u);
    };
    uint64_t a0[4] = {}, a1[4] = {};
#pragma unroll
    for (int r = 0; r < 4; r++)
      if (r < cs.beta) {
        int o[4];
        offsets(cs.gal[r], o);
        const uint32_t *dr = st + r * kIhUnit, *kb = st + KR + 2 * r * kIhUnit + l;
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const uint32_t ev = dr[o[e]];
          a0[e] += (uint64_t)ev * kb[32 * e];
          a1[e] += (uint64_t)ev * kb[kIhUnit + 32 * e];
        }
      }
    uint32_t r0[4], r1[4];
#pragma unroll
    for (int e = 0; e < 4; e++) {
      r0[e] = reduce_u64(a0[e], cs.P);
      r1[e] = reduce_u64(a1[e], cs.P);
    }
    if (cs.src[4]) {  // pass-through term: u_0 += P * sigma(c0)
      int o[4];
      offsets(cs.gal[4], o);
      const uint32_t *pr = st + beta_max * kIhUnit, q = cs.P.q;
#pragma unroll
      for (int e = 0; e < 4; e++) r0[e] = add_mod(r0[e], shoup(pr[o[e]], cs.pm.x, cs.pm.y, q), q);
    }
    // streaming stores: u is read by the next kernel, not reused here, and would otherwise push
    // the digits (read by every rotation of the set) out of L2
    uint32_t *d0 = cs.d0 + c0 + l;
#pragma unroll
    for (int e = 0; e < 4; e++) {
      __stcs(d0 + 32 * e, r0[e]);
      __stcs(d0 + cs.d1_off + 32 * e, r1[e]);
    }
    __syncwarp();  // every lane is done with stage k % D before it is refilled
  }
  cp_async_wait_group<0>();  // nothing in flight when the warp leaves
}

}  // namespace fhe
