// Shared device definitions of the GB300 key-switching library: word-sized
// modular arithmetic on 31-bit primes and the launch descriptors every kernel
// reads.  Device-only (plus plain structs the host fills in).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fhe {

constexpr int kMaxPrimes = 64;
constexpr int kMaxSeg = 96;       // segments passed by value per launch (kernel parameters up to 32 KB)
constexpr int kTile = 4096;       // elements per NTT tile (16 KB)
constexpr int kNttThreads = 256;  // 16 elements per thread

// Per-prime constants (host-computed).  q < 2^31 so that 2q fits in 32 bits.
struct PrimeC {
  uint32_t q;
  uint32_t r32, r32s;   // 2^32 mod q and its Shoup companion floor(r32 2^32 / q)
  uint32_t div32;       // floor(2^32 / q) = Shoup companion of 1
  uint32_t r64, r64s;   // 2^64 mod q and companion
  uint32_t r34;         // 2^34 mod q (the diagonal pass's fold constant)
  uint32_t pad1;
};

// ---------------------------------------------------------------- arithmetic
// [0, 2q) -> [0, q): if x < q then x - q wraps above x and min keeps x.
__device__ __forceinline__ uint32_t red2(uint32_t x, uint32_t q) { return min(x, x - q); }

// Shoup product a * w mod q in [0, 2q) for any a < 2^32, w < q, ws = floor(w 2^32 / q).
__device__ __forceinline__ uint32_t shoup_lazy(uint32_t a, uint32_t w, uint32_t ws, uint32_t q) {
  return a * w - __umulhi(a, ws) * q;
}
__device__ __forceinline__ uint32_t shoup(uint32_t a, uint32_t w, uint32_t ws, uint32_t q) {
  return red2(shoup_lazy(a, w, ws, q), q);
}
__device__ __forceinline__ uint32_t shoup(uint32_t a, uint2 w, uint32_t q) { return shoup(a, w.x, w.y, q); }

__device__ __forceinline__ uint32_t add_mod(uint32_t a, uint32_t b, uint32_t q) { return red2(a + b, q); }
__device__ __forceinline__ uint32_t sub_mod(uint32_t a, uint32_t b, uint32_t q) { return red2(a + q - b, q); }

// Exact x mod q for any 64-bit x: x = xh 2^32 + xl, xh * (2^32 mod q) and xl
// each reduced with a Shoup product (the second with w = 1).
__device__ __forceinline__ uint32_t reduce_u64(uint64_t x, const PrimeC &P) {
  const uint32_t xh = (uint32_t)(x >> 32), xl = (uint32_t)x;
  const uint32_t t1 = red2(shoup_lazy(xh, P.r32, P.r32s, P.q), P.q);
  const uint32_t t2 = red2(xl - __umulhi(xl, P.div32) * P.q, P.q);
  return red2(t1 + t2, P.q);
}

__device__ __forceinline__ uint32_t mul_mod(uint32_t a, uint32_t b, const PrimeC &P) {
  return reduce_u64((uint64_t)a * b, P);
}

// ---------------------------------------------------------------- automorphism
// NTT-form Galois map sigma_k: slot i (value at psi^(2 brv(i)+1)) of the
// output is slot j of the input with 2 brv(j) + 1 = (2 brv(i) + 1) k mod 2N,
// i.e. brv(j) = brv(i) k + (k - 1)/2 mod N.
__device__ __forceinline__ uint32_t galois_src(uint32_t i, uint32_t k, int logn) {
  const uint32_t r = __brev(i) >> (32 - logn);
  const uint32_t rj = (r * k + (k >> 1)) & ((1u << logn) - 1u);
  return __brev(rj) >> (32 - logn);
}

// ---------------------------------------------------------------- descriptors
// A segment is a run of n limbs whose primes are consecutive (prime, prime+1,
// ...).  Limb l of the run reads src + l * src_stride * N and writes dst + l * N.
struct Seg {
  const uint32_t *src;
  uint32_t *dst;
  const uint32_t *src2;  // second operand (element-wise kernels), limb stride N, or null
  int n;             // limbs in the run
  int prime;         // prime index (into q_0.., p_0..) of the first limb
  int src_stride;    // in limbs (0: every limb reads the same source limb)
  int src_prime;     // prime of the source limb if it differs (rescale), else -1
  const uint2 *scale;  // per-limb Shoup constant pairs (inverse-NTT output scale), or null
  int t0;            // extended-basis index of the first limb (inner product)
  int key_row0;      // key row of the first limb
  int c;             // which half (0: b / c0, 1: a / c1) a combine uses
  int item;          // index of this segment's key-switching arguments
  uint32_t galois;   // element-wise gather: Galois element applied to src (1: none)
};

// Key-switching arguments of one item (one key switch) for the inner product,
// the automorphism gathers and the ModDown combine.
struct KsArgs {
  const uint32_t *ext;   // [beta][n_ext][N] ModUp outputs (NTT form); own-digit limbs unused
  const uint32_t *own;   // [level][N] the key-switched polynomial in NTT form (own-digit limbs)
  const uint32_t *key;   // [dnum][2][L+K][N]
  const uint32_t *addp;  // [2][level][N] pass-through polynomial (c = 0, 1) of the output, or null; the
                         // inner product adds P * addp to u's q-limbs, so ModDown's (u - r) P^-1 carries it
  const uint2 *pinv;     // [L] Shoup pairs of P^-1 mod q_i
  const uint2 *pmod;     // [L] Shoup pairs of P mod q_i
  int level, n_ext, beta, alpha, L, K;
  uint32_t galois_own;   // sigma applied when reading `own` (1 = none)
  uint32_t galois_ext;   // sigma applied when reading `ext` (hoisted rotations; 1 = none)
  uint32_t galois_add;   // sigma applied when reading `addp` (1 = none)
  int add_c1;            // addp's second polynomial also goes to c = 1 (HMult); a rotation adds c0 only
};

constexpr int kMaxInlineItems = 16;

// A launch's work list: segments and per-item arguments, either inline (by
// value, single operations) or in device memory (batched plans).
struct SegList {
  int nseg;
  int total;              // total limbs over all segments
  const Seg *dev;         // if non-null: segments in device memory
  const int2 *vmap;       // optional [total] (segment, limb within) for device lists
  const KsArgs *ksdev;    // if non-null: per-item arguments in device memory
  // optional limb-major order of an inline list, read by the hoisted inner product (0 groups:
  // list order): group g is lm_count[g] consecutive segments from lm_first[g], all of one size
  // and first extended-basis index, whose limbs are taken limb by limb across the segments
  int lm_groups;
  int lm_first[4], lm_count[4];
  Seg seg[kMaxSeg];
  KsArgs ks[kMaxInlineItems];
};

__device__ __forceinline__ const Seg &seg_at(const SegList &L, int i) { return L.dev ? L.dev[i] : L.seg[i]; }
__device__ __forceinline__ const KsArgs &item_ks(const SegList &L, const Seg &s) {
  return L.ksdev ? L.ksdev[s.item] : L.ks[s.item];
}

// Locate limb v (0 <= v < total) of a segment list: returns segment index and limb within it.
__device__ __forceinline__ int seg_find(const SegList &L, int v, int &within) {
  if (L.vmap) {
    const int2 m = L.vmap[v];
    within = m.y;
    return m.x;
  }
  int s = 0;
  for (; s < L.nseg; s++) {
    const int n = seg_at(L, s).n;
    if (v < n) break;
    v -= n;
  }
  within = v;
  return s;
}

}  // namespace fhe
