// Negacyclic NTT / INTT of RNS limbs as two stage-range passes (Section
// II-B butterflies; Section III-D explains why a 2^16-point limb needs two
// kernels: it does not fit one block's shared memory).
//
// Forward: natural-order coefficients -> bit-reversed evaluations,
//   out[i] = sum_n a[n] psi^((2 brv(i)+1) n).  Cooley-Tukey stage s (pair
//   distance 2^(logN-1-s)) uses psi^brv(2^s + (j >> (logN - s))) for the pair's
//   lower index j.
// Inverse: Gentleman-Sande mirror with psi^-brv(...) and a final scale
//   (N^-1 times an optional per-limb constant, e.g. the BConv pre-factor).
//
// Pass A ("column"): the first logN-8 stages, on 2^(logN-8)-point strided
//   sub-transforms; pass B ("block"): the last 8 stages on contiguous
//   256-element blocks.  The inverse runs B then A.  A tile is 4096 elements
//   (16 KB of shared memory), 256 threads, 16 elements per thread held in
//   registers through 4 butterfly stages per shared-memory round trip.
//   Butterflies keep values lazily in [0, 2q) (q < 2^31).
#pragma once
#include "common.cuh"

namespace fhe {

struct NttTables {
  const PrimeC *pc;
  const uint2 *tw_fwd;  // [primes][N] (w, floor(w 2^32 / q)), w = psi^brv(index)
  const uint2 *tw_inv;  // [primes][N] with psi^-1
  const uint2 *ninv;    // [primes] N^-1
};

// Prologue modes (how pass 1 reads an element)
enum : int {
  PRO_PLAIN = 0,   // src[j]
  PRO_GATHER = 1,  // src[sigma(j)], sigma = ks.galois_own (NTT form input)
  PRO_REDUCE = 2,  // src[j] reduced from another prime (rescale: src_prime)
};
// Epilogue modes (how the last pass writes an element)
enum : int {
  EPI_LAZY = 0,     // write [0, 2q) (intermediate)
  EPI_PLAIN = 1,    // write reduced
  EPI_SCALE = 2,    // write v * scale (inverse final: N^-1 * constant)
  EPI_COMBINE = 3,  // ModDown combine: (src2[j] - v) P^-1 (+ add), src2 = inner product u
  EPI_RESCALE = 4,  // (src2[j] - v) * scale
};

template <int LOGN, bool COLUMN>
struct NttGeom {
  static constexpr int N = 1 << LOGN;
  static constexpr int R = COLUMN ? LOGN - 8 : 8;  // stages in this pass
  static constexpr int S = 1 << R;                 // points per sub-transform
  static constexpr int C = kTile / S;              // sub-transforms per tile
  static constexpr int LOGD = COLUMN ? LOGN - R : 0;
  static constexpr int TILES = N / kTile;
  static constexpr int SMEM = (COLUMN && R == 4) ? kTile : kTile + 256;
  // shared-memory address of element k of sub-transform c (bank-conflict free for the rounds)
  static __device__ __forceinline__ int addr(int c, int k) {
    if (COLUMN) {
      if (R == 4) return k * 256 + c;
      return k * 16 + c + ((k >> 4) << 4);
    }
    return c * 272 + ((k >> 4) << 4) + ((k & 15) ^ (k >> 4));
  }
  // index within the limb of element k of sub-transform c in tile `tile`
  static __device__ __forceinline__ uint32_t gidx(int tile, int c, int k) {
    if (COLUMN) return (uint32_t)(tile * C + c + (k << LOGD));
    return (uint32_t)(((tile * C + c) << 8) + k);
  }
};

template <int LOGN, bool COLUMN, bool FWD, int PRO, int EPI>
__global__ void __launch_bounds__(kNttThreads) k_ntt(const __grid_constant__ SegList sl, const NttTables tb,
                                                     const __grid_constant__ KsArgs ks) {
  using G = NttGeom<LOGN, COLUMN>;
  constexpr int R = G::R, C = G::C, N = G::N, LOGD = G::LOGD;
  __shared__ uint32_t sm[G::SMEM];
  __shared__ uint2 tws[COLUMN ? G::S : 1];

  const int v = blockIdx.x / G::TILES, tile = blockIdx.x % G::TILES;
  int within;
  const int si = seg_find(sl, v, within);
  const Seg &sg = seg_at(sl, si);
  const int prime = sg.prime + within;
  const PrimeC P = tb.pc[prime];
  const uint32_t q = P.q;
  const uint2 *tw = (FWD ? tb.tw_fwd : tb.tw_inv) + (size_t)prime * N;
  const uint32_t *src = sg.src + (size_t)within * sg.src_stride * N;
  uint32_t *dst = sg.dst + (size_t)within * N;
  const int tid = threadIdx.x;

  if (COLUMN) {
    for (int i = tid; i < G::S; i += kNttThreads) tws[i] = __ldg(tw + i);
  }

  // ---- load the tile (coalesced along the contiguous direction)
#pragma unroll 4
  for (int it = 0; it < 16; it++) {
    const int idx = it * kNttThreads + tid;
    int c, k;
    if (COLUMN) {
      c = idx % C;
      k = idx / C;
    } else {
      k = idx & 255;
      c = idx >> 8;
    }
    const uint32_t j = G::gidx(tile, c, k);
    uint32_t x;
    if (PRO == PRO_PLAIN) {
      x = __ldg(src + j);
    } else if (PRO == PRO_GATHER) {
      x = __ldg(src + galois_src(j, ks.galois_own, LOGN));
    } else {  // PRO_REDUCE: value of another prime's limb, reduced exactly mod q
      x = reduce_u64(__ldg(src + j), P);
    }
    sm[G::addr(c, k)] = x;
  }
  __syncthreads();

  // ---- butterfly rounds, 4 stages per round in registers
  int c, tau;
  if (COLUMN && R == 4) {
    c = tid;
    tau = 0;
  } else if (COLUMN) {
    c = tid & 15;
    tau = tid >> 4;
  } else {
    c = tid >> 4;
    tau = tid & 15;
  }
  constexpr int ROUNDS = R / 4;
#pragma unroll
  for (int rho = 0; rho < ROUNDS; rho++) {
    // hi round: e occupies k bits 7..4; lo round: k bits 3..0 (R == 4: k = e)
    const bool hi = (R == 8) && (FWD ? rho == 0 : rho == 1);
    uint32_t x[16];
#pragma unroll
    for (int e = 0; e < 16; e++) {
      const int k = (R == 4) ? e : (hi ? ((e << 4) | tau) : ((tau << 4) | e));
      x[e] = sm[G::addr(c, k)];
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
      const int bit = FWD ? 3 - i : i;
      const int kbit = hi ? bit + 4 : bit;
      const int gbit = LOGD + kbit;                 // pair distance 2^gbit in the limb
      const int s = LOGN - 1 - gbit;                // Cooley-Tukey stage index
#pragma unroll
      for (int e = 0; e < 16; e++) {
        if (e & (1 << bit)) continue;
        const int e2 = e | (1 << bit);
        const int klo = (R == 4) ? e : (hi ? ((e << 4) | tau) : ((tau << 4) | e));
        const uint32_t jlo = G::gidx(tile, c, klo);
        const uint32_t widx = (1u << s) + (jlo >> (gbit + 1));
        const uint2 W = COLUMN ? tws[widx] : __ldg(tw + widx);
        if (FWD) {
          const uint32_t t = red2(shoup_lazy(x[e2], W.x, W.y, q), q);
          const uint32_t u = red2(x[e], q);
          x[e] = u + t;
          x[e2] = u - t + q;
        } else {
          const uint32_t u = red2(x[e], q), w = red2(x[e2], q);
          x[e] = u + w;
          x[e2] = shoup_lazy(u - w + q, W.x, W.y, q);
        }
      }
    }
#pragma unroll
    for (int e = 0; e < 16; e++) {
      const int k = (R == 4) ? e : (hi ? ((e << 4) | tau) : ((tau << 4) | e));
      sm[G::addr(c, k)] = x[e];
    }
    __syncthreads();
  }

  // ---- store the tile
  uint2 scale = make_uint2(0, 0);
  if (EPI == EPI_SCALE || EPI == EPI_RESCALE) scale = sg.scale ? sg.scale[within] : tb.ninv[prime];
  uint2 pinv = make_uint2(0, 0);
  if (EPI == EPI_COMBINE) pinv = ks.pinv[prime];
#pragma unroll 4
  for (int it = 0; it < 16; it++) {
    const int idx = it * kNttThreads + tid;
    int cc, k;
    if (COLUMN) {
      cc = idx % C;
      k = idx / C;
    } else {
      k = idx & 255;
      cc = idx >> 8;
    }
    const uint32_t j = G::gidx(tile, cc, k);
    const uint32_t val = sm[G::addr(cc, k)];
    uint32_t o;
    if (EPI == EPI_LAZY) {
      o = val;
    } else if (EPI == EPI_PLAIN) {
      o = red2(val, q);
    } else if (EPI == EPI_SCALE) {
      o = shoup(val, scale.x, scale.y, q);
    } else if (EPI == EPI_RESCALE) {
      const uint32_t a = __ldg(sg.src2 + (size_t)within * N + j);
      o = shoup(a + q - red2(val, q), scale.x, scale.y, q);
    } else {  // EPI_COMBINE: limb t = t0 + within is a q-limb (< level)
      const int t = sg.t0 + within;
      const uint32_t u = __ldg(sg.src2 + (size_t)within * N + j);
      o = shoup(u + q - red2(val, q), pinv.x, pinv.y, q);
      if (ks.addp && (sg.c == 0 || ks.add_c1)) {
        const uint32_t ja = ks.galois_add == 1u ? j : galois_src(j, ks.galois_add, LOGN);
        o = add_mod(o, __ldg(ks.addp + ((size_t)sg.c * ks.level + t) * N + ja), q);
      }
    }
    dst[j] = o;
  }
}

}  // namespace fhe
