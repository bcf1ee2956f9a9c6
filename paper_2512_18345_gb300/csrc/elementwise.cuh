// Element-wise kernels of the plain (per-kernel) pipeline: automorphism
// gather, scaling, key inner product, ModDown combine, HMult tensor product,
// addition and plaintext multiplication (Section II-B "The rest": element-wise
// parallel operations over L x N).  Four elements per thread; contiguous
// reads and writes are 128-bit.
#pragma once
#include "common.cuh"
#include "ntt.cuh"

namespace fhe {

constexpr int kEwThreads = 256;

enum : int {
  EW_GATHER = 0,   // dst = src[sigma(j)]               (galois = ks.galois_own)
  EW_SCALE = 1,    // dst = src * scale[l]
  EW_IP = 2,       // (k_ip) both halves of the key inner product
  EW_COMBINE = 3,  // dst = (src - src2) P^-1 (+ add)  (src = u, src2 = NTT(r))
  EW_ADD = 4,      // dst = src + src2
  EW_MUL = 5,      // dst = src * src2
  EW_COPY = 6,     // dst = src
};

template <int OP>
__global__ void __launch_bounds__(kEwThreads) k_ew(const __grid_constant__ SegList sl, const PrimeC *pc,
                                                   const __grid_constant__ KsArgs ks, int logn) {
  const size_t N = (size_t)1 << logn;
  const int blocks_per_limb = (int)(N / (4 * kEwThreads));
  const int v = blockIdx.x / blocks_per_limb;
  const uint32_t j0 = (uint32_t)((blockIdx.x % blocks_per_limb) * 4 * kEwThreads + threadIdx.x * 4);
  int within;
  const Seg &sg = seg_at(sl, seg_find(sl, v, within));
  const int prime = sg.prime + within;
  const PrimeC P = pc[prime];
  const uint32_t q = P.q;
  const uint32_t *src = sg.src ? sg.src + (size_t)within * sg.src_stride * N : nullptr;
  const uint32_t *src2 = sg.src2 ? sg.src2 + (size_t)within * N : nullptr;
  uint32_t *dst = sg.dst + (size_t)within * N;
  uint32_t o[4];
  if (OP == EW_GATHER) {
#pragma unroll
    for (int e = 0; e < 4; e++) o[e] = __ldg(src + galois_src(j0 + e, ks.galois_own, logn));
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
      else {  // EW_COMBINE
        uint32_t r = shoup(av[e] + q - bv[e], sc.x, sc.y, q);
        const int t = sg.t0 + within;
        if (ks.addp && (sg.c == 0 || ks.add_c1)) {
          const uint32_t ja = ks.galois_add == 1u ? j0 + e : galois_src(j0 + e, ks.galois_add, logn);
          r = add_mod(r, __ldg(ks.addp + ((size_t)sg.c * ks.level + t) * N + ja), q);
        }
        o[e] = r;
      }
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
__global__ void __launch_bounds__(kEwThreads) k_ip(const __grid_constant__ SegList sl, const PrimeC *pc,
                                                   const __grid_constant__ KsArgs ks, int logn) {
  const size_t N = (size_t)1 << logn;
  const int blocks_per_limb = (int)(N / (4 * kEwThreads));
  const int v = blockIdx.x / blocks_per_limb;
  const uint32_t j0 = (uint32_t)((blockIdx.x % blocks_per_limb) * 4 * kEwThreads + threadIdx.x * 4);
  int within;
  const Seg &sg = seg_at(sl, seg_find(sl, v, within));
  const int t = sg.t0 + within, row = sg.key_row0 + within;
  const PrimeC P = pc[sg.prime + within];
  const size_t kstride = (size_t)2 * (ks.L + ks.K) * N;
  uint64_t a0[4] = {0, 0, 0, 0}, a1[4] = {0, 0, 0, 0};
#pragma unroll
  for (int jd = 0; jd < 4; jd++) {
    if (jd >= ks.beta) break;
    const bool own = t < ks.level && t >= jd * ks.alpha && t < (jd + 1) * ks.alpha;
    uint32_t e[4];
    if (own) {
      const uint32_t *p = ks.own + (size_t)t * N;
      if (GOWN) {
#pragma unroll
        for (int i = 0; i < 4; i++) e[i] = __ldg(p + galois_src(j0 + i, ks.galois_own, logn));
      } else {
        const uint4 x = __ldg(reinterpret_cast<const uint4 *>(p + j0));
        e[0] = x.x; e[1] = x.y; e[2] = x.z; e[3] = x.w;
      }
    } else {
      const uint32_t *p = ks.ext + ((size_t)jd * ks.n_ext + t) * N;
      if (GEXT) {
#pragma unroll
        for (int i = 0; i < 4; i++) e[i] = __ldg(p + galois_src(j0 + i, ks.galois_ext, logn));
      } else {
        const uint4 x = __ldg(reinterpret_cast<const uint4 *>(p + j0));
        e[0] = x.x; e[1] = x.y; e[2] = x.z; e[3] = x.w;
      }
    }
    const uint32_t *kp = ks.key + jd * kstride + (size_t)row * N + j0;
    const uint4 k0 = __ldg(reinterpret_cast<const uint4 *>(kp));
    const uint4 k1 = __ldg(reinterpret_cast<const uint4 *>(kp + (size_t)(ks.L + ks.K) * N));
    const uint32_t kk0[4] = {k0.x, k0.y, k0.z, k0.w}, kk1[4] = {k1.x, k1.y, k1.z, k1.w};
#pragma unroll
    for (int i = 0; i < 4; i++) {
      a0[i] += (uint64_t)e[i] * kk0[i];
      a1[i] += (uint64_t)e[i] * kk1[i];
    }
  }
  uint32_t *d0 = sg.dst + (size_t)within * N + j0, *d1 = d0 + (size_t)ks.n_ext * N;
  *reinterpret_cast<uint4 *>(d0) = make_uint4(reduce_u64(a0[0], P), reduce_u64(a0[1], P), reduce_u64(a0[2], P),
                                              reduce_u64(a0[3], P));
  *reinterpret_cast<uint4 *>(d1) = make_uint4(reduce_u64(a1[0], P), reduce_u64(a1[1], P), reduce_u64(a1[2], P),
                                              reduce_u64(a1[3], P));
}

}  // namespace fhe
