// The key inner product of the special limbs fused with the first pass of
// ModDown's inverse NTT (Section IV, stage 2 feeding stage 3; Section III-D's
// fusion of element-wise producers into a transform).
//
// In the key switch, the inner product's K special limbs u_c[p_k] are read by
// one kernel only: the inverse block pass that starts ModDown (INTT of u_c | P,
// Section IV stage 3).  A CTA here owns one 4096-coefficient block tile of one
// special limb of one half c: every thread forms u_c at its 16 coefficients
// (sum over the beta digits of ModUp_j * key_j[c], 64-bit lazy accumulation,
// one reduction, as the streaming inner product does), holding them in the
// layout the inverse block pass's first (lo) round wants (16 contiguous
// coefficients), then runs that pass -- lo round, exchange within its
// half-warp, hi round -- and writes the pass's lazy output in place of the
// separate launch's.  u_c's special limbs never reach memory.
//
// The arithmetic is the inner product's and the block pass's exactly, so the
// result is bit-identical to the unfused pair.  N = 2^16; digits of the
// extended basis read directly (not through an automorphism: hoisted rotations
// keep the unfused pair).
#pragma once
#include "ntt_bulk.cuh"

namespace fhe {

constexpr int kIpIttThreads = 256;

template <int BMAX>
__global__ void __launch_bounds__(kIpIttThreads, 3) k_ip_intt(const __grid_constant__ SegList sl, const NttTables tb) {
  constexpr int N = 1 << 16, S0 = 8;
  __shared__ __align__(16) uint32_t xs[kNbDataWords];  // exchange, block layout of ntt_bulk.cuh
  __shared__ uint2 tws[240];                            // hi-round twiddles of the tile's 16 blocks
  const int tid = threadIdx.x, c = tid >> 4, tau = tid & 15;
  const int tile = blockIdx.x & 15, cc = (blockIdx.x >> 4) & 1, v = blockIdx.x >> 5;
  int within;
  const Seg &sg = seg_at(sl, seg_find(sl, v, within));
  const KsArgs &ks = item_ks(sl, sg);
  const int t = sg.t0 + within, row = sg.key_row0 + within, prime = sg.prime + within;
  const PrimeC P = tb.pc[prime];
  const uint32_t q = P.q;
  const uint2 *tw = tb.tw_inv + (size_t)prime * N;
  // hi-round twiddles: psi^-brv(2^(8 + m) + (16 tile << m) + i), i < 16 2^m, at 16 (2^m - 1)
#pragma unroll
  for (int m = 0; m < 4; m++)
    if (tid < (16 << m)) tws[16 * ((1 << m) - 1) + tid] = __ldg(tw + (1 << (S0 + m)) + ((tile * 16) << m) + tid);

  // u_c at this thread's 16 coefficients (the lo layout of block c: 16 tau + e)
  const size_t j0 = (size_t)tile * kTile + c * 256 + tau * 16;
  const size_t kstride = (size_t)2 * (ks.L + ks.K) * N, half = (size_t)(ks.L + ks.K) * N;
  uint64_t acc[16];
#pragma unroll
  for (int e = 0; e < 16; e++) acc[e] = 0;
#pragma unroll
  for (int jd = 0; jd < BMAX; jd++) {
    if (jd < ks.beta) {
      const uint4 *ep = reinterpret_cast<const uint4 *>(ks.ext + ((size_t)jd * ks.n_ext + t) * N + j0);
      const uint4 *kp = reinterpret_cast<const uint4 *>(ks.key + jd * kstride + cc * half + (size_t)row * N + j0);
#pragma unroll
      for (int e4 = 0; e4 < 4; e4++) {
        const uint4 ev = __ldg(ep + e4), kv = __ldcs(kp + e4);  // keys are read once: stream them
        acc[4 * e4] += (uint64_t)ev.x * kv.x;
        acc[4 * e4 + 1] += (uint64_t)ev.y * kv.y;
        acc[4 * e4 + 2] += (uint64_t)ev.z * kv.z;
        acc[4 * e4 + 3] += (uint64_t)ev.w * kv.w;
      }
    }
  }
  uint32_t x[16];
#pragma unroll
  for (int e = 0; e < 16; e++) x[e] = reduce_u64(acc[e], P);

  // the inverse block pass: lo round (register twiddles), exchange, hi round (staged twiddles)
  {
    uint2 Lw[15];
    nb_twiddles<false>(tw, tile, c, tau, Lw);
    nb_round<false>(x, [&](int m, int j) { return Lw[(1 << m) - 1 + j]; }, q);
  }
#pragma unroll
  for (int m = 0; m < 4; m++)
    *reinterpret_cast<uint4 *>(xs + nb_blk_addr(c, (tau << 4) | (4 * m))) =
        make_uint4(x[4 * m], x[4 * m + 1], x[4 * m + 2], x[4 * m + 3]);
  __syncthreads();  // the staged twiddles (all threads) and this half-warp's exchange
#pragma unroll
  for (int e = 0; e < 16; e++) x[e] = xs[nb_blk_addr(c, (e << 4) | tau)];
  nb_round<false>(x, [&](int m, int j) { return tws[16 * ((1 << m) - 1) + (c << m) + j]; }, q);
  uint32_t *dst = sg.dst + ((size_t)cc * ks.K + within) * N + (size_t)tile * kTile + c * 256 + tau;
#pragma unroll
  for (int e = 0; e < 16; e++) dst[e * 16] = x[e];  // lazy, hi layout (16 e + tau)
}

}  // namespace fhe
