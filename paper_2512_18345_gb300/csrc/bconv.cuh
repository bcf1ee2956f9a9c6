// Fast base conversion on CUDA cores (Section II-B "BConv", Section III-C).
//
// Input: n_in limbs already multiplied by [(Qstar/q_j)^-1]_{q_j} (that factor is
// folded into the preceding inverse NTT's output scale).  Output limb o with
// prime p_o:  out_o = (sum_j y_j T[o][j]) mod p_o,  T[o][j] = (Qstar/q_j) mod p_o.
// The sum is formed exactly: products are < 2^62, so groups of four fit in a
// 64-bit accumulator (IMAD.WIDE chains); group sums are added with a carry
// count, and the result (carry 2^64 + sum) is reduced once.  The paper's
// single-accumulator condition (sum_j T[i][j] Q_j < 2^64) is not needed and
// fails for about half of the word-sized prime pairs used here.
#pragma once
#include "common.cuh"

namespace fhe {

struct BconvGroup {
  const uint32_t *in;   // n_in consecutive limbs
  uint32_t *out;        // output o is written to out + omap[o].x * N
  const uint32_t *T;    // [n_out][n_in] device table
  const int2 *omap;     // [n_out] (limb offset from out, prime index)
  int n_in, n_out;
};

constexpr int kMaxBconvGroups = 8;
struct BconvArgs {
  int ngroups;
  const BconvGroup *dev;  // device array (batched plans), else g[]
  BconvGroup g[kMaxBconvGroups];
};

constexpr int kBconvThreads = 256;

// Exact (sum of n products) mod p, products y[k] * T[k] < 2^62.
template <int MAXIN>
__device__ __forceinline__ uint32_t bconv_dot(const uint32_t (&y)[MAXIN], const uint32_t *Trow, int n_in,
                                              const PrimeC &P) {
  uint64_t s = 0;
  uint32_t carry = 0;
#pragma unroll
  for (int g = 0; g < MAXIN; g += 4) {
    if (g >= n_in) break;
    uint64_t acc = 0;
#pragma unroll
    for (int k = g; k < g + 4 && k < MAXIN; k++)
      if (k < n_in) acc += (uint64_t)y[k] * Trow[k];
    const uint64_t s2 = s + acc;
    carry += s2 < s;
    s = s2;
  }
  uint32_t r = reduce_u64(s, P);
  if (carry) r = red2(r + red2(shoup_lazy(carry, P.r64, P.r64s, P.q), P.q), P.q);
  return r;
}

template <int MAXIN>
__global__ void __launch_bounds__(kBconvThreads) k_bconv(const __grid_constant__ BconvArgs a, const PrimeC *pc,
                                                         int logn) {
  __shared__ uint32_t sT[64 * 32];
  __shared__ int2 sM[64];
  const BconvGroup &g = a.dev ? a.dev[blockIdx.y] : a.g[blockIdx.y];
  const int n_in = g.n_in, n_out = g.n_out;
  for (int i = threadIdx.x; i < n_out * n_in; i += kBconvThreads) sT[i] = g.T[i];
  for (int i = threadIdx.x; i < n_out; i += kBconvThreads) sM[i] = g.omap[i];
  __syncthreads();
  const size_t N = (size_t)1 << logn;
  const size_t n = (size_t)blockIdx.x * kBconvThreads + threadIdx.x;
  uint32_t y[MAXIN];
#pragma unroll
  for (int k = 0; k < MAXIN; k++) y[k] = k < n_in ? __ldg(g.in + k * N + n) : 0u;
  for (int o = 0; o < n_out; o++) {
    const int2 m = sM[o];
    const PrimeC P = pc[m.y];
    g.out[(size_t)m.x * N + n] = bconv_dot<MAXIN>(y, sT + o * n_in, n_in, P);
  }
}

}  // namespace fhe
