// Fast base conversion on CUDA cores (Section II-B "BConv", Section III-C).
//
// Input: n_in limbs already multiplied by [(Qstar/q_j)^-1]_{q_j} (that factor is
// folded into the preceding inverse NTT's output scale), values y_j in [0, q_j).
// Output limb o with prime p_o:
//     out_o = (sum_j y_j T[o][j]) mod p_o,   T[o][j] = (Qstar/q_j) mod p_o.
// The sum is formed exactly.  Every product is below 2^62, so a group of four
// fits a 64-bit accumulator (one IMAD.WIDE per term); group sums are added
// with a carry count and the result (carry 2^64 + sum) is reduced once.  The
// paper's single-accumulator condition (sum_j T[i][j] Q_j < 2^64) is not
// needed, and it fails for about half of the 31-bit prime pairs used here.
//
// Work split: a thread converts 4 consecutive coefficients (128-bit loads and
// stores) for a chunk of up to kBconvOutChunk output limbs; the grid is
// (coefficient blocks, output chunks, groups), the table chunk sits in
// shared memory.
#pragma once
#include "common.cuh"

namespace fhe {

struct BconvGroup {
  const uint32_t *in;   // n_in consecutive limbs
  uint32_t *out;        // output o is written to out + omap[o].x * N
  const uint32_t *T;    // [n_out][n_in] device table
  const int2 *omap;     // [n_out] (limb offset from out, prime index)
  int n_in, n_out;
  const uint16_t *Btc;  // tensor-core path: digit table, canonical layout, npad x K f16 (K = 48 or 64)
  int npad;             // tc_npad(n_out)
};

// tensor-core base conversion: 128 coefficients per MMA, K = 32 data slots
// (4 bytes of at most 8 inputs) + 4 offset slots + 12 zero slots
// tensor-core base conversion: M = 128 coefficients per MMA; the contraction width K is
// 48 for at most 8 input limbs (unsigned offset slots) and 64 for 9..12 (signed offsets)
constexpr int kTcM = 128, kTcK = 48, kTcMaxIn = 8;
constexpr int kTcK12 = 64, kTcMaxIn12 = 12;
__host__ __device__ constexpr int tc_k_for(int max_in) { return max_in <= kTcMaxIn ? kTcK : kTcK12; }
__host__ __device__ constexpr int tc_npad(int n_out) { return (4 * n_out + 15) / 16 * 16; }

constexpr int kMaxBconvGroups = 48;
struct BconvArgs {
  int ngroups;
  int lazy;               // outputs may be left in [0, 2p) (they feed a forward NTT); else reduced
  const BconvGroup *dev;  // device array (batched plans), else g[]
  BconvGroup g[kMaxBconvGroups];
};

constexpr int kBconvThreads = 256;
constexpr int kBconvOutChunk = 8;

template <int NIN>
__device__ __forceinline__ void bconv_out4(const uint32_t (&y)[NIN][4], const uint32_t *Trow, const PrimeC &P,
                                           uint32_t (&r)[4]) {
  uint64_t s[4] = {0, 0, 0, 0};
  uint32_t carry[4] = {0, 0, 0, 0};
#pragma unroll
  for (int g = 0; g < NIN; g += 4) {
    uint64_t acc[4] = {0, 0, 0, 0};
#pragma unroll
    for (int k = g; k < g + 4 && k < NIN; k++) {
      const uint32_t t = Trow[k];
#pragma unroll
      for (int e = 0; e < 4; e++) acc[e] += (uint64_t)y[k][e] * t;
    }
    if (g == 0) {
#pragma unroll
      for (int e = 0; e < 4; e++) s[e] = acc[e];
    } else {
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const uint64_t s2 = s[e] + acc[e];
        carry[e] += s2 < s[e];
        s[e] = s2;
      }
    }
  }
#pragma unroll
  for (int e = 0; e < 4; e++) {
    uint32_t v = reduce_u64(s[e], P);
    if (NIN > 4 && carry[e]) v = red2(v + red2(shoup_lazy(carry[e], P.r64, P.r64s, P.q), P.q), P.q);
    r[e] = v;
  }
}

template <int NIN>
__global__ void __launch_bounds__(kBconvThreads) k_bconv(const __grid_constant__ BconvArgs a, const PrimeC *pc,
                                                         int logn) {
  __shared__ uint32_t sT[kBconvOutChunk * NIN];
  __shared__ int2 sM[kBconvOutChunk];
  __shared__ PrimeC sP[kBconvOutChunk];
  const BconvGroup &g = a.dev ? a.dev[blockIdx.z] : a.g[blockIdx.z];
  const int o0 = blockIdx.y * kBconvOutChunk;
  if (o0 >= g.n_out) return;  // uniform per block
  const int no = min(kBconvOutChunk, g.n_out - o0);
  const int n_in = g.n_in;  // <= NIN; missing inputs count as zero
  for (int i = threadIdx.x; i < no * NIN; i += kBconvThreads) {
    const int o = i / NIN, k = i - o * NIN;
    sT[i] = k < n_in ? g.T[(size_t)(o0 + o) * n_in + k] : 0u;
  }
  if (threadIdx.x < no) {
    sM[threadIdx.x] = g.omap[o0 + threadIdx.x];
    sP[threadIdx.x] = pc[sM[threadIdx.x].y];
  }
  __syncthreads();
  const size_t N = (size_t)1 << logn;
  const size_t n = ((size_t)blockIdx.x * kBconvThreads + threadIdx.x) * 4;
  uint32_t y[NIN][4];
#pragma unroll
  for (int k = 0; k < NIN; k++) {
    const uint4 v = k < n_in ? __ldg(reinterpret_cast<const uint4 *>(g.in + k * N + n)) : make_uint4(0, 0, 0, 0);
    y[k][0] = v.x;
    y[k][1] = v.y;
    y[k][2] = v.z;
    y[k][3] = v.w;
  }
  for (int o = 0; o < no; o++) {
    uint32_t r[4];
    bconv_out4<NIN>(y, sT + o * NIN, sP[o], r);
    *reinterpret_cast<uint4 *>(g.out + (size_t)sM[o].x * N + n) = make_uint4(r[0], r[1], r[2], r[3]);
  }
}

}  // namespace fhe
