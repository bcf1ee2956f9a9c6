// Base conversion on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// BConv is a dense contraction (Section II-B: Red(T . a)).  sm_103a has no
// integer tcgen05 MMA (.kind::i8 does not assemble for it), so the exact
// integer product is built from bf16 operands that hold bytes:
//   y_j = sum_a y_{j,a} 2^(8a)          (4 bytes of the 31-bit input)
//   T'_a[o][j] = (2^(8a) T[o][j]) mod p_o = sum_b D_{a,b}[o][j] 2^(8b)
//   sum_j y_j T[o][j] = sum_b 2^(8b) S_b[o]  (mod p_o),
//   S_b[o] = sum_{(j,a)} y_{j,a} D_{a,b}[o][j].
// S_b is a GEMM with M = 128 coefficients, K = 4 n_in (byte digits of the
// inputs) and N = 4 n_out ((output, weight-byte) pairs).  Bytes are exact in
// bf16; every partial sum is an integer below 4 n_in 255^2 < 2^23 (n_in <= 16),
// so the fp32 accumulation in tensor memory is exact.  The epilogue reads the
// four S_b of each output from tensor memory, forms sum_b 2^(8b) S_b < 2^46
// exactly in 64 bits and reduces it once modulo p_o: bit-identical to the
// CUDA-core path.
//
// A 128-coefficient tile of one group is one M = 128 MMA; persistent CTAs of
// 256 threads walk the tiles (see k_bconv_tc).
// Operands sit in shared memory in the canonical K-major layout without
// swizzle: 8 x 16-byte core matrices, core matrices adjacent along K 128 bytes
// apart (leading byte offset), 8-row groups (K / 8) x 128 bytes apart (stride
// byte offset).
#include <algorithm>
#include <cstring>

#include "ctx.h"
#include "internal.h"

namespace fhe {

constexpr int kTcM = 128;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared memory matrix descriptor: start address, leading / stride byte offsets,
// descriptor version 1 (bits 46..48), no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::f16 with bf16 A and B (K-major), fp32 D, shape M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// bounded wait: false when the limit expired
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase) {
  for (uint32_t it = 0; it < (1u << 20); it++) {
    if (mbar_try_wait(bar, phase)) return true;
    __nanosleep(32);
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

constexpr int kTcThreads = 256;  // 8 warps: warps w and w + 4 share accumulator lanes 32 (w % 4)..

// Persistent: a CTA walks tiles (group, 128-coefficient block) in group-major
// order, reloading the digit table only when the group changes; tensor memory
// is allocated once per CTA.  Per tile: every thread writes its half of one A
// row, thread 0 issues the MMAs and commits to the mbarrier (phase = tile
// parity), all wait (bounded), then each warp reads its lane quarter for half
// of the outputs and writes the reduced results.
__global__ void __launch_bounds__(kTcThreads) k_bconv_tc(const __grid_constant__ BconvArgs a, const PrimeC *pc,
                                                         int logn, unsigned int *status, int kpad_max, int npad_max,
                                                         int tiles_per_group) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  uint8_t *sA = smem;
  uint8_t *sB = smem + kTcM * kpad_max * 2;
  PrimeC *sP = reinterpret_cast<PrimeC *>(sB + (size_t)npad_max * kpad_max * 2);
  int2 *sM = reinterpret_cast<int2 *>(sP + 64);
  uint64_t *bar = reinterpret_cast<uint64_t *>(sM + 64);
  uint32_t *s_taddr = reinterpret_cast<uint32_t *>(bar + 1);
  const uint32_t ncols = npad_max <= 32 ? 32u : npad_max <= 64 ? 64u : npad_max <= 128 ? 128u : 256u;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_taddr)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) mbar_init(bar, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *s_taddr;

  const size_t N = (size_t)1 << logn;
  const int total = tiles_per_group * a.ngroups;
  const int per_cta = (total + gridDim.x - 1) / gridDim.x;
  const int t0 = blockIdx.x * per_cta, t1 = min(total, t0 + per_cta);
  int cur_group = -1, kpad = 0, npad = 0, n_in = 0, n_out = 0;
  const BconvGroup *gp = nullptr;
  uint32_t phase = 0;
  bool ok = true;
  for (int tile = t0; tile < t1 && ok; tile++) {
    const int grp = tile / tiles_per_group;
    const size_t n0 = (size_t)(tile % tiles_per_group) * kTcM;
    if (grp != cur_group) {  // load this group's table, output map and output primes
      cur_group = grp;
      gp = a.dev ? &a.dev[grp] : &a.g[grp];
      kpad = gp->kpad;
      npad = gp->npad;
      n_in = gp->n_in;
      n_out = gp->n_out;
      const uint4 *src = reinterpret_cast<const uint4 *>(gp->Btc);
      uint4 *dst = reinterpret_cast<uint4 *>(sB);
      const int n16 = npad * kpad * 2 / 16;
      for (int i = tid; i < n16; i += kTcThreads) dst[i] = __ldg(src + i);
      for (int o = tid; o < n_out; o += kTcThreads) {
        const int2 m = gp->omap[o];
        sM[o] = m;
        sP[o] = pc[m.y];
      }
    }
    // A: row r = tile coefficient r; column k = 4 j + a holds byte a of y_j as bf16.
    // Threads t and t + 128 build the even / odd 8-column chunks of row t % 128.
    const uint32_t sbo_a = (uint32_t)(kpad / 8) * 128u;
    {
      const int r = tid & (kTcM - 1);
      const size_t n = n0 + r;
      for (int kc = tid >> 7; kc < kpad / 8; kc += 2) {
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const int j = 2 * kc + h;
          const uint32_t y = j < n_in ? __ldg(gp->in + (size_t)j * N + n) : 0u;
          uint32_t bf[4];
#pragma unroll
          for (int d = 0; d < 4; d++) {  // exact: float(byte) = bits(2^23 + byte) - 2^23, upper half = bf16
            const float f = __uint_as_float(0x4B000000u | ((y >> (8 * d)) & 0xFFu)) - 8388608.0f;
            bf[d] = __float_as_uint(f) >> 16;
          }
          w[2 * h] = bf[0] | (bf[1] << 16);
          w[2 * h + 1] = bf[2] | (bf[3] << 16);
        }
        *reinterpret_cast<uint4 *>(sA + (r >> 3) * sbo_a + kc * 128 + (r & 7) * 16) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      const uint32_t aaddr = smem_addr(sA), baddr = smem_addr(sB);
      const uint32_t sbo_b = (uint32_t)(kpad / 8) * 128u;
      const uint32_t idesc = idesc_bf16(kTcM, npad);
      for (int kk = 0; kk < kpad / 16; kk++) {
        const uint64_t ad = smem_desc(aaddr + kk * 256u, 128u, sbo_a);
        const uint64_t bd = smem_desc(baddr + kk * 256u, 128u, sbo_b);
        const uint32_t acc = kk > 0 ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_addr(bar))
                   : "memory");
    }
    // bounded wait, made CTA-uniform (the tensor-memory loads are warp-synchronous)
    ok = __syncthreads_and(mbar_wait_bounded(bar, phase) ? 1 : 0) != 0;
    phase ^= 1u;
    tc_fence_after();
    if (ok) {
      // epilogue: warp w reads lanes 32 (w % 4).. = coefficients n0 + 32 (w % 4) + lane, and
      // the 4-output chunks c with c % 2 == w / 4; columns 4 o + b hold S_b[o]
      const int q4 = warp & 3;
      const size_t n = n0 + (size_t)q4 * 32 + (tid & 31);
      const uint32_t tbase = taddr + ((uint32_t)(q4 * 32) << 16);
      for (int o0 = 4 * (warp >> 2); o0 < n_out; o0 += 8) {
        uint32_t rr[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
            "%15}, [%16];"
            : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]), "=r"(rr[7]),
              "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]), "=r"(rr[14]),
              "=r"(rr[15])
            : "r"(tbase + (uint32_t)(4 * o0)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int i = 0; i < 4; i++) {
          const int o = o0 + i;
          if (o >= n_out) break;
          uint64_t x = 0;
#pragma unroll
          for (int b = 0; b < 4; b++) {  // exact integer S_b < 2^23: bits(S + 2^23) - bits(2^23)
            const uint32_t sv = __float_as_uint(__uint_as_float(rr[4 * i + b]) + 8388608.0f) - 0x4B000000u;
            x += (uint64_t)sv << (8 * b);
          }
          gp->out[(size_t)sM[o].x * N + n] = reduce_u64(x, sP[o]);
        }
      }
    } else {
      atomicOr(status, 1u);  // expired wait: report, give the MMA a second bounded chance
      mbar_wait_bounded(bar, phase ^ 1u);
    }
    tc_fence_before();
    __syncthreads();  // A, B and the accumulator are reused by the next tile
  }
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
  }
}

static int round16(int x) { return (x + 15) / 16 * 16; }

cudaError_t launch_bconv_tc(const DevTables &t, const BconvArgs &a, int max_in, int max_out, cudaStream_t s) {
  if (a.ngroups == 0) return cudaSuccess;
  const int kpad = round16(4 * max_in), npad = round16(4 * max_out);
  if (kpad > 64 || npad > 256 || max_out > 64) return cudaErrorInvalidValue;
  const int ncols = npad <= 32 ? 32 : npad <= 64 ? 64 : npad <= 128 ? 128 : 256;
  // operands, output primes and map, barrier; at least enough shared memory that no
  // more CTAs fit on an SM than its 512 tensor-memory columns hold
  const int need = kTcM * kpad * 2 + npad * kpad * 2 + 64 * (int)sizeof(PrimeC) + 64 * 8 + 64;
  const int per_sm = std::min(512 / ncols, 2048 / kTcThreads);
  int smem = std::max(need, 233472 / (per_sm + 1) + 1024);  // 228 KB of shared memory per SM
  if (smem > 232448) smem = 232448;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_bconv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles_per_group = (int)((1u << t.logn) / kTcM);
  const int total = tiles_per_group * a.ngroups;
  const int grid = std::min(total, std::max(1, sms * per_sm));
  TraceScope ts(t, "bconv_tc", s);
  k_bconv_tc<<<grid, kTcThreads, smem, s>>>(a, t.pc, t.logn, t.status, kpad, npad, tiles_per_group);
  note_launch();
  return cudaGetLastError();
}

// Host side: the digit table of one conversion (inputs with primes q_in, outputs
// with primes p_out, T[o][j] row-major) in the canonical layout of B (npad x kpad bf16).
std::vector<uint16_t> bconv_tc_table(const std::vector<uint32_t> &T, int n_in, const std::vector<uint32_t> &p_out) {
  const int n_out = (int)p_out.size();
  const int kpad = round16(4 * n_in), npad = round16(4 * n_out);
  std::vector<uint16_t> B((size_t)npad * kpad, 0);
  for (int o = 0; o < n_out; o++) {
    const uint32_t p = p_out[o];
    for (int j = 0; j < n_in; j++)
      for (int a = 0; a < 4; a++) {
        const uint32_t ta = (uint32_t)(((unsigned __int128)T[(size_t)o * n_in + j] << (8 * a)) % p);
        for (int b = 0; b < 4; b++) {
          const uint32_t byte = (ta >> (8 * b)) & 0xFFu;
          float f = (float)byte;
          uint32_t bits;
          memcpy(&bits, &f, 4);
          const int nn = 4 * o + b, kk = 4 * j + a;
          const size_t idx = (size_t)(nn / 8) * (kpad / 8) * 64 + (size_t)(kk / 8) * 64 + (nn % 8) * 8 + (kk % 8);
          B[idx] = (uint16_t)(bits >> 16);
        }
      }
  }
  return B;
}

}  // namespace fhe

bool fhe_tc_available() { return true; }
