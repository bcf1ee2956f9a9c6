// Base conversion on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// BConv is a dense contraction (Section II-B: Red(T . a)).  sm_103a has no
// integer tcgen05 MMA (.kind::i8 does not assemble for it), so the exact
// integer product is built from f16 operands that hold small integers:
//   y_j = sum_a y_{j,a} 2^(8a)          (4 bytes of the 31-bit input)
//   T'_a[o][j] = (2^(8a) T[o][j]) mod p_o = sum_b D_{a,b}[o][j] 2^(8b)
//   sum_j y_j T[o][j] = sum_b 2^(8b) S_b[o]  (mod p_o),
//   S_b[o] = sum_{(j,a)} y_{j,a} D_{a,b}[o][j]  <  32 * 255^2 < 2^21  (n_in <= 8).
// The MMA has M = 128 coefficients, N = 4 n_out ((output, weight-byte) pairs)
// and K = 48: 32 data slots (k = 4 j + a), 4 offset slots, 12 zero slots.
//
// Operand encoding.  The f16 pattern 0x6400 | b is the integer 1024 + b, so
// a byte permute of y_j against 0x64006400 yields two A operands at once.  The
// offset slots hold A = 1024 and B pieces (each <= 2048, exact in f16) summing
// to 8192 - sum_k D[n][k], so every accumulator ends at exactly
//   sum_k (1024 + y_k) D_k + 1024 (8192 - sum_k D_k) = 2^23 + S_b.
// Every A and B entry is a nonnegative integer, so every partial sum of the
// accumulation lies in [0, 2^23 + S_b] with 2^23 + S_b < 2^24: the fp32
// accumulation in tensor memory is exact in any order, and the accumulator's
// bit pattern is 0x4B000000 + S_b (no conversion instruction needed).
// The epilogue forms lo = S_0 + 2^8 S_1 and hi = S_2 + 2^8 S_3 (both < 2^30)
// and reduces lo + 2^16 hi modulo p_o once: bit-identical to the CUDA-core path.
//
// Digits of 9..12 limbs (the paper's alpha = 12) use K = 64: 48 data slots and 8
// offset slots whose B pieces may be negative (each in [-2048, 2048], summing to
// 8192 - the row sum, which now reaches 48 * 255 = 12240).  The accumulator still
// ends at 2^23 + S_b with S_b < 48 * 255^2 < 2^22; every partial sum lies between the
// sum of the negative terms (> -2^22 * 1.0) and the sum of the positive ones
// (< 1024 * 12240 + 2^22 < 2^24), so the fp32 accumulation stays exact in any order.
// The epilogue's lo, hi < 2^30 + 2^22, so one conditional subtraction after adding
// 2^16 hi mod p suffices for primes above 2^30 + 2^23.
//
// A 128-coefficient tile of one group is one M = 128 MMA of K / 16 steps;
// persistent CTAs of 256 threads walk the tiles (see k_bconv_tc).  Operands sit
// in shared memory in the canonical K-major layout without swizzle: 8 x 16-byte
// core matrices, core matrices adjacent along K 128 bytes apart (leading byte
// offset), 8-row groups (K / 8) x 128 bytes apart (stride byte offset).
#include <algorithm>
#include <cstring>

#include "async.cuh"
#include "ctx.h"
#include "internal.h"

namespace fhe {

// shared memory matrix descriptor: start address, leading / stride byte offsets,
// descriptor version 1 (bits 46..48), no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::f16 with f16 A and B (both K-major), fp32 D, shape M x N
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// 32 lanes x 16 columns of 32-bit words from tensor memory (one value per column per thread)
__device__ __forceinline__ void tmem_ld16(uint32_t *r, uint32_t addr) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

constexpr int kTcThreads = 256;  // 8 warps: warps w and w + 4 share accumulator lanes 32 (w % 4)..

struct TcOut {  // per output prime of the current group, read by whole warps (one 16-byte broadcast)
  uint32_t q, w16s, div32, off;  // prime, Shoup companion of 2^16, floor(2^32 / q), limb offset * N
};

// One warp's share of a tile's epilogue: outputs [o_beg, o_end) of the accumulator at tbase
// (columns 4 o + b hold 2^23 + S_b[o]) for coefficient n, four outputs (one 16-column load)
// at a time with no predicated slots except in a last partial group.  lo = S_0 + 2^8 S_1 and
// hi = S_2 + 2^8 S_3 (the 0x4B000000 of each accumulator cancels modulo 2^32), then
// lo + (2^16 hi mod p) reduced once.  LAZY: the value is left in [0, 2p) (the conversions
// inside the key-switching pipeline feed a forward NTT, which takes such inputs).
template <bool LAZY>
__device__ __forceinline__ void tc_out1(const uint32_t *r, const TcOut &t, uint32_t *gn, bool big_primes) {
  const uint32_t lo = r[1] * 256u + r[0] - 0x4B000000u;
  const uint32_t hi = r[3] * 256u + r[2] - 0x4B000000u;
  const uint32_t sum = lo + red2(shoup_lazy(hi, 65536u, t.w16s, t.q), t.q);  // < 2^30 + 2^22 + q
  uint32_t v;
  if (big_primes) v = LAZY ? sum : red2(sum, t.q);
  else {
    v = shoup_lazy(sum, 1u, t.div32, t.q);
    if (!LAZY) v = red2(v, t.q);
  }
  gn[t.off] = v;
}
template <bool LAZY>
__device__ __forceinline__ void tc_reduce_outputs(uint32_t tbase, int o_beg, int o_end, const TcOut *sO, uint32_t *gn,
                                                  bool big_primes) {
  for (int o0 = o_beg; o0 < o_end; o0 += 4) {
    uint32_t rr[16];
    tmem_ld16(rr, tbase + (uint32_t)(4 * o0));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (o0 + 4 <= o_end) {
#pragma unroll
      for (int i = 0; i < 4; i++) tc_out1<LAZY>(rr + 4 * i, sO[o0 + i], gn, big_primes);
    } else {
#pragma unroll
      for (int i = 0; i < 3; i++)
        if (o0 + i < o_end) tc_out1<LAZY>(rr + 4 * i, sO[o0 + i], gn, big_primes);
    }
  }
}

// Persistent: a CTA walks tiles (group, 128-coefficient block) in group-major
// order, reloading the digit table only when the group changes; tensor memory
// is allocated once per CTA.  Per tile: every thread permutes the bytes of two
// input pairs into A, thread 0 issues the MMAs and commits to the mbarrier
// (phase = tile parity), all wait (bounded), then each warp reads its lane
// quarter for half of the outputs and writes the reduced results.
template <int KT>
__global__ void __launch_bounds__(kTcThreads, 4) k_bconv_tc(const __grid_constant__ BconvArgs a, const PrimeC *pc,
                                                         int logn, unsigned int *status, int npad_max,
                                                         int tiles_per_group) {
  static_assert(KT == kTcK || KT == kTcK12, "K is 48 or 64");
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  constexpr uint32_t kRowBytes = KT * 2;             // one A / B row: K f16
  constexpr uint32_t kSbo = (KT / 8) * 128u;         // 8-row group stride
  constexpr int kDataChunks = KT == kTcK ? 4 : 6;    // 8-slot K chunks holding inputs (two each)
  constexpr int kNch = kDataChunks / 2;              // data chunks built by each thread
  constexpr uint32_t kBigPrime = KT == kTcK ? (1u << 30) : (1u << 30) + (1u << 23);
  uint8_t *sA = smem;
  uint8_t *sB = smem + kTcM * kRowBytes;
  TcOut *sO = reinterpret_cast<TcOut *>(sB + (size_t)npad_max * kRowBytes);
  uint64_t *bar = reinterpret_cast<uint64_t *>(sO + 64);
  uint32_t *s_taddr = reinterpret_cast<uint32_t *>(bar + 1);
  const uint32_t ncols = npad_max <= 32 ? 32u : npad_max <= 64 ? 64u : npad_max <= 128 ? 128u : 256u;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_taddr)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) mbar_init(bar, 1);
  // constant K chunks of A (written once): K = 48: chunk 4 = four offset slots (1024) and
  // four zero slots, chunk 5 = zero slots; K = 64: chunk 6 = eight offset slots, chunk 7 = zero
  if (tid < kTcM) {
    uint8_t *row = sA + (tid >> 3) * kSbo + (tid & 7) * 16;
    if (KT == kTcK)
      *reinterpret_cast<uint4 *>(row + kDataChunks * 128) = make_uint4(0x64006400u, 0x64006400u, 0u, 0u);
    else
      *reinterpret_cast<uint4 *>(row + kDataChunks * 128) =
          make_uint4(0x64006400u, 0x64006400u, 0x64006400u, 0x64006400u);
    *reinterpret_cast<uint4 *>(row + (kDataChunks + 1) * 128) = make_uint4(0u, 0u, 0u, 0u);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *s_taddr;

  const size_t N = (size_t)1 << logn;
  const int total = tiles_per_group * a.ngroups;
  const int ltg = __ffs(tiles_per_group) - 1;  // tiles_per_group = N / 128, a power of two
  const int per_cta = (total + gridDim.x - 1) / gridDim.x;
  const int t0 = blockIdx.x * per_cta, t1 = min(total, t0 + per_cta);
  int cur_group = -1, npad = 0, n_in = 0, n_out = 0;
  const BconvGroup *gp = nullptr;
  uint32_t phase = 0;
  bool ok = true;
  const int r = tid & (kTcM - 1);  // A row built by this thread
  const int kc0 = tid >> 7;        // its K chunks: kc0, kc0 + 2 (, kc0 + 4) (inputs 2 kc, 2 kc + 1)
  uint32_t y[2 * kNch];
  auto load_inputs = [&](const BconvGroup *g, int nin, size_t m0) {
#pragma unroll
    for (int h = 0; h < 2 * kNch; h++) {
      const int j = 2 * (kc0 + 2 * (h >> 1)) + (h & 1);
      y[h] = j < nin ? __ldg(g->in + (size_t)j * N + m0 + r) : 0u;
    }
  };
#pragma unroll
  for (int h = 0; h < 2 * kNch; h++) y[h] = 0u;
  bool prefetched = false;  // y holds the current tile's inputs
  bool big_primes = true;   // the current group's output primes all exceed 2^30
  for (int tile = t0; tile < t1 && ok; tile++) {
    const int grp = tile >> ltg;
    const size_t n0 = (size_t)(tile & (tiles_per_group - 1)) * kTcM;
    if (grp != cur_group) {  // load this group's table and output constants
      cur_group = grp;
      gp = a.dev ? &a.dev[grp] : &a.g[grp];
      npad = gp->npad;
      n_in = gp->n_in;
      n_out = gp->n_out;
      const uint4 *src = reinterpret_cast<const uint4 *>(gp->Btc);
      uint4 *dst = reinterpret_cast<uint4 *>(sB);
      const int n16 = npad * (int)kRowBytes / 16;
      for (int i = tid; i < n16; i += kTcThreads) dst[i] = __ldg(src + i);
      bool big = true;  // every output prime above kBigPrime: one conditional subtraction suffices
      for (int o = tid; o < n_out; o += kTcThreads) {
        const int2 m = gp->omap[o];
        const PrimeC p = pc[m.y];
        TcOut t;
        t.q = p.q;
        t.w16s = (uint32_t)(((uint64_t)65536u << 32) / p.q);
        t.div32 = p.div32;
        t.off = (uint32_t)m.x << logn;
        sO[o] = t;
        big = big && p.q > kBigPrime;
      }
      big_primes = __syncthreads_and(big ? 1 : 0) != 0;
    }
    // A: row r = coefficient n0 + r; chunk kc holds inputs 2 kc, 2 kc + 1 as the f16
    // values 1024 + byte (byte permutes against 0x64006400), absent inputs as 1024.
    // The inputs were loaded during the previous tile (prefetch), except for the
    // first tile of a group.
    {
      if (!prefetched) load_inputs(gp, n_in, n0);
      uint8_t *row = sA + (r >> 3) * kSbo + (r & 7) * 16;
#pragma unroll
      for (int i = 0; i < kNch; i++) {
        const uint32_t y0 = y[2 * i], y1 = y[2 * i + 1];
        *reinterpret_cast<uint4 *>(row + (kc0 + 2 * i) * 128) =
            make_uint4(__byte_perm(y0, 0x64006400u, 0x7150), __byte_perm(y0, 0x64006400u, 0x7352),
                       __byte_perm(y1, 0x64006400u, 0x7150), __byte_perm(y1, 0x64006400u, 0x7352));
      }
    }
    // prefetch the next tile's inputs when it belongs to the same group
    prefetched = tile + 1 < t1 && ((tile + 1) >> ltg) == grp;
    if (prefetched) load_inputs(gp, n_in, (size_t)((tile + 1) & (tiles_per_group - 1)) * kTcM);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      const uint32_t aaddr = smem_addr(sA), baddr = smem_addr(sB);
      const uint32_t idesc = idesc_f16(kTcM, npad);
#pragma unroll
      for (int kk = 0; kk < KT / 16; kk++) {
        const uint64_t ad = smem_desc(aaddr + kk * 256u, 128u, kSbo);
        const uint64_t bd = smem_desc(baddr + kk * 256u, 128u, kSbo);
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
    // every thread waits (bounded) for the MMA itself, made warp-uniform for the
    // warp-synchronous tensor-memory loads; the CTA-wide verdict rides on the tile's
    // closing barrier
    const bool w = __all_sync(0xffffffffu, mbar_wait_bounded(bar, phase));
    phase ^= 1u;
    tc_fence_after();
    if (w) {
      // epilogue: warp w reads lanes 32 (w % 4).. = coefficients n0 + 32 (w % 4) + lane; warps
      // w < 4 take outputs [0, H), the others [H, n_out) (H a multiple of 4), eight outputs
      // (two 16-column loads, one wait) at a time; columns 4 o + b hold 2^23 + S_b[o]
      const int q4 = warp & 3;
      const uint32_t n = (uint32_t)(n0 + (size_t)q4 * 32 + (tid & 31));
      const uint32_t tbase = taddr + ((uint32_t)(q4 * 32) << 16);
      const int H = ((n_out + 1) / 2 + 3) & ~3;
      const int o_end = (warp >> 2) ? n_out : min(H, n_out);
      uint32_t *gn = gp->out + n;  // this thread's coefficient of the group's output limb 0
      if (a.lazy) tc_reduce_outputs<true>(tbase, (warp >> 2) ? H : 0, o_end, sO, gn, big_primes);
      else tc_reduce_outputs<false>(tbase, (warp >> 2) ? H : 0, o_end, sO, gn, big_primes);
    } else {
      if ((tid & 31) == 0) atomicOr(status, 1u);  // expired wait: report, give the MMA a second bounded chance
      mbar_wait_bounded(bar, phase ^ 1u);
    }
    tc_fence_before();
    ok = __syncthreads_and(w ? 1 : 0) != 0;  // A, B and the accumulator are reused by the next tile
  }
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
  }
}

// Pipelined form (kernel shape bconv_tc_pipeline): two A buffers and two accumulators per
// CTA, so that tile t's MMA runs while the CTA reduces tile t - 1's accumulator.  Per
// iteration: build A(t) (inputs prefetched one tile ahead), one barrier, thread 0 issues
// MMA(t) into accumulator t & 1 and commits to mbarrier t & 1, every thread then waits
// (bounded) for MMA(t - 1) and runs its epilogue, one barrier (which also carries the
// CTA-wide verdict of the waits).  A group change first drains the pending epilogue.  The
// arithmetic is the unpipelined kernel's exactly.  Tensor memory: 2 x ncols per CTA, so at
// most two CTAs per SM for outputs of more than 16 limbs.
template <int KT>
__global__ void __launch_bounds__(kTcThreads, 2) k_bconv_tc_pipe(const __grid_constant__ BconvArgs a, const PrimeC *pc,
                                                              int logn, unsigned int *status, int npad_max,
                                                              int tiles_per_group) {
  static_assert(KT == kTcK || KT == kTcK12, "K is 48 or 64");
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  constexpr uint32_t kRowBytes = KT * 2;
  constexpr uint32_t kSbo = (KT / 8) * 128u;
  constexpr int kDataChunks = KT == kTcK ? 4 : 6;
  constexpr int kNch = kDataChunks / 2;
  constexpr uint32_t kBigPrime = KT == kTcK ? (1u << 30) : (1u << 30) + (1u << 23);
  constexpr uint32_t kAbytes = kTcM * kRowBytes;
  uint8_t *sA = smem;  // two buffers
  uint8_t *sB = smem + 2 * kAbytes;
  TcOut *sO = reinterpret_cast<TcOut *>(sB + (size_t)npad_max * kRowBytes);
  uint64_t *bar = reinterpret_cast<uint64_t *>(sO + 64);  // two
  uint32_t *s_taddr = reinterpret_cast<uint32_t *>(bar + 2);
  const uint32_t ncols = npad_max <= 32 ? 32u : npad_max <= 64 ? 64u : npad_max <= 128 ? 128u : 256u;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_taddr)),
                 "r"(2 * ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
  }
  if (tid < kTcM)  // the constant K chunks of both A buffers
    for (int b = 0; b < 2; b++) {
      uint8_t *row = sA + b * kAbytes + (tid >> 3) * kSbo + (tid & 7) * 16;
      if (KT == kTcK)
        *reinterpret_cast<uint4 *>(row + kDataChunks * 128) = make_uint4(0x64006400u, 0x64006400u, 0u, 0u);
      else
        *reinterpret_cast<uint4 *>(row + kDataChunks * 128) =
            make_uint4(0x64006400u, 0x64006400u, 0x64006400u, 0x64006400u);
      *reinterpret_cast<uint4 *>(row + (kDataChunks + 1) * 128) = make_uint4(0u, 0u, 0u, 0u);
    }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr0 = *s_taddr;

  const size_t N = (size_t)1 << logn;
  const int total = tiles_per_group * a.ngroups;
  const int ltg = __ffs(tiles_per_group) - 1;  // tiles_per_group = N / 128, a power of two
  const int per_cta = (total + gridDim.x - 1) / gridDim.x;
  const int t0 = blockIdx.x * per_cta, t1 = min(total, t0 + per_cta);
  int cur_group = -1, n_in = 0, n_out = 0;
  const BconvGroup *gp = nullptr;
  uint32_t ph = 0u;  // bit b: the phase the next wait on bar[b] expects
  bool ok = true;
  const int r = tid & (kTcM - 1);
  const int kc0 = tid >> 7;
  uint32_t y[2 * kNch];
  auto load_inputs = [&](const BconvGroup *g, int nin, size_t m0) {
#pragma unroll
    for (int h = 0; h < 2 * kNch; h++) {
      const int j = 2 * (kc0 + 2 * (h >> 1)) + (h & 1);
      y[h] = j < nin ? __ldg(g->in + (size_t)j * N + m0 + r) : 0u;
    }
  };
#pragma unroll
  for (int h = 0; h < 2 * kNch; h++) y[h] = 0u;
  bool prefetched = false;
  bool big_primes = true;
  int pending = -1;  // tile whose MMA is in flight and whose epilogue has not run
  // epilogue of tile p (accumulator p & 1): the unpipelined kernel's
  auto epilogue = [&](int p) {
    const int b = p & 1;
    const bool w = __all_sync(0xffffffffu, mbar_wait_bounded(&bar[b], (ph >> b) & 1u));
    ph ^= 1u << b;
    if (!w) {
      ok = false;
      if ((tid & 31) == 0) atomicOr(status, 1u);
      return;
    }
    tc_fence_after();
    const size_t n0 = (size_t)(p & (tiles_per_group - 1)) * kTcM;
    const int q4 = warp & 3;
    const uint32_t n = (uint32_t)(n0 + (size_t)q4 * 32 + (tid & 31));
    const uint32_t tbase = taddr0 + (uint32_t)b * ncols + ((uint32_t)(q4 * 32) << 16);
    const int H = ((n_out + 1) / 2 + 3) & ~3;
    const int o_end = (warp >> 2) ? n_out : min(H, n_out);
    uint32_t *gn = gp->out + n;
    if (a.lazy) tc_reduce_outputs<true>(tbase, (warp >> 2) ? H : 0, o_end, sO, gn, big_primes);
    else tc_reduce_outputs<false>(tbase, (warp >> 2) ? H : 0, o_end, sO, gn, big_primes);
  };
  for (int tile = t0; tile < t1 && ok; tile++) {
    const int grp = tile >> ltg;
    const size_t n0 = (size_t)(tile & (tiles_per_group - 1)) * kTcM;
    if (grp != cur_group) {
      if (pending >= 0) {  // drain: the table and output constants are about to change
        epilogue(pending);
        pending = -1;
        tc_fence_before();
        ok = __syncthreads_and(ok ? 1 : 0) != 0;
        if (!ok) break;
      }
      cur_group = grp;
      gp = a.dev ? &a.dev[grp] : &a.g[grp];
      n_in = gp->n_in;
      n_out = gp->n_out;
      const uint4 *src = reinterpret_cast<const uint4 *>(gp->Btc);
      uint4 *dst = reinterpret_cast<uint4 *>(sB);
      const int n16 = gp->npad * (int)kRowBytes / 16;
      for (int i = tid; i < n16; i += kTcThreads) dst[i] = __ldg(src + i);
      bool big = true;
      for (int o = tid; o < n_out; o += kTcThreads) {
        const int2 m = gp->omap[o];
        const PrimeC pr = pc[m.y];
        TcOut t;
        t.q = pr.q;
        t.w16s = (uint32_t)(((uint64_t)65536u << 32) / pr.q);
        t.div32 = pr.div32;
        t.off = (uint32_t)m.x << logn;
        sO[o] = t;
        big = big && pr.q > kBigPrime;
      }
      big_primes = __syncthreads_and(big ? 1 : 0) != 0;
    }
    uint8_t *Ab = sA + (tile & 1) * kAbytes;
    {
      if (!prefetched) load_inputs(gp, n_in, n0);
      uint8_t *row = Ab + (r >> 3) * kSbo + (r & 7) * 16;
#pragma unroll
      for (int i = 0; i < kNch; i++) {
        const uint32_t y0 = y[2 * i], y1 = y[2 * i + 1];
        *reinterpret_cast<uint4 *>(row + (kc0 + 2 * i) * 128) =
            make_uint4(__byte_perm(y0, 0x64006400u, 0x7150), __byte_perm(y0, 0x64006400u, 0x7352),
                       __byte_perm(y1, 0x64006400u, 0x7150), __byte_perm(y1, 0x64006400u, 0x7352));
      }
    }
    prefetched = tile + 1 < t1 && ((tile + 1) >> ltg) == grp;
    if (prefetched) load_inputs(gp, n_in, (size_t)((tile + 1) & (tiles_per_group - 1)) * kTcM);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      const uint32_t aaddr = smem_addr(Ab), baddr = smem_addr(sB);
      const uint32_t idesc = idesc_f16(kTcM, gp->npad);
      const uint32_t tacc = taddr0 + (uint32_t)(tile & 1) * ncols;
#pragma unroll
      for (int kk = 0; kk < KT / 16; kk++) {
        const uint64_t ad = smem_desc(aaddr + kk * 256u, 128u, kSbo);
        const uint64_t bd = smem_desc(baddr + kk * 256u, 128u, kSbo);
        const uint32_t acc = kk > 0 ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tacc),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_addr(&bar[tile & 1]))
                   : "memory");
    }
    if (pending >= 0) epilogue(pending);
    pending = tile;
    tc_fence_before();
    ok = __syncthreads_and(ok ? 1 : 0) != 0;  // A and the accumulator of tile - 1 are free
  }
  if (ok && pending >= 0) epilogue(pending);
  if (!ok) {  // give the MMAs in flight a second bounded chance before the memory goes away
    mbar_wait_bounded(&bar[0], ph & 1u);
    mbar_wait_bounded(&bar[1], (ph >> 1) & 1u);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr0), "r"(2 * ncols) : "memory");
  }
}

template <int KT>
static cudaError_t bconv_tc_go(const DevTables &t, const BconvArgs &a, int max_out, cudaStream_t s) {
  const int npad = tc_npad(max_out);
  const int ncols = npad <= 32 ? 32 : npad <= 64 ? 64 : npad <= 128 ? 128 : 256;
  // operands, output constants, barrier; at least enough shared memory that no
  // more CTAs fit on an SM than its 512 tensor-memory columns hold
  const int need = kTcM * KT * 2 + npad * KT * 2 + 64 * (int)sizeof(TcOut) + 64;
  // resident CTAs per SM: what the 512 tensor-memory columns hold, capped by the context's shape
  const int per_sm = std::max(1, std::min(std::min(512 / ncols, 2048 / kTcThreads), t.bconv_tc_ctas));
  int smem = std::max(need, 233472 / (per_sm + 1) + 1024);  // 228 KB of shared memory per SM
  if (smem > 232448) smem = 232448;
  static PerDeviceOnce configured;
  const cudaError_t ce = configured.run(
      [] { return cudaFuncSetAttribute(k_bconv_tc<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448); });
  if (ce != cudaSuccess) return ce;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles_per_group = (int)((1u << t.logn) / kTcM);
  const int total = tiles_per_group * a.ngroups;
  TraceScope ts(t, "bconv_tc", s);
  if (t.bconv_tc_pipe) {
    // two accumulators per CTA: what the 512 tensor-memory columns hold, within the shape's cap
    const int per_sm2 = std::max(1, std::min(std::min(256 / ncols, 2048 / kTcThreads), t.bconv_tc_ctas));
    const int need2 = 2 * kTcM * KT * 2 + npad * KT * 2 + 64 * (int)sizeof(TcOut) + 64;
    int smem2 = std::max(need2, 233472 / (per_sm2 + 1) + 1024);
    if (smem2 > 232448) smem2 = 232448;
    static PerDeviceOnce configured2;
    const cudaError_t ce2 = configured2.run(
        [] { return cudaFuncSetAttribute(k_bconv_tc_pipe<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448); });
    if (ce2 != cudaSuccess) return ce2;
    const int grid2 = std::min(total, std::max(1, sms * per_sm2));
    k_bconv_tc_pipe<KT><<<grid2, kTcThreads, smem2, s>>>(a, t.pc, t.logn, t.status, npad, tiles_per_group);
  } else {
    const int grid = std::min(total, std::max(1, sms * per_sm));
    k_bconv_tc<KT><<<grid, kTcThreads, smem, s>>>(a, t.pc, t.logn, t.status, npad, tiles_per_group);
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bconv_tc(const DevTables &t, const BconvArgs &a, int max_in, int max_out, cudaStream_t s, int kt) {
  if (a.ngroups == 0) return cudaSuccess;
  if (max_out > 64) return cudaErrorInvalidValue;
  if (kt == kTcK && max_in <= kTcMaxIn) return bconv_tc_go<kTcK>(t, a, max_out, s);
  if (kt == kTcK12 && max_in <= kTcMaxIn12) return bconv_tc_go<kTcK12>(t, a, max_out, s);
  return cudaErrorInvalidValue;
}

// exact f16 bit pattern of an integer -2048 <= v <= 2048
static uint16_t f16_int(int v) {
  if (v == 0) return 0;
  const uint16_t sign = v < 0 ? 0x8000u : 0u;
  const uint32_t m = (uint32_t)(v < 0 ? -v : v);
  const int e = 31 - __builtin_clz(m);
  const uint32_t mant = e <= 10 ? (m << (10 - e)) & 0x3FFu : (m >> (e - 10)) & 0x3FFu;
  return (uint16_t)(sign | ((uint32_t)(e + 15) << 10) | mant);
}

// Host side: the digit table of one conversion (inputs with primes q_in, outputs
// with primes p_out, T[o][j] row-major) in the canonical layout of B
// (tc_npad(n_out) x K f16): row 4 o + b, column 4 j + a holds byte b of
// (2^(8a) T[o][j]) mod p_o; the offset columns (32..35 for K = 48, 48..51 for
// K = 64) hold pieces of 8192 - (the row sum of the data columns): nonnegative and
// <= 2048 for K = 48 (row sums <= 32 * 255), in [-2048, 2048] for K = 64; every
// other entry is zero.
std::vector<uint16_t> bconv_tc_table(const std::vector<uint32_t> &T, int n_in, const std::vector<uint32_t> &p_out,
                                     int kt) {
  const int n_out = (int)p_out.size();
  const int npad = tc_npad(n_out);
  const int data = kt == kTcK ? 32 : 48;
  std::vector<uint16_t> B((size_t)npad * kt, 0);
  if (n_in > data / 4) return B;  // callers check n_in against the chosen K
  auto at = [&](int nn, int kk) -> uint16_t & {
    return B[(size_t)(nn / 8) * (kt / 8) * 64 + (size_t)(kk / 8) * 64 + (nn % 8) * 8 + (kk % 8)];
  };
  for (int o = 0; o < n_out; o++) {
    const uint32_t p = p_out[o];
    int rowsum[4] = {0, 0, 0, 0};
    for (int j = 0; j < n_in; j++)
      for (int a = 0; a < 4; a++) {
        const uint32_t ta = (uint32_t)(((unsigned __int128)T[(size_t)o * n_in + j] << (8 * a)) % p);
        for (int b = 0; b < 4; b++) {
          const int byte = (int)((ta >> (8 * b)) & 0xFFu);
          at(4 * o + b, 4 * j + a) = f16_int(byte);
          rowsum[b] += byte;
        }
      }
    for (int b = 0; b < 4; b++) {
      int rest = 8192 - rowsum[b];  // K = 48: >= 8192 - 8160; K = 64: >= 8192 - 12240
      for (int e = 0; e < 4; e++) {
        const int piece = std::max(-2048, std::min(rest, 2048));
        at(4 * o + b, data + e) = f16_int(piece);
        rest -= piece;
      }
    }
  }
  return B;
}

}  // namespace fhe

bool fhe_tc_available() { return true; }
