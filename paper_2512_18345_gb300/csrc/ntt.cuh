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
//
// Variants (chosen per context, measured by the autotuner):
//   * on-the-fly twiddles (Section III-C cites them for the second NTT kernel):
//     the block pass's register twiddles of a run of 2^m consecutive indices are
//     formed as w_0 * psi^brv(k) from one loaded twiddle and a staged 8-entry
//     table instead of 2^m loads;
//   * single pass: one launch per limb group with a cluster of 16 CTAs (one per
//     tile); the first pass leaves its tile in shared memory and the second
//     reads its tile from the cluster's shared memory (no global round trip).
#pragma once
#include <cooperative_groups.h>

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

// Element k (0..S) of a thread's sub-transform for register slot e in a round:
// the "hi" round puts e on k's bits 7..4 (tau on 3..0), the "lo" round on bits
// 3..0; with R == 4 there is one round and k = e.
template <int R>
__device__ __forceinline__ int kmap(bool hi, int e, int tau) {
  return R == 4 ? e : (hi ? ((e << 4) | tau) : ((tau << 4) | e));
}

// dynamic shared memory of a pass: its staged twiddles (the column pass: the S - 1
// twiddles of its R stages, shared by every column; the block pass: the 240
// twiddles of its first four stages for its 16 blocks, 16 2^sigma at 16 (2^sigma - 1),
// then the 8 entries psi^brv(k), k < 8, of the on-the-fly variant)
__host__ __device__ constexpr int ntt_twiddle_smem(bool column, int S) { return (column ? S : 248) * 8; }

// Split cluster barrier (all threads of every CTA of the cluster): arrive releases this
// thread's earlier shared-memory accesses to the cluster, wait acquires the others'.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// Where a pass reads its round-0 elements and writes its results.
enum : int { SRC_GLOBAL = 0, SRC_CLUSTER = 1 };
enum : int { DST_GLOBAL = 0, DST_LOCAL = 1 };

// Number of staged twiddle entries of a pass (see ntt_twiddle_smem) plus, for on-the-fly
// twiddles, the 8 entries psi^brv(k), k < 8.
constexpr int kOtfSmall = 8;

// One pass over tile `tile` of a limb.  The single-pass kernel's transfer layouts (row r =
// index >> 8, column col = index & 255 of the 256 x 256 view of a 2^16 limb):
//   forward, after the column pass of column tile t (columns 16 t .. 16 t + 15):
//     xfer[r * 16 + (col & 15)];
//   inverse, after the block pass of row tile t (rows 16 t .. 16 t + 15):
//     xfer[(r & 15) * 256 + col];
// and the second pass reads the value of (r, col) from the CTA that owns it.
template <int LOGN, bool COLUMN, bool FWD, int PRO, int EPI, bool OTF, int SRCM, int DSTM>
__device__ __forceinline__ void ntt_pass(const Seg &sg, const KsArgs &ks, int within, int prime, const NttTables &tb,
                                         int tile, uint32_t *sm, uint2 *tws, uint32_t *xfer) {
  using G = NttGeom<LOGN, COLUMN>;
  constexpr int R = G::R, N = G::N, S0 = COLUMN ? 0 : LOGN - 8;
  const PrimeC P = tb.pc[prime];
  const uint32_t q = P.q;
  const uint2 *tw = (FWD ? tb.tw_fwd : tb.tw_inv) + (size_t)prime * N;
  const uint32_t *src = sg.src + (size_t)within * sg.src_stride * N;
  uint32_t *dst = sg.dst + (size_t)within * N;
  const int tid = threadIdx.x;

  if (COLUMN) {
    for (int i = tid; i < G::S; i += kNttThreads) tws[i] = __ldg(tw + i);
  } else {
    const int blk0 = tile * 16;
#pragma unroll
    for (int sig = 0; sig < 4; sig++) {
      const int cnt = 16 << sig;
      const uint2 *from = tw + (1 << (S0 + sig)) + (blk0 << sig);
      if (tid < cnt) tws[16 * ((1 << sig) - 1) + tid] = __ldg(from + tid);
    }
    if (OTF && tid < kOtfSmall) tws[240 + tid] = __ldg(tw + tid);
  }

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
  // round 0 is the hi round going forward (large distances first), lo going backward
  const bool hi0 = (R == 8) && FWD;

  // block pass, lo round (stages sigma = 4 + m, m = 0..3): thread (c, tau) uses the 2^m
  // consecutive twiddles 2^(S0+sigma) + ((blk0 + c) << sigma) + (tau << m) + [0, 2^m), each
  // exactly once; prefetch them into registers (tl[2^m - 1 + k]) with vector loads.
  uint2 tl[COLUMN ? 1 : 15];
  if (!COLUMN && !OTF) {
    const int blk = tile * 16 + c;
#pragma unroll
    for (int m = 0; m < 4; m++) {
      const int sig = 4 + m;
      const uint2 *from = tw + (1 << (S0 + sig)) + (blk << sig) + (tau << m);
      if (m == 0) {
        tl[0] = __ldg(from);
      } else {
#pragma unroll
        for (int k2 = 0; k2 < (1 << m) / 2; k2++) {
          const uint4 w = __ldg(reinterpret_cast<const uint4 *>(from) + k2);
          tl[(1 << m) - 1 + 2 * k2] = make_uint2(w.x, w.y);
          tl[(1 << m) - 1 + 2 * k2 + 1] = make_uint2(w.z, w.w);
        }
      }
    }
  }
  uint2 tbase[OTF && !COLUMN ? 4 : 1];
  if (!COLUMN && OTF) {
    const int blk = tile * 16 + c;
#pragma unroll
    for (int m = 0; m < 4; m++) tbase[m] = __ldg(tw + (1 << (S0 + 4 + m)) + (blk << (4 + m)) + (tau << m));
  }

  // ---- round-0 elements (prologue applied)
  uint32_t x[16];
  if constexpr (SRCM == SRC_CLUSTER) {
    static_assert(LOGN == 16, "the single-pass kernel splits a 2^16 limb into 16 tiles");
    cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
    cluster_wait();  // every CTA's first-pass tile is in its shared memory (its arrive ended pass 1)
#pragma unroll
    for (int e = 0; e < 16; e++) {
      if (FWD) {  // block pass: element (r, col) = ((16 tile + c), 16 e + tau), owned by column tile e
        const uint32_t *peer = cl.map_shared_rank(xfer, e);
        x[e] = peer[(tile * 16 + c) * 16 + tau];
      } else {  // column pass: element (16 tau + e, 16 tile + c), owned by row tile tau
        const uint32_t *peer = cl.map_shared_rank(xfer, tau);
        x[e] = peer[e * 256 + tile * 16 + c];
      }
    }
    cluster_arrive();  // this CTA's reads of the others' buffers are done (waited for at the kernel's end)
  } else if (!COLUMN && !hi0 && PRO == PRO_PLAIN) {
    // inverse block pass: a thread's 16 elements are contiguous
    const uint4 *p = reinterpret_cast<const uint4 *>(src + G::gidx(tile, c, kmap<R>(false, 0, tau)));
#pragma unroll
    for (int e4 = 0; e4 < 4; e4++) {
      const uint4 w = __ldg(p + e4);
      x[4 * e4] = w.x;
      x[4 * e4 + 1] = w.y;
      x[4 * e4 + 2] = w.z;
      x[4 * e4 + 3] = w.w;
    }
  } else {
#pragma unroll
    for (int e = 0; e < 16; e++) {
      const uint32_t j = G::gidx(tile, c, kmap<R>(hi0, e, tau));
      if (PRO == PRO_GATHER)
        x[e] = __ldg(src + galois_src(j, ks.galois_own, LOGN));
      else if (PRO == PRO_REDUCE)  // value of another prime's limb, reduced exactly mod q
        x[e] = reduce_u64(__ldg(src + j), P);
      else
        x[e] = __ldg(src + j);
    }
  }
  __syncthreads();  // staged twiddles

  // on-the-fly register twiddles: the run 2^(S0+sigma) + t0 + k (t0 = 0 mod 2^m, k < 2^m)
  // has psi^brv = psi^brv(2^(S0+sigma) + t0) psi^brv(k) (disjoint bits), so each is the
  // loaded base times a staged small twiddle, with its Shoup companion
  // floor(w 2^32 / q) = w floor(2^32 / q) + floor(w (2^32 mod q) / q) (the last quotient
  // from a Shoup estimate and one correction).
  if (!COLUMN && OTF) {
#pragma unroll
    for (int m = 0; m < 4; m++) {
      tl[(1 << m) - 1] = tbase[m];
#pragma unroll
      for (int k = 1; k < (1 << m); k++) {
        const uint2 sk = tws[240 + k];
        const uint32_t w = shoup(tbase[m].x, sk.x, sk.y, q);
        uint32_t qh = __umulhi(w, P.r32s);
        const uint32_t rem = w * P.r32 - qh * q;  // w (2^32 mod q) - qh q, in [0, 2q)
        qh += rem >= q ? 1u : 0u;
        tl[(1 << m) - 1 + k] = make_uint2(w, w * P.div32 + qh);
      }
    }
  }

#pragma unroll
  for (int rho = 0; rho < ROUNDS; rho++) {
    const bool hi = (R == 8) && (FWD ? rho == 0 : rho == 1);
    if (rho > 0) {  // exchange through shared memory between the rounds
#pragma unroll
      for (int e = 0; e < 16; e++) sm[G::addr(c, kmap<R>(!hi, e, tau))] = x[e];
      __syncthreads();
#pragma unroll
      for (int e = 0; e < 16; e++) x[e] = sm[G::addr(c, kmap<R>(hi, e, tau))];
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
      const int bit = FWD ? 3 - i : i;          // register-slot bit of this butterfly stage
      const int kbit = hi ? bit + 4 : bit;      // bit of k (pair distance 2^kbit inside the sub-transform)
      // twiddle index = base (runtime, per round and stage) + (e >> (bit + 1))
      int base;
      if (COLUMN) {
        const int s = R - 1 - kbit;  // Cooley-Tukey stage: psi^brv(2^s + (k_lo >> (kbit + 1)))
        base = (1 << s) + ((R == 8 && !hi) ? (tau << (3 - bit)) : 0);
      } else {
        const int sig = 7 - kbit;    // stage within the pass; local index (c << sig) + (k_lo >> (kbit + 1))
        base = 16 * ((1 << sig) - 1) + (c << sig);  // hi round only (sig < 4)
      }
      // the stage's 2^(3 - bit) staged twiddles are consecutive from an even base: fetch them
      // in 16-byte pairs (the block pass's lo round uses its register twiddles instead)
      constexpr int kMaxTw = 8;
      uint2 ws[kMaxTw];
      if (COLUMN || hi) {
        const int cnt = 1 << (3 - bit);
        if (cnt == 1) {
          ws[0] = tws[base];
        } else {
#pragma unroll
          for (int k2 = 0; k2 < cnt / 2; k2++) {
            const uint4 w = *reinterpret_cast<const uint4 *>(tws + base + 2 * k2);
            ws[2 * k2] = make_uint2(w.x, w.y);
            ws[2 * k2 + 1] = make_uint2(w.z, w.w);
          }
        }
      }
#pragma unroll
      for (int e = 0; e < 16; e++) {
        if (e & (1 << bit)) continue;
        const int e2 = e | (1 << bit);
        // block pass lo round: register twiddle tl[2^m - 1 + (e >> (bit + 1))], m = 3 - bit
        const uint2 W = (!COLUMN && !hi) ? tl[(1 << (3 - bit)) - 1 + (e >> (bit + 1))] : ws[e >> (bit + 1)];
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
  }

  // ---- epilogue straight from registers
  const bool hiL = (R == 8) && !FWD;  // the last round
  if constexpr (DSTM == DST_LOCAL) {  // single-pass kernel: the tile stays in shared memory (lazy values)
    static_assert(LOGN == 16, "the single-pass kernel splits a 2^16 limb into 16 tiles");
#pragma unroll
    for (int e = 0; e < 16; e++) {
      const int k = kmap<R>(hiL, e, tau);
      if (COLUMN) xfer[k * 16 + c] = x[e];  // (r, col & 15) = (k, c)
      else xfer[c * 256 + k] = x[e];         // (r & 15, col) = (c, k)
    }
    cluster_arrive();  // the tile is published; the second pass waits before reading the cluster
    return;
  }
  uint2 scale = make_uint2(0, 0);
  if (EPI == EPI_SCALE || EPI == EPI_RESCALE) scale = sg.scale ? sg.scale[within] : tb.ninv[prime];
  uint2 pinv = make_uint2(0, 0);
  if (EPI == EPI_COMBINE) pinv = ks.pinv[prime];
  const bool contiguous = !COLUMN && !hiL;  // forward block pass: 16 consecutive elements per thread
  const uint32_t j0 = G::gidx(tile, c, kmap<R>(hiL, 0, tau));
  uint32_t a[16];  // second operand of the combine / rescale epilogues
  if (EPI == EPI_RESCALE || EPI == EPI_COMBINE) {
    const uint32_t *s2 = sg.src2 + (size_t)within * N;
    if (contiguous) {
#pragma unroll
      for (int e4 = 0; e4 < 4; e4++) {
        const uint4 w = __ldg(reinterpret_cast<const uint4 *>(s2 + j0) + e4);
        a[4 * e4] = w.x;
        a[4 * e4 + 1] = w.y;
        a[4 * e4 + 2] = w.z;
        a[4 * e4 + 3] = w.w;
      }
    } else {
#pragma unroll
      for (int e = 0; e < 16; e++) a[e] = __ldg(s2 + G::gidx(tile, c, kmap<R>(hiL, e, tau)));
    }
  }
#pragma unroll
  for (int e = 0; e < 16; e++) {
    const uint32_t val = x[e];
    uint32_t o;
    if (EPI == EPI_LAZY) {
      o = val;
    } else if (EPI == EPI_PLAIN) {
      o = red2(val, q);
    } else if (EPI == EPI_SCALE) {
      o = shoup(val, scale.x, scale.y, q);
    } else if (EPI == EPI_RESCALE) {
      o = shoup(a[e] + q - red2(val, q), scale.x, scale.y, q);
    } else {  // EPI_COMBINE: a = inner product u (with P times the pass-through term folded in)
      o = shoup(a[e] + q - red2(val, q), pinv.x, pinv.y, q);
    }
    x[e] = o;
  }
  if (contiguous) {
    uint4 *p = reinterpret_cast<uint4 *>(dst + j0);
#pragma unroll
    for (int e4 = 0; e4 < 4; e4++) p[e4] = make_uint4(x[4 * e4], x[4 * e4 + 1], x[4 * e4 + 2], x[4 * e4 + 3]);
  } else {
#pragma unroll
    for (int e = 0; e < 16; e++) dst[G::gidx(tile, c, kmap<R>(hiL, e, tau))] = x[e];
  }
}

// Resident CTAs per SM asked of the register allocator for each pass (the occupancy the
// passes were measured best at: 8 for the forward column passes, 6 for the inverse column
// pass, 5 or 4 for the block passes; 6 for ModUp's forward block pass cost a register
// spill and 1.5 % of its time).
template <bool COLUMN, bool FWD, int PRO, int EPI, bool OTF>
constexpr int ntt_min_blocks() {
  if (COLUMN) return FWD ? 8 : 6;
  if (!FWD) return 5;
  return EPI == EPI_RESCALE ? 4 : 5;
}

template <int LOGN, bool COLUMN, bool FWD, int PRO, int EPI, bool OTF>
__global__ void __launch_bounds__(kNttThreads, ntt_min_blocks<COLUMN, FWD, PRO, EPI, OTF>())
    k_ntt(const __grid_constant__ SegList sl, const NttTables tb) {
  using G = NttGeom<LOGN, COLUMN>;
  constexpr int R = G::R;
  // staged twiddles: the column pass needs the S - 1 twiddles of stages 0..R-1 (shared
  // by all columns); the block pass needs, per stage sigma of its 8, the 16 2^sigma
  // twiddles of its 16 blocks, stored at 16 (2^sigma - 1).
  __shared__ uint32_t sm[R == 8 ? G::SMEM : 1];
  extern __shared__ __align__(16) uint2 tws[];  // dynamic: ntt_twiddle_smem(COLUMN, S) bytes (+ the small table)

  const int v = blockIdx.x / G::TILES, tile = blockIdx.x % G::TILES;
  int within;
  const int si = seg_find(sl, v, within);
  const Seg &sg = seg_at(sl, si);
  const KsArgs &ks = item_ks(sl, sg);
  ntt_pass<LOGN, COLUMN, FWD, PRO, EPI, OTF, SRC_GLOBAL, DST_GLOBAL>(sg, ks, within, sg.prime + within, tb, tile, sm,
                                                                     tws, nullptr);
}

// Both passes of a 2^16-point transform in one launch: a cluster of 16 CTAs per limb, CTA
// t does the first pass on tile t into its shared memory, the cluster synchronises, and CTA
// t does the second pass on tile t reading from the 16 CTAs' shared memory.  `first` and
// `second` enumerate the same limbs (same segment sizes and primes): the first pass's
// source and prologue come from `first`, the second pass's destination and epilogue from
// `second`.
template <bool FWD, int PRO, int EPI, bool OTF>
__global__ void __cluster_dims__(16, 1, 1) __launch_bounds__(kNttThreads)
    k_ntt1(const __grid_constant__ SegList first, const __grid_constant__ SegList second, const NttTables tb) {
  constexpr int LOGN = 16;
  using GB = NttGeom<LOGN, false>;
  __shared__ uint32_t sm[GB::SMEM];
  __shared__ uint32_t xfer[kTile];
  extern __shared__ __align__(16) uint2 tws[];  // the larger of the two passes' staged twiddles
  const int v = blockIdx.x / 16, tile = blockIdx.x % 16;
  int w1, w2;
  const Seg &s1 = seg_at(first, seg_find(first, v, w1));
  const Seg &s2 = seg_at(second, seg_find(second, v, w2));
  const KsArgs &k1 = item_ks(first, s1);
  const KsArgs &k2 = item_ks(second, s2);
  const int prime = s1.prime + w1;
  // forward: column pass then block pass; inverse: block pass then column pass
  // (the passes pair a split cluster barrier: pass 1 arrives after publishing its tile and
  // pass 2 waits just before reading the cluster, so pass 2's twiddle loads overlap the
  // wait; pass 2 arrives after its reads and the CTA waits before exiting, so no CTA's
  // shared memory goes away while another reads it)
  ntt_pass<LOGN, FWD, FWD, PRO, EPI_LAZY, OTF, SRC_GLOBAL, DST_LOCAL>(s1, k1, w1, prime, tb, tile, sm, tws, xfer);
  __syncthreads();  // pass 1's last reads of the staged twiddles come before pass 2 restages them
  ntt_pass<LOGN, !FWD, FWD, PRO_PLAIN, EPI, OTF, SRC_CLUSTER, DST_GLOBAL>(s2, k2, w2, prime, tb, tile, sm, tws, xfer);
  cluster_wait();
}

// Grid-wide barrier of a cooperative launch (every CTA resident): thread 0 of each CTA
// arrives on the launch's own zeroed counter and waits, bounded, until every CTA has; false
// when the wait expired.  Writes before the barrier are visible to every CTA after it.
__device__ __forceinline__ bool grid_barrier_bounded(unsigned int *ctr, unsigned int nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1u);
    int ok = 0;
    for (uint32_t it = 0; it < (1u << 22) && !ok; it++) {
      unsigned int v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
      if (v >= nblocks) ok = 1;
      else __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Both passes of a 2^16-point transform in one persistent, cooperative launch (a
// measured alternative to the two launches and to the cluster kernel): the CTAs walk the
// first pass's tiles exactly as the first launch's blocks would, meet at a grid-wide
// barrier, then walk the second pass's tiles.  The passes, their segments and their
// global round trip are the two-launch form's, so the results are identical; what goes is
// the second launch's ramp and the first one's tail.  An expired barrier sets status bit 4
// and skips the second pass.
template <bool FWD, int PRO, int EPI>
__global__ void __launch_bounds__(kNttThreads)
    k_nttp(const __grid_constant__ SegList first, const __grid_constant__ SegList second, const NttTables tb,
           unsigned int *ctr, unsigned int *status) {
  constexpr int LOGN = 16;
  using GB = NttGeom<LOGN, false>;
  __shared__ uint32_t sm[GB::SMEM];  // both passes' tile (R = 8 on both sides at N = 2^16)
  extern __shared__ __align__(16) uint2 tws[];     // the larger of the two passes' staged twiddles
  const int units = first.total * 16;
  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    int w;
    const Seg &sg = seg_at(first, seg_find(first, u >> 4, w));
    ntt_pass<LOGN, FWD, FWD, PRO, EPI_LAZY, false, SRC_GLOBAL, DST_GLOBAL>(sg, item_ks(first, sg), w, sg.prime + w, tb,
                                                                         u & 15, sm, tws, nullptr);
    __syncthreads();  // the tile and the staged twiddles are reused by the next unit
  }
  if (!grid_barrier_bounded(ctr, gridDim.x)) {
    if (threadIdx.x == 0) atomicOr(status, 16u);
    return;
  }
  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    int w;
    const Seg &sg = seg_at(second, seg_find(second, u >> 4, w));
    ntt_pass<LOGN, !FWD, FWD, PRO_PLAIN, EPI, false, SRC_GLOBAL, DST_GLOBAL>(sg, item_ks(second, sg), w, sg.prime + w,
                                                                           tb, u & 15, sm, tws, nullptr);
    __syncthreads();
  }
}

}  // namespace fhe
