// Streaming NTT passes: the column and block passes of ntt.cuh as persistent
// kernels fed by a producer warp (Section III-B: the transforms' per-kernel
// utilisation; Section III-C: their twiddles).
//
// The arithmetic is the one of ntt_pass (same butterflies, same lazy [0, 2q)
// ranges, same twiddle tables, same rounds); what changes is how tiles and
// twiddles reach the registers:
//   * a CTA walks a contiguous range of units (one 4096-element tile of one
//     limb each); one producer warp copies each unit's tile into a ring of
//     shared-memory stages with 16-byte cp.async copies, up to `stages` units
//     ahead, and signals a stage's full mbarrier when the copies land;
//   * eight consumer warps read a tile from its stage, run the two radix-16
//     rounds with the exchange done in place in the stage, release the stage on
//     its empty mbarrier and write the results from registers;
//   * the hi round's twiddles (15 per prime in the column pass, 15 per block in
//     the block pass) travel with the tile in its stage; each consumer thread
//     keeps the 15 lo-round twiddles its butterflies use in registers and
//     reloads them only when the unit's prime (column pass) or prime and tile
//     (block pass) changes.  Units are ordered so that this is rare: the
//     column pass takes a limb's 16 tiles in a row; the block pass takes runs
//     of kNbRun limbs per tile, and batched plans list their limbs grouped by
//     prime, so that a run shares one prime;
//   * in the block pass a 256-element block belongs to one half-warp, so its
//     exchange needs only the warp's own synchronisation; the column pass
//     exchanges across the CTA's consumer warps with one named barrier.
// Stage layouts (32-bit words, 16-byte chunks so that cp.async can place them):
//   column tile, row k (16 columns): k * 16 + 16 (k >> 4) + column;
//   block tile, block c, row r = k >> 4 of 16 elements, chunk m = (k >> 2) & 3:
//     c * 272 + 16 r + 4 (m ^ ((r >> 1) & 3)) + (k & 3),
// which keep the round reads free of bank conflicts (scalar reads of a row,
// 16-byte reads of a chunk) for both directions; then the hi-round twiddles
// (w, floor(w 2^32 / q)) pairs: the column pass's psi^brv(i), i < 16; the block
// pass's runs psi^brv(2^(8 + m) + (16 tile << m) + i), i < 16 2^m, at 16 (2^m - 1).
#pragma once
#include "async.cuh"
#include "ntt.cuh"

namespace fhe {

constexpr int kNbConsumers = kNttThreads;            // 8 consumer warps
constexpr int kNbThreads = kNbConsumers + 32;        // + one producer warp
constexpr int kNbDataWords = kTile + 256;            // both padded tile layouts
constexpr int kNbStageWords = kNbDataWords + 2 * 256;  // + up to 256 staged twiddle pairs
constexpr int kNbRun = 8;                            // block pass: limbs per tile run
constexpr int kNbTiles = (1 << 16) / kTile;          // tiles per limb at N = 2^16

struct NbUnit {
  const uint32_t *src;   // the unit's limb (source)
  uint32_t *dst;         // the unit's limb (destination)
  const uint32_t *src2;  // EPI_COMBINE: the inner-product limb u
  uint2 scale;           // EPI_SCALE: the output factor
  uint2 pinv;            // EPI_COMBINE: P^-1 mod q
  int prime, tile;
};

__device__ __forceinline__ uint32_t nb_col_addr(int k, int c) { return (uint32_t)(k * 16 + ((k >> 4) << 4) + c); }
__device__ __forceinline__ uint32_t nb_blk_addr(int c, int k) {
  const int r = k >> 4;
  return (uint32_t)(c * 272 + r * 16 + ((((k >> 2) & 3) ^ ((r >> 1) & 3)) << 2) + (k & 3));
}

// unit u of a launch -> (limb v, tile): column pass limb-major; block pass in runs of
// kNbRun limbs per tile (the last run may be shorter)
template <bool COLUMN>
__device__ __forceinline__ void nb_unit(int u, int total, int &v, int &tile) {
  if (COLUMN) {
    v = u / kNbTiles;
    tile = u % kNbTiles;
    return;
  }
  const int run = u / (kNbTiles * kNbRun);
  const int r = u - run * kNbTiles * kNbRun;
  const int v0 = run * kNbRun;
  const int len = min(kNbRun, total - v0);
  tile = r / len;
  v = v0 + r % len;
}

__device__ __forceinline__ void cp_async16(uint32_t dst_smem, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst_smem), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t *bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void nb_consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kNbConsumers) : "memory"); }

// The 15 lo-round twiddles of a consumer thread, entry (1 << m) - 1 + j for register bit
// m = 3 - bit and j = e >> (bit + 1).
template <bool COLUMN>
__device__ __forceinline__ void nb_twiddles(const uint2 *tw, int tile, int c, int tau, uint2 (&Lw)[15]) {
  constexpr int S0 = 8;  // LOGN - 8 at N = 2^16
#pragma unroll
  for (int m = 0; m < 4; m++) {
    const uint2 *from = COLUMN ? tw + (16 << m) + (tau << m)
                               : tw + (1 << (S0 + 4 + m)) + ((tile * 16 + c) << (4 + m)) + (tau << m);
    if (m == 0) {
      Lw[0] = __ldg(from);
    } else {
#pragma unroll
      for (int k2 = 0; k2 < (1 << m) / 2; k2++) {
        const uint4 w = __ldg(reinterpret_cast<const uint4 *>(from) + k2);
        Lw[(1 << m) - 1 + 2 * k2] = make_uint2(w.x, w.y);
        Lw[(1 << m) - 1 + 2 * k2 + 1] = make_uint2(w.z, w.w);
      }
    }
  }
}

// one radix-16 round (4 butterfly stages on the 16 register values); tw(m, j) is the
// twiddle of register bit 3 - m for butterfly group j
template <bool FWD, class TW>
__device__ __forceinline__ void nb_round(uint32_t (&x)[16], TW tw, uint32_t q) {
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int bit = FWD ? 3 - i : i;
    const int m = 3 - bit;
#pragma unroll
    for (int e = 0; e < 16; e++) {
      if (e & (1 << bit)) continue;
      const int e2 = e | (1 << bit);
      const uint2 w = tw(m, e >> (bit + 1));
      if (FWD) {
        const uint32_t t = red2(shoup_lazy(x[e2], w.x, w.y, q), q);
        const uint32_t u = red2(x[e], q);
        x[e] = u + t;
        x[e2] = u - t + q;
      } else {
        const uint32_t u = red2(x[e], q), v = red2(x[e2], q);
        x[e] = u + v;
        x[e2] = shoup_lazy(u - v + q, w.x, w.y, q);
      }
    }
  }
}

// Supported: column forward (PRO_PLAIN, EPI_LAZY), column inverse (PRO_PLAIN, EPI_SCALE),
// block forward (PRO_PLAIN, EPI_PLAIN or EPI_COMBINE), block inverse (PRO_PLAIN, EPI_LAZY);
// N = 2^16.
template <bool COLUMN, bool FWD, int EPI>
__global__ void __launch_bounds__(kNbThreads, 3)
    k_ntt_bulk(const __grid_constant__ SegList sl, const NttTables tb, unsigned int *status, int stages) {
  constexpr int N = 1 << 16;
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t *buf = reinterpret_cast<uint32_t *>(smem);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)stages * kNbStageWords * 4);
  uint64_t *empty = full + stages;
  NbUnit *desc = reinterpret_cast<NbUnit *>(empty + stages);
  const int tid = threadIdx.x;
  const int U = sl.total * kNbTiles;
  const int u0 = (int)(((long long)blockIdx.x * U) / gridDim.x);
  const int u1 = (int)(((long long)(blockIdx.x + 1) * U) / gridDim.x);
  const int nunits = u1 - u0;

  if (tid == 0) {
    for (int st = 0; st < stages; st++) {
      mbar_init(&full[st], 33);  // 32 producer lanes' copy completions + the descriptor
      mbar_init(&empty[st], kNbConsumers);
    }
  }
  __syncthreads();

  if (tid >= kNbConsumers) {  // ---------------------------------------------- producer warp
    const int lane = tid - kNbConsumers;
    bool ok = true;
    for (int k = 0; k < nunits && ok; k++) {
      const int st = k % stages;
      if (k >= stages) {
        bool w = true;
        if (lane == 0) w = mbar_wait_bounded(&empty[st], (uint32_t)(k / stages - 1) & 1u);
        ok = __shfl_sync(0xffffffffu, w ? 1 : 0, 0) != 0;
        if (!ok) break;
      }
      int v, tile;
      nb_unit<COLUMN>(u0 + k, sl.total, v, tile);
      int within;
      const Seg &sg = seg_at(sl, seg_find(sl, v, within));
      const uint32_t *src = sg.src + (size_t)within * sg.src_stride * N;
      const uint32_t sbase = smem_addr(buf + (size_t)st * kNbStageWords);
#pragma unroll 8
      for (int i = 0; i < 32; i++) {
        const int qd = lane + 32 * i;  // 16-byte chunk of the tile
        uint32_t off, dw;
        if (COLUMN) {
          const int k2 = qd >> 2, m = qd & 3;
          off = (uint32_t)(tile * 16 + k2 * 256 + 4 * m);
          dw = nb_col_addr(k2, 4 * m);
        } else {
          const int c = qd >> 6, r = (qd >> 2) & 15, m = qd & 3;
          off = (uint32_t)(tile * kTile + c * 256 + r * 16 + 4 * m);
          dw = (uint32_t)(c * 272 + r * 16 + ((m ^ ((r >> 1) & 3)) << 2));
        }
        cp_async16(sbase + dw * 4u, src + off);
      }
      // the hi-round twiddles of the unit (column: 8 chunks; block: four runs, 120 chunks)
      const uint2 *twp = (FWD ? tb.tw_fwd : tb.tw_inv) + (size_t)(sg.prime + within) * N;
      const uint32_t hbase = sbase + (uint32_t)kNbDataWords * 4u;
      if (COLUMN) {
        if (lane < 8) cp_async16(hbase + 16u * lane, twp + 2 * lane);
      } else {
        for (int h = lane; h < 120; h += 32) {
          const int m = h < 8 ? 0 : h < 24 ? 1 : h < 56 ? 2 : 3;
          const int first = 8 * ((1 << m) - 1);  // chunks of the runs before run m
          const int i2 = 2 * (h - first);        // twiddle index within run m
          cp_async16(hbase + (uint32_t)(16 * ((1 << m) - 1) + i2) * 8u, twp + (1 << (8 + m)) + ((tile * 16) << m) + i2);
        }
      }
      cp_async_arrive_noinc(&full[st]);
      if (lane == 0) {
        const KsArgs &ks = item_ks(sl, sg);
        NbUnit d;
        d.src = src;
        d.dst = sg.dst + (size_t)within * N;
        d.src2 = EPI == EPI_COMBINE ? sg.src2 + (size_t)within * N : nullptr;
        d.prime = sg.prime + within;
        d.tile = tile;
        d.scale = EPI == EPI_SCALE ? (sg.scale ? sg.scale[within] : tb.ninv[d.prime]) : make_uint2(0, 0);
        d.pinv = EPI == EPI_COMBINE ? ks.pinv[d.prime] : make_uint2(0, 0);
        desc[st] = d;
        mbar_arrive(&full[st]);  // the descriptor is readable (release)
      }
    }
    cp_async_wait_all();  // no copy of this warp is still in flight when it leaves
    return;
  }

  // ---------------------------------------------------------------- consumer warps
  int c, tau;
  if (COLUMN) {
    c = tid & 15;
    tau = tid >> 4;
  } else {
    c = tid >> 4;
    tau = tid & 15;
  }
  uint2 Lw[15];
  int cur_prime = -1, cur_tile = -1;
  bool ok = true;
  int k = 0;
  for (; k < nunits; k++) {
    const int st = k % stages;
    const bool w = mbar_wait_bounded(&full[st], (uint32_t)(k / stages) & 1u);
    ok = __all_sync(0xffffffffu, w);
    if (!ok) break;
    const NbUnit d = desc[st];
    const PrimeC P = tb.pc[d.prime];
    const uint32_t q = P.q;
    if (d.prime != cur_prime || (!COLUMN && d.tile != cur_tile)) {
      nb_twiddles<COLUMN>((FWD ? tb.tw_fwd : tb.tw_inv) + (size_t)d.prime * N, d.tile, c, tau, Lw);
      cur_prime = d.prime;
      cur_tile = d.tile;
    }
    uint32_t a[16];
    if (EPI == EPI_COMBINE) {  // the inner product's values at this thread's outputs (lo layout, contiguous)
      const uint4 *p = reinterpret_cast<const uint4 *>(d.src2 + d.tile * kTile + c * 256 + tau * 16);
#pragma unroll
      for (int e4 = 0; e4 < 4; e4++) {
        const uint4 t = __ldg(p + e4);
        a[4 * e4] = t.x, a[4 * e4 + 1] = t.y, a[4 * e4 + 2] = t.z, a[4 * e4 + 3] = t.w;
      }
    }
    uint32_t *sb = buf + (size_t)st * kNbStageWords;
    const uint2 *hs = reinterpret_cast<const uint2 *>(sb + kNbDataWords);
    auto hw = [&](int m, int j) { return COLUMN ? hs[(1 << m) + j] : hs[16 * ((1 << m) - 1) + (c << m) + j]; };
    auto lw = [&](int m, int j) { return Lw[(1 << m) - 1 + j]; };
    uint32_t x[16];
    // round 0 (hi going forward, lo going backward) straight from the stage
    if (COLUMN) {
#pragma unroll
      for (int e = 0; e < 16; e++) x[e] = sb[nb_col_addr(FWD ? ((e << 4) | tau) : ((tau << 4) | e), c)];
    } else if (FWD) {
#pragma unroll
      for (int e = 0; e < 16; e++) x[e] = sb[nb_blk_addr(c, (e << 4) | tau)];
    } else {
#pragma unroll
      for (int m = 0; m < 4; m++) {
        const uint4 t = *reinterpret_cast<const uint4 *>(sb + nb_blk_addr(c, (tau << 4) | (4 * m)));
        x[4 * m] = t.x, x[4 * m + 1] = t.y, x[4 * m + 2] = t.z, x[4 * m + 3] = t.w;
      }
    }
    if (FWD) nb_round<FWD>(x, hw, q);
    else nb_round<FWD>(x, lw, q);
    // exchange in place: each thread writes back the words it read, then reads the other round's
    if (COLUMN) {
#pragma unroll
      for (int e = 0; e < 16; e++) sb[nb_col_addr(FWD ? ((e << 4) | tau) : ((tau << 4) | e), c)] = x[e];
      nb_consumer_sync();
#pragma unroll
      for (int e = 0; e < 16; e++) x[e] = sb[nb_col_addr(FWD ? ((tau << 4) | e) : ((e << 4) | tau), c)];
    } else if (FWD) {
#pragma unroll
      for (int e = 0; e < 16; e++) sb[nb_blk_addr(c, (e << 4) | tau)] = x[e];
      __syncwarp();
#pragma unroll
      for (int m = 0; m < 4; m++) {
        const uint4 t = *reinterpret_cast<const uint4 *>(sb + nb_blk_addr(c, (tau << 4) | (4 * m)));
        x[4 * m] = t.x, x[4 * m + 1] = t.y, x[4 * m + 2] = t.z, x[4 * m + 3] = t.w;
      }
    } else {
#pragma unroll
      for (int m = 0; m < 4; m++)
        *reinterpret_cast<uint4 *>(sb + nb_blk_addr(c, (tau << 4) | (4 * m))) =
            make_uint4(x[4 * m], x[4 * m + 1], x[4 * m + 2], x[4 * m + 3]);
      __syncwarp();
#pragma unroll
      for (int e = 0; e < 16; e++) x[e] = sb[nb_blk_addr(c, (e << 4) | tau)];
    }
    if (FWD) {
      mbar_arrive(&empty[st]);  // this thread is done with the stage
      nb_round<FWD>(x, lw, q);
    } else {
      nb_round<FWD>(x, hw, q);  // the hi round reads its twiddles from the stage
      mbar_arrive(&empty[st]);
    }

    // epilogue: forward results are in lo layout (k = 16 tau + e), inverse in hi (k = 16 e + tau)
#pragma unroll
    for (int e = 0; e < 16; e++) {
      uint32_t o = x[e];
      if (EPI == EPI_PLAIN) o = red2(o, q);
      else if (EPI == EPI_SCALE) o = shoup(o, d.scale.x, d.scale.y, q);
      else if (EPI == EPI_COMBINE) o = shoup(a[e] + q - red2(o, q), d.pinv.x, d.pinv.y, q);
      x[e] = o;
    }
    if (COLUMN) {
      uint32_t *dst = d.dst + d.tile * 16 + c;
#pragma unroll
      for (int e = 0; e < 16; e++) dst[(size_t)(FWD ? ((tau << 4) | e) : ((e << 4) | tau)) * 256] = x[e];
    } else if (FWD) {
      uint4 *p = reinterpret_cast<uint4 *>(d.dst + d.tile * kTile + c * 256 + tau * 16);
#pragma unroll
      for (int e4 = 0; e4 < 4; e4++) p[e4] = make_uint4(x[4 * e4], x[4 * e4 + 1], x[4 * e4 + 2], x[4 * e4 + 3]);
    } else {
      uint32_t *dst = d.dst + d.tile * kTile + c * 256 + tau;
#pragma unroll
      for (int e = 0; e < 16; e++) dst[e * 16] = x[e];
    }
  }
  if (!ok && (tid & 31) == 0) atomicOr(status, 8u);  // an expired wait (the producer drains its copies)
}

// shared memory of a launch with `stages` stages
__host__ __device__ constexpr int ntt_bulk_smem(int stages) {
  return stages * (kNbStageWords * 4 + 16 + (int)sizeof(NbUnit));
}

}  // namespace fhe
