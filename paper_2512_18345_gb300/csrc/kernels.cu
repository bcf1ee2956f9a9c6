// Kernel instantiations and launch wrappers.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <string>

#include "bconv.cuh"
#include "elementwise.cuh"
#include "internal.h"
#include "ntt.cuh"
#include "ntt_bulk.cuh"
#include "ip_intt.cuh"
#include "ip_hoisted.cuh"

namespace fhe {

static std::atomic<long long> g_launches{0};
long long kernel_launches() { return g_launches.load(); }

cudaEvent_t Tracer::get() {
  if (used == pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    pool.push_back(e);
  }
  return pool[used++];
}
void Tracer::begin(const char *name, cudaStream_t s) {
  TraceRec r{name, get(), get()};
  cudaEventRecord(r.a, s);
  recs.push_back(r);
}
void Tracer::end(cudaStream_t s) { cudaEventRecord(recs.back().b, s); }
Tracer::~Tracer() {
  for (auto e : pool) cudaEventDestroy(e);
}

void note_launch() { g_launches++; }

template <int LOGN, bool COLUMN, bool FWD, int PRO, int EPI, bool OTF>
static const char *ntt_name() {
  static const char *pro[] = {"", "+gather", "+reduce"};
  static const char *epi[] = {"", "", "+scale", "+combine", "+rescale"};
  static const std::string name = [] {  // initialised once, thread-safe
    char buf[64];
    snprintf(buf, sizeof buf, "%s_%s%s%s%s", FWD ? "ntt" : "intt", COLUMN ? "col" : "blk", pro[PRO], epi[EPI],
             OTF ? "+otf" : "");
    return std::string(buf);
  }();
  return name.c_str();
}

template <int LOGN, bool COLUMN, bool FWD, int PRO, int EPI, bool OTF>
static cudaError_t ntt_go(const DevTables &t, const SegList &sl, cudaStream_t s) {
  using G = NttGeom<LOGN, COLUMN>;
  const unsigned grid = (unsigned)(sl.total * G::TILES);
  if (grid == 0) return cudaSuccess;
  constexpr int smem = ntt_twiddle_smem(COLUMN, G::S);
  static PerDeviceOnce configured;  // opt in to > 48 KB of shared memory once per instantiation and device
  cudaError_t e = configured.run([] {
    return cudaFuncSetAttribute(k_ntt<LOGN, COLUMN, FWD, PRO, EPI, OTF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem);
  });
  if (e != cudaSuccess) return e;
  TraceScope ts(t, ntt_name<LOGN, COLUMN, FWD, PRO, EPI, OTF>(), s);
  k_ntt<LOGN, COLUMN, FWD, PRO, EPI, OTF><<<grid, kNttThreads, smem, s>>>(sl, t.ntt);
  g_launches++;
  return cudaGetLastError();
}

// Streaming pass (ntt_bulk.cuh): persistent CTAs, two per SM, each walking a contiguous
// range of the launch's units.
template <bool COLUMN, bool FWD, int EPI>
static cudaError_t ntt_bulk_go(const DevTables &t, const SegList &sl, cudaStream_t s) {
  const int units = sl.total * kNbTiles;
  if (units == 0) return cudaSuccess;
  const int stages = t.ntt_stream_stages;
  const int smem = ntt_bulk_smem(stages);
  static PerDeviceOnce configured;
  cudaError_t e = configured.run([] {
    return cudaFuncSetAttribute(k_ntt_bulk<COLUMN, FWD, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                ntt_bulk_smem(8));
  });
  if (e != cudaSuccess) return e;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::min(units, std::max(1, std::min(3, t.ntt_stream_ctas)) * sms);
  static const char *names[2][2] = {{"intt_blk", "ntt_blk"}, {"intt_col", "ntt_col"}};
  const char *name = EPI == EPI_COMBINE ? "ntt_blk+combine" : EPI == EPI_SCALE ? "intt_col+scale"
                     : EPI == EPI_PLAIN ? "ntt_blk" : names[COLUMN][FWD];
  TraceScope ts(t, name, s);
  k_ntt_bulk<COLUMN, FWD, EPI><<<grid, kNbThreads, smem, s>>>(sl, t.ntt, t.status, stages);
  g_launches++;
  return cudaGetLastError();
}

// The (column, fwd, pro, epi) combinations the library uses; on-the-fly twiddles apply to
// the block passes.
template <int LOGN>
static cudaError_t ntt_dispatch(const DevTables &t, bool column, bool fwd, int pro, int epi, const SegList &sl,
                                cudaStream_t s) {
  const bool otf = t.ntt_otf != 0;
  if constexpr (LOGN == 16) {
    if (t.ntt_stream && pro == PRO_PLAIN) {
      if (column && fwd && epi == EPI_LAZY) return ntt_bulk_go<true, true, EPI_LAZY>(t, sl, s);
      if (column && !fwd && epi == EPI_SCALE) return ntt_bulk_go<true, false, EPI_SCALE>(t, sl, s);
      if (!column && fwd && epi == EPI_PLAIN) return ntt_bulk_go<false, true, EPI_PLAIN>(t, sl, s);
      if (!column && fwd && epi == EPI_COMBINE) return ntt_bulk_go<false, true, EPI_COMBINE>(t, sl, s);
      if (!column && !fwd && epi == EPI_LAZY) return ntt_bulk_go<false, false, EPI_LAZY>(t, sl, s);
    }
  }
#define NTT_CASE(COL, FWDV, P, E)                                                              \
  if (column == COL && fwd == FWDV && pro == P && epi == E) {                                  \
    if constexpr (!COL) {                                                                      \
      if (otf) return ntt_go<LOGN, COL, FWDV, P, E, true>(t, sl, s);                           \
    }                                                                                          \
    return ntt_go<LOGN, COL, FWDV, P, E, false>(t, sl, s);                                     \
  }
  NTT_CASE(true, true, PRO_PLAIN, EPI_LAZY)
  NTT_CASE(true, true, PRO_REDUCE, EPI_LAZY)
  NTT_CASE(false, true, PRO_PLAIN, EPI_PLAIN)
  NTT_CASE(false, true, PRO_PLAIN, EPI_COMBINE)
  NTT_CASE(false, true, PRO_PLAIN, EPI_RESCALE)
  NTT_CASE(false, false, PRO_PLAIN, EPI_LAZY)
  NTT_CASE(false, false, PRO_GATHER, EPI_LAZY)
  NTT_CASE(true, false, PRO_PLAIN, EPI_SCALE)
#undef NTT_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_ntt_pass(const DevTables &t, bool column, bool fwd, int pro, int epi, const SegList &sl,
                            cudaStream_t s) {
  switch (t.logn) {
    case 12: return ntt_dispatch<12>(t, column, fwd, pro, epi, sl, s);
    case 16: return ntt_dispatch<16>(t, column, fwd, pro, epi, sl, s);
    default: return cudaErrorInvalidValue;
  }
}

template <bool FWD, int PRO, int EPI, bool OTF>
static cudaError_t ntt1_go(const DevTables &t, const SegList &first, const SegList &second, cudaStream_t s) {
  const unsigned grid = (unsigned)(first.total * 16);
  if (grid == 0) return cudaSuccess;
  constexpr int smem = ntt_twiddle_smem(true, 256);  // the larger of the two passes' tables
  static PerDeviceOnce configured;
  cudaError_t e = configured.run(
      [] { return cudaFuncSetAttribute(k_ntt1<FWD, PRO, EPI, OTF>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1); });
  if (e != cudaSuccess) return e;
  static const char *name = FWD ? (OTF ? "ntt1+otf" : "ntt1") : (OTF ? "intt1+otf" : "intt1");
  TraceScope ts(t, name, s);
  k_ntt1<FWD, PRO, EPI, OTF><<<grid, kNttThreads, smem, s>>>(first, second, t.ntt);
  g_launches++;
  return cudaGetLastError();
}

int ntt_single_pass_clusters() {
  auto kern = k_ntt1<true, PRO_PLAIN, EPI_PLAIN, false>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) return 0;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = 16;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.gridDim = dim3(16 * 64);
  cfg.blockDim = dim3(kNttThreads);
  cfg.dynamicSmemBytes = ntt_twiddle_smem(true, 256);
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

bool ntt_single_pass_ok(const DevTables &t, int pro, int epi, bool fwd) {
  if (t.logn != 16) return false;
  if (fwd) return (pro == PRO_PLAIN && (epi == EPI_PLAIN || epi == EPI_COMBINE)) || (pro == PRO_REDUCE && epi == EPI_RESCALE);
  return (pro == PRO_PLAIN || pro == PRO_GATHER) && epi == EPI_SCALE;
}

// grid-barrier counters of the persistent transform: each launch takes the next slot (one
// 32-byte sector each) and zeroes it on its stream first; two launches share a slot only
// with kGbarSlots launches between them, none of which may still be running
static std::atomic<unsigned> g_gbar_next{0};

template <bool FWD, int PRO, int EPI>
static cudaError_t nttp_go(const DevTables &t, const SegList &first, const SegList &second, cudaStream_t s) {
  const int units = first.total * 16;
  if (units == 0) return cudaSuccess;
  if (!t.gbar) return cudaErrorInvalidValue;
  constexpr int smem = ntt_twiddle_smem(true, 256);  // the larger of the two passes' tables
  auto kern = k_nttp<FWD, PRO, EPI>;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kNttThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const unsigned grid = (unsigned)std::min(units, per_sm * sms);  // every CTA resident at once
  unsigned int *ctr = t.gbar + 8 * (g_gbar_next.fetch_add(1) % kGbarSlots);
  if ((e = cudaMemsetAsync(ctr, 0, sizeof(unsigned int), s)) != cudaSuccess) return e;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeCooperative;
  attr.val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kNttThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  TraceScope ts(t, FWD ? "nttp" : "inttp", s);
  e = cudaLaunchKernelEx(&cfg, kern, first, second, t.ntt, ctr, t.status);
  g_launches++;
  return e;
}

cudaError_t launch_ntt_single(const DevTables &t, bool fwd, int pro, int epi, const SegList &first,
                              const SegList &second, cudaStream_t s) {
  if (t.ntt_persist) {
#define NTTP_CASE(FWDV, P, E) \
  if (fwd == FWDV && pro == P && epi == E) return nttp_go<FWDV, P, E>(t, first, second, s);
    NTTP_CASE(true, PRO_PLAIN, EPI_PLAIN)
    NTTP_CASE(true, PRO_PLAIN, EPI_COMBINE)
    NTTP_CASE(true, PRO_REDUCE, EPI_RESCALE)
    NTTP_CASE(false, PRO_PLAIN, EPI_SCALE)
    NTTP_CASE(false, PRO_GATHER, EPI_SCALE)
#undef NTTP_CASE
    return cudaErrorInvalidValue;
  }
  const bool otf = t.ntt_otf != 0;
#define NTT1_CASE(FWDV, P, E)                                                  \
  if (fwd == FWDV && pro == P && epi == E)                                     \
    return otf ? ntt1_go<FWDV, P, E, true>(t, first, second, s) : ntt1_go<FWDV, P, E, false>(t, first, second, s);
  NTT1_CASE(true, PRO_PLAIN, EPI_PLAIN)
  NTT1_CASE(true, PRO_PLAIN, EPI_COMBINE)
  NTT1_CASE(true, PRO_REDUCE, EPI_RESCALE)
  NTT1_CASE(false, PRO_PLAIN, EPI_SCALE)
  NTT1_CASE(false, PRO_GATHER, EPI_SCALE)
#undef NTT1_CASE
  return cudaErrorInvalidValue;
}

static bool same_limbs(const SegList &a, const SegList &b) {
  if (a.dev || b.dev || a.nseg != b.nseg || a.total != b.total) return false;
  for (int i = 0; i < a.nseg; i++)
    if (a.seg[i].n != b.seg[i].n || a.seg[i].prime != b.seg[i].prime) return false;
  return true;
}

cudaError_t launch_ntt(const DevTables &t, bool fwd, int pro, int epi, const SegList &first, const SegList &second,
                       cudaStream_t s) {
  if ((t.ntt_single || t.ntt_persist) && ntt_single_pass_ok(t, pro, epi, fwd) && same_limbs(first, second))
    return launch_ntt_single(t, fwd, pro, epi, first, second, s);
  cudaError_t e;
  if (fwd) {
    if ((e = launch_ntt_pass(t, true, true, pro, EPI_LAZY, first, s)) != cudaSuccess) return e;
    return launch_ntt_pass(t, false, true, PRO_PLAIN, epi, second, s);
  }
  if ((e = launch_ntt_pass(t, false, false, pro, EPI_LAZY, first, s)) != cudaSuccess) return e;
  return launch_ntt_pass(t, true, false, PRO_PLAIN, epi, second, s);
}

cudaError_t launch_bconv(const DevTables &t, const BconvArgs &a, int max_in, int max_out, cudaStream_t s) {
  if (a.ngroups == 0) return cudaSuccess;
  const dim3 grid((unsigned)((1u << t.logn) / (4 * kBconvThreads)), (unsigned)((max_out + kBconvOutChunk - 1) / kBconvOutChunk),
                  (unsigned)a.ngroups);
  TraceScope ts(t, "bconv", s);
  switch (max_in) {
#define BC(n) \
  case n: k_bconv<n><<<grid, kBconvThreads, 0, s>>>(a, t.pc, t.logn); break;
    BC(1) BC(2) BC(3) BC(4) BC(5) BC(6) BC(7) BC(8)
#undef BC
    default:
      if (max_in <= 12) k_bconv<12><<<grid, kBconvThreads, 0, s>>>(a, t.pc, t.logn);
      else if (max_in <= 16) k_bconv<16><<<grid, kBconvThreads, 0, s>>>(a, t.pc, t.logn);
      else return cudaErrorInvalidValue;
  }
  g_launches++;
  return cudaGetLastError();
}

cudaError_t launch_ip(const DevTables &t, const SegList &sl, bool gather_own, bool gather_ext, bool add_c1,
                      int beta_max, cudaStream_t s) {
  if (sl.total == 0) return cudaSuccess;
  TraceScope ts(t, "inner_product", s);
  const bool go = gather_own, ge = gather_ext;
  if (ge && t.ip_staged && !add_c1 && beta_max >= 1 && beta_max <= 4 && (1 << t.logn) % kIpChunk == 0) {
    // hoisted: every row's permuted 32-coefficient blocks staged in shared memory by each warp
    // for itself (ip_hoisted.cuh): one or two CTAs per SM, each warp with D stages (2..4; by
    // default 2), as many warps as the shared memory holds (at most 16 per SM)
    const int ctas = std::max(1, std::min(2, t.ip_staged_ctas));
    const int budget = (ctas == 2 ? 113 : 227) * 1024;
    const int ws = ip_hoisted_stage_words(beta_max) * 4;  // one stage of one warp
    int D = t.ip_staged_depth >= 2 && t.ip_staged_depth <= 4 ? t.ip_staged_depth : 2;
    while (D > 2 && budget / (D * ws) < 1) D--;
    const int warps = std::max(1, std::min(kIhMaxWarps / ctas, budget / (D * ws)));
    static PerDeviceOnce configured[3];
    const cudaError_t e = configured[D - 2].run([D] {
      constexpr int kMax = 227 * 1024;
      return D == 2   ? cudaFuncSetAttribute(k_ip_hoisted<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMax)
             : D == 3 ? cudaFuncSetAttribute(k_ip_hoisted<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMax)
                      : cudaFuncSetAttribute(k_ip_hoisted<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMax);
    });
    if (e != cudaSuccess) return e;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int wunits = sl.total * ((1 << t.logn) / kIhUnit);
    const unsigned grid = (unsigned)std::min((wunits + warps - 1) / warps, ctas * sms);
    const int smem = warps * D * ws;
    if (D == 2) k_ip_hoisted<2><<<grid, warps * 32, smem, s>>>(sl, t.pc, t.logn, beta_max);
    else if (D == 3) k_ip_hoisted<3><<<grid, warps * 32, smem, s>>>(sl, t.pc, t.logn, beta_max);
    else k_ip_hoisted<4><<<grid, warps * 32, smem, s>>>(sl, t.pc, t.logn, beta_max);
    g_launches++;
    return cudaGetLastError();
  }
  if (beta_max >= 1 && beta_max <= 4 && (1 << t.logn) % kIpChunk == 0) {
    // streaming kernel, one or two CTAs per SM.  Two stages per CTA where each stage holds
    // the ModUp values and the keys (with the producer warp refilling a stage as soon as it
    // is released, a third stage bought nothing and took shared memory from the transforms
    // running beside it on other lanes); with the digits gathered through the automorphism
    // (hoisted rotations) a stage holds the keys alone, and up to four stages fill the same
    // shared memory.
    const int stage_bytes = (ge ? 2 : 3) * beta_max * kIpChunk * 4;
    const int per_stage = stage_bytes + 24 + (int)sizeof(IpUnit);  // data, three mbarriers, descriptor
    const int stages = std::min(ge ? 4 : 2, (113 * 1024 - 256) / per_stage);
    const int smem = stages * per_stage;
    static PerDeviceOnce configured[4];
    const int variant = (go ? 1 : 0) + (ge ? 2 : 0);
    const cudaError_t e = configured[variant].run([variant] {
      constexpr int kMax = 113 * 1024;
      switch (variant) {
        case 0: return cudaFuncSetAttribute(k_ip_bulk<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMax);
        case 1: return cudaFuncSetAttribute(k_ip_bulk<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMax);
        case 2: return cudaFuncSetAttribute(k_ip_bulk<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMax);
        default: return cudaFuncSetAttribute(k_ip_bulk<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMax);
      }
    });
    if (e != cudaSuccess) return e;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int units = sl.total * ((1 << t.logn) / kIpChunk);
    const unsigned grid = (unsigned)std::min(units, std::max(1, std::min(2, t.ip_ctas_per_sm)) * sms);
    switch (variant) {
      case 0: k_ip_bulk<false, false><<<grid, kIpThreads + 32, smem, s>>>(sl, t.pc, t.logn, t.status, beta_max, stages); break;
      case 1: k_ip_bulk<true, false><<<grid, kIpThreads + 32, smem, s>>>(sl, t.pc, t.logn, t.status, beta_max, stages); break;
      case 2: k_ip_bulk<false, true><<<grid, kIpThreads + 32, smem, s>>>(sl, t.pc, t.logn, t.status, beta_max, stages); break;
      default: k_ip_bulk<true, true><<<grid, kIpThreads + 32, smem, s>>>(sl, t.pc, t.logn, t.status, beta_max, stages); break;
    }
    g_launches++;
    return cudaGetLastError();
  }
  const unsigned per_limb = (unsigned)((1u << t.logn) / (4 * kEwThreads));
  const unsigned grid = (unsigned)sl.total * per_limb;
  if (go && ge) k_ip<true, true><<<grid, kEwThreads, 0, s>>>(sl, t.pc, t.logn);
  else if (go) k_ip<true, false><<<grid, kEwThreads, 0, s>>>(sl, t.pc, t.logn);
  else if (ge) k_ip<false, true><<<grid, kEwThreads, 0, s>>>(sl, t.pc, t.logn);
  else k_ip<false, false><<<grid, kEwThreads, 0, s>>>(sl, t.pc, t.logn);
  g_launches++;
  return cudaGetLastError();
}

cudaError_t launch_ew(const DevTables &t, int op, const SegList &sl, cudaStream_t s) {
  const unsigned per_limb = (unsigned)((1u << t.logn) / (4 * kEwThreads));
  const unsigned grid = (unsigned)sl.total * per_limb;
  if (grid == 0) return cudaSuccess;
  static const char *names[] = {"ew_gather", "ew_scale", "ew_ip", "ew_combine", "ew_add", "ew_mul", "ew_copy",
                                "tensor"};
  TraceScope ts(t, op >= 0 && op < 8 ? names[op] : "ew", s);
  switch (op) {
    case EW_GATHER: k_ew<EW_GATHER><<<grid, kEwThreads, 0, s>>>(sl, t.pc, t.logn); break;
    case EW_SCALE: k_ew<EW_SCALE><<<grid, kEwThreads, 0, s>>>(sl, t.pc, t.logn); break;
    case EW_COMBINE: k_ew<EW_COMBINE><<<grid, kEwThreads, 0, s>>>(sl, t.pc, t.logn); break;
    case EW_ADD: k_ew<EW_ADD><<<grid, kEwThreads, 0, s>>>(sl, t.pc, t.logn); break;
    case EW_MUL: k_ew<EW_MUL><<<grid, kEwThreads, 0, s>>>(sl, t.pc, t.logn); break;
    case EW_COPY: k_ew<EW_COPY><<<grid, kEwThreads, 0, s>>>(sl, t.pc, t.logn); break;
    case EW_TENSOR: k_ew<EW_TENSOR><<<grid, kEwThreads, 0, s>>>(sl, t.pc, t.logn); break;
    default: return cudaErrorInvalidValue;
  }
  g_launches++;
  return cudaGetLastError();
}

cudaError_t launch_ip_intt(const DevTables &t, const SegList &sl, int beta_max, cudaStream_t s) {
  if (sl.total == 0) return cudaSuccess;
  if (t.logn != 16 || beta_max < 1 || beta_max > 4) return cudaErrorInvalidValue;
  TraceScope ts(t, "ip+intt_blk", s);
  const unsigned grid = (unsigned)sl.total * 32u;  // 16 tiles x 2 halves per special limb
  switch (beta_max) {
    case 1: k_ip_intt<1><<<grid, kIpIttThreads, 0, s>>>(sl, t.ntt); break;
    case 2: k_ip_intt<2><<<grid, kIpIttThreads, 0, s>>>(sl, t.ntt); break;
    case 3: k_ip_intt<3><<<grid, kIpIttThreads, 0, s>>>(sl, t.ntt); break;
    default: k_ip_intt<4><<<grid, kIpIttThreads, 0, s>>>(sl, t.ntt); break;
  }
  g_launches++;
  return cudaGetLastError();
}

}  // namespace fhe
