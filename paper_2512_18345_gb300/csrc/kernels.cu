// Kernel instantiations and launch wrappers.
#include <atomic>
#include <cstdio>

#include "bconv.cuh"
#include "elementwise.cuh"
#include "internal.h"
#include "ntt.cuh"

namespace fhe {

// HMult tensor product per limb i: d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1.
__global__ void __launch_bounds__(kEwThreads) k_tensor(const uint32_t *a, const uint32_t *b, uint32_t *d, int level,
                                                       const PrimeC *pc, int logn) {
  const size_t N = (size_t)1 << logn;
  const int blocks_per_limb = (int)(N / (4 * kEwThreads));
  const int i = blockIdx.x / blocks_per_limb;
  const size_t j0 = (size_t)(blockIdx.x % blocks_per_limb) * 4 * kEwThreads + threadIdx.x * 4;
  const PrimeC P = pc[i];
  const size_t poly = (size_t)level * N, off = (size_t)i * N + j0;
  const uint4 A0 = __ldg(reinterpret_cast<const uint4 *>(a + off)), A1 = __ldg(reinterpret_cast<const uint4 *>(a + poly + off));
  const uint4 B0 = __ldg(reinterpret_cast<const uint4 *>(b + off)), B1 = __ldg(reinterpret_cast<const uint4 *>(b + poly + off));
  const uint32_t a0[4] = {A0.x, A0.y, A0.z, A0.w}, a1[4] = {A1.x, A1.y, A1.z, A1.w};
  const uint32_t b0[4] = {B0.x, B0.y, B0.z, B0.w}, b1[4] = {B1.x, B1.y, B1.z, B1.w};
  uint32_t d0[4], d1[4], d2[4];
#pragma unroll
  for (int e = 0; e < 4; e++) {
    d0[e] = mul_mod(a0[e], b0[e], P);
    d1[e] = reduce_u64((uint64_t)a0[e] * b1[e] + (uint64_t)a1[e] * b0[e], P);  // < 2^63
    d2[e] = mul_mod(a1[e], b1[e], P);
  }
  *reinterpret_cast<uint4 *>(d + off) = make_uint4(d0[0], d0[1], d0[2], d0[3]);
  *reinterpret_cast<uint4 *>(d + poly + off) = make_uint4(d1[0], d1[1], d1[2], d1[3]);
  *reinterpret_cast<uint4 *>(d + 2 * poly + off) = make_uint4(d2[0], d2[1], d2[2], d2[3]);
}


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

// bracket one launch with trace events when tracing is on
struct TraceScope {
  Tracer *t;
  cudaStream_t s;
  TraceScope(const DevTables &tb, const char *name, cudaStream_t st) : t(tb.tracer), s(st) {
    if (t) t->begin(name, s);
  }
  ~TraceScope() {
    if (t) t->end(s);
  }
};

template <int LOGN, bool COLUMN, bool FWD, int PRO, int EPI>
static const char *ntt_name() {
  static const char *pro[] = {"", "+gather", "+reduce"};
  static const char *epi[] = {"", "", "+scale", "+combine", "+rescale"};
  static char buf[64];
  static bool init = false;
  if (!init) {
    snprintf(buf, sizeof buf, "%s_%s%s%s", FWD ? "ntt" : "intt", COLUMN ? "col" : "blk", pro[PRO], epi[EPI]);
    init = true;
  }
  return buf;
}

template <int LOGN, bool COLUMN, bool FWD, int PRO, int EPI>
static cudaError_t ntt_go(const DevTables &t, const SegList &sl, const KsArgs &ks, cudaStream_t s) {
  using G = NttGeom<LOGN, COLUMN>;
  const unsigned grid = (unsigned)(sl.total * G::TILES);
  if (grid == 0) return cudaSuccess;
  TraceScope ts(t, ntt_name<LOGN, COLUMN, FWD, PRO, EPI>(), s);
  k_ntt<LOGN, COLUMN, FWD, PRO, EPI><<<grid, kNttThreads, 0, s>>>(sl, t.ntt, ks);
  g_launches++;
  return cudaGetLastError();
}

// The (column, fwd, pro, epi) combinations the library uses.
template <int LOGN>
static cudaError_t ntt_dispatch(const DevTables &t, bool column, bool fwd, int pro, int epi, const SegList &sl,
                                const KsArgs &ks, cudaStream_t s) {
#define NTT_CASE(COL, FWDV, P, E) \
  if (column == COL && fwd == FWDV && pro == P && epi == E) return ntt_go<LOGN, COL, FWDV, P, E>(t, sl, ks, s);
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
                            const KsArgs &ks, cudaStream_t s) {
  switch (t.logn) {
    case 12: return ntt_dispatch<12>(t, column, fwd, pro, epi, sl, ks, s);
    case 16: return ntt_dispatch<16>(t, column, fwd, pro, epi, sl, ks, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_ntt(const DevTables &t, bool fwd, int pro, int epi, const SegList &first, const SegList &second,
                       const KsArgs &ks, cudaStream_t s) {
  cudaError_t e;
  if (fwd) {
    if ((e = launch_ntt_pass(t, true, true, pro, EPI_LAZY, first, ks, s)) != cudaSuccess) return e;
    return launch_ntt_pass(t, false, true, PRO_PLAIN, epi, second, ks, s);
  }
  if ((e = launch_ntt_pass(t, false, false, pro, EPI_LAZY, first, ks, s)) != cudaSuccess) return e;
  return launch_ntt_pass(t, true, false, PRO_PLAIN, epi, second, ks, s);
}

cudaError_t launch_bconv(const DevTables &t, const BconvArgs &a, int max_in, cudaStream_t s) {
  if (a.ngroups == 0) return cudaSuccess;
  int max_out = 0;
  for (int i = 0; i < a.ngroups && !a.dev; i++) max_out = a.g[i].n_out > max_out ? a.g[i].n_out : max_out;
  if (a.dev) max_out = 64;
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

cudaError_t launch_ip(const DevTables &t, const SegList &sl, const KsArgs &ks, cudaStream_t s) {
  const unsigned per_limb = (unsigned)((1u << t.logn) / (4 * kEwThreads));
  const unsigned grid = (unsigned)sl.total * per_limb;
  if (grid == 0) return cudaSuccess;
  TraceScope ts(t, "inner_product", s);
  const bool go = ks.galois_own != 1u, ge = ks.galois_ext != 1u;
  if (go && ge) k_ip<true, true><<<grid, kEwThreads, 0, s>>>(sl, t.pc, ks, t.logn);
  else if (go) k_ip<true, false><<<grid, kEwThreads, 0, s>>>(sl, t.pc, ks, t.logn);
  else if (ge) k_ip<false, true><<<grid, kEwThreads, 0, s>>>(sl, t.pc, ks, t.logn);
  else k_ip<false, false><<<grid, kEwThreads, 0, s>>>(sl, t.pc, ks, t.logn);
  g_launches++;
  return cudaGetLastError();
}

cudaError_t launch_ew(const DevTables &t, int op, const SegList &sl, const KsArgs &ks, cudaStream_t s) {
  const unsigned per_limb = (unsigned)((1u << t.logn) / (4 * kEwThreads));
  const unsigned grid = (unsigned)sl.total * per_limb;
  if (grid == 0) return cudaSuccess;
  static const char *names[] = {"ew_gather", "ew_scale", "ew_ip", "ew_combine", "ew_add", "ew_mul", "ew_copy"};
  TraceScope ts(t, op >= 0 && op < 7 ? names[op] : "ew", s);
  switch (op) {
    case EW_GATHER: k_ew<EW_GATHER><<<grid, kEwThreads, 0, s>>>(sl, t.pc, ks, t.logn); break;
    case EW_SCALE: k_ew<EW_SCALE><<<grid, kEwThreads, 0, s>>>(sl, t.pc, ks, t.logn); break;
    case EW_COMBINE: k_ew<EW_COMBINE><<<grid, kEwThreads, 0, s>>>(sl, t.pc, ks, t.logn); break;
    case EW_ADD: k_ew<EW_ADD><<<grid, kEwThreads, 0, s>>>(sl, t.pc, ks, t.logn); break;
    case EW_MUL: k_ew<EW_MUL><<<grid, kEwThreads, 0, s>>>(sl, t.pc, ks, t.logn); break;
    case EW_COPY: k_ew<EW_COPY><<<grid, kEwThreads, 0, s>>>(sl, t.pc, ks, t.logn); break;
    default: return cudaErrorInvalidValue;
  }
  g_launches++;
  return cudaGetLastError();
}

cudaError_t launch_tensor(const DevTables &t, const uint32_t *a, const uint32_t *b, uint32_t *d, int level,
                          cudaStream_t s) {
  const unsigned per_limb = (unsigned)((1u << t.logn) / (4 * kEwThreads));
  TraceScope ts(t, "tensor", s);
  k_tensor<<<per_limb * (unsigned)level, kEwThreads, 0, s>>>(a, b, d, level, t.pc, t.logn);
  g_launches++;
  return cudaGetLastError();
}

}  // namespace fhe
