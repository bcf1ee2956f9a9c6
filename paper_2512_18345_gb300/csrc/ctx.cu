// Host side of the C ABI (include/fhe.h): parameter validation, the device
// tables (twiddles, base-conversion tables), switching keys, the workspace
// and the key-switching pipelines built from the kernels in kernels.cu.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/fhe.h"
#include "bconv.cuh"
#include "elementwise.cuh"
#include "internal.h"
#include "ctx.h"

using namespace fhe;

// ---------------------------------------------------------------- errors
static thread_local std::string g_err;

int fhe_fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

extern "C" const char *fhe_last_error(void) { return g_err.c_str(); }

#define CUDA_OR_FAIL(call)                                                                     \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fhe_fail(e_ == cudaErrorMemoryAllocation ? FHE_ENOMEM : FHE_ECUDA, "%s: %s (%s:%d)", \
                      #call, cudaGetErrorString(e_), __FILE__, __LINE__);                      \
  } while (0)

// ---------------------------------------------------------------- host number theory
static uint32_t h_mul(uint32_t a, uint32_t b, uint32_t q) { return (uint32_t)((uint64_t)a * b % q); }
static uint32_t h_pow(uint32_t a, uint64_t e, uint32_t q) {
  uint64_t r = 1 % q, b = a % q;
  for (; e; e >>= 1) {
    if (e & 1) r = r * b % q;
    b = b * b % q;
  }
  return (uint32_t)r;
}
static uint32_t h_inv(uint32_t a, uint32_t q) { return h_pow(a, q - 2, q); }
static bool h_is_prime(uint32_t n) {  // deterministic Miller-Rabin for 32-bit n (bases 2, 7, 61)
  if (n < 2) return false;
  for (uint32_t p : {2u, 3u, 5u, 7u, 11u, 13u, 61u})
    if (n % p == 0) return n == p;
  uint32_t d = n - 1;
  int s = 0;
  while (!(d & 1)) d >>= 1, s++;
  for (uint32_t a : {2u, 7u, 61u}) {
    uint32_t x = h_pow(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int i = 1; i < s && comp; i++) {
      x = h_mul(x, x, n);
      if (x == n - 1) comp = false;
    }
    if (comp) return false;
  }
  return true;
}
// psi = g^((q-1)/2N) for the smallest g >= 2 with psi^N = -1
static uint32_t h_psi(uint32_t q, uint32_t N) {
  for (uint32_t g = 2; g < q; g++) {
    const uint32_t psi = h_pow(g, (q - 1) / (2ull * N), q);
    if (h_pow(psi, N, q) == q - 1) return psi;
  }
  return 0;
}
static uint32_t h_shoup(uint32_t w, uint32_t q) { return (uint32_t)(((uint64_t)w << 32) / q); }
static uint2 h_pair(uint32_t w, uint32_t q) { return make_uint2(w, h_shoup(w, q)); }
static uint32_t h_brv(uint32_t x, int bits) {
  uint32_t r = 0;
  for (int i = 0; i < bits; i++) r |= ((x >> i) & 1u) << (bits - 1 - i);
  return r;
}

static int ceil_div(int a, int b) { return (a + b - 1) / b; }
uint32_t h_mulmod_pub(uint32_t a, uint32_t b, uint32_t q) { return h_mul(a, b, q); }
uint32_t h_invmod_pub(uint32_t a, uint32_t q) { return h_inv(a, q); }

// ---------------------------------------------------------------- context

int fhe_ctx::beta(int level) const { return ceil_div(level, alpha); }

int fhe_ctx::ext_prime(int level, int t) const { return t < level ? t : L + (t - level); }

void fhe_ctx::order_stream(cudaStream_t s) {
  if (capturing) return;
  if (have_last && s != last_stream) {
    cudaEventRecord(order_ev, last_stream);
    cudaStreamWaitEvent(s, order_ev, 0);
  }
  last_stream = s;
  have_last = true;
}

template <class T>
static cudaError_t upload(T **dptr, const std::vector<T> &v) {
  cudaError_t e = cudaMalloc((void **)dptr, sizeof(T) * (v.empty() ? 1 : v.size()));
  if (e != cudaSuccess) return e;
  if (!v.empty()) e = cudaMemcpy(*dptr, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
  return e;
}

static int build_tables(fhe_ctx *c) {
  const uint32_t N = c->N;
  const int NP = c->L + c->K;
  const std::vector<uint32_t> &pr = c->primes;
  // the tensor-core BConv's contraction width for this digit size and special-prime count
  const int wide = std::max(c->alpha, c->K);
  c->tabs.tc_k = wide <= fhe::kTcMaxIn ? fhe::kTcK : wide <= fhe::kTcMaxIn12 ? fhe::kTcK12 : 0;
  // per-prime constants
  std::vector<PrimeC> pcs(NP);
  for (int i = 0; i < NP; i++) {
    const uint32_t q = pr[i];
    PrimeC p{};
    p.q = q;
    p.r32 = (uint32_t)((1ull << 32) % q);
    p.r32s = h_shoup(p.r32, q);
    p.div32 = (uint32_t)((1ull << 32) / q);
    p.r64 = h_mul(p.r32, p.r32, q);
    p.r64s = h_shoup(p.r64, q);
    p.r34 = (uint32_t)((1ull << 34) % q);
    pcs[i] = p;
    c->psi[i] = h_psi(q, N);
  }
  CUDA_OR_FAIL(upload(&c->d_pc, pcs));
  // twiddles: tw[k] = psi^brv(k), itw[k] = psi^-brv(k), with Shoup companions
  std::vector<uint2> tw((size_t)NP * N), itw((size_t)NP * N), ninv(NP);
  std::vector<uint32_t> pw(N), ipw(N);
  for (int i = 0; i < NP; i++) {
    const uint32_t q = pr[i], psi = c->psi[i], ipsi = h_inv(psi, q);
    pw[0] = ipw[0] = 1;
    for (uint32_t k = 1; k < N; k++) {
      pw[k] = h_mul(pw[k - 1], psi, q);
      ipw[k] = h_mul(ipw[k - 1], ipsi, q);
    }
    for (uint32_t k = 0; k < N; k++) {
      const uint32_t b = h_brv(k, c->logn);
      tw[(size_t)i * N + k] = h_pair(pw[b], q);
      itw[(size_t)i * N + k] = h_pair(ipw[b], q);
    }
    ninv[i] = h_pair(h_inv(N % q, q), q);
  }
  CUDA_OR_FAIL(upload(&c->d_tw, tw));
  CUDA_OR_FAIL(upload(&c->d_itw, itw));
  CUDA_OR_FAIL(upload(&c->d_ninv, ninv));

  // ModUp tables per level: pre-factor of each q-limb ((D/q_t)^-1 mod q_t, with and
  // without N^-1) and the BConv table of every digit (rows in ext-limb order).
  const int L = c->L, K = c->K, A = c->alpha;
  std::vector<uint2> mu_scale((size_t)L * L), mu_qhinv((size_t)L * L);
  c->modup_T.assign((size_t)L * c->dnum, nullptr);
  c->modup_map.assign((size_t)L * c->dnum, nullptr);
  c->modup_Btc.assign((size_t)L * c->dnum, nullptr);
  for (int level = 1; level <= L; level++) {
    const int beta = c->beta(level);
    for (int j = 0; j < beta; j++) {
      const int lo = j * A, hi = std::min((j + 1) * A, level), a = hi - lo;
      for (int t = lo; t < hi; t++) {
        const uint32_t q = pr[t];
        uint32_t prod = 1;
        for (int k = lo; k < hi; k++)
          if (k != t) prod = h_mul(prod, pr[k] % q, q);
        const uint32_t qh = h_inv(prod, q);
        mu_qhinv[(size_t)(level - 1) * L + t] = h_pair(qh, q);
        mu_scale[(size_t)(level - 1) * L + t] = h_pair(h_mul(qh, h_inv(N % q, q), q), q);
      }
      std::vector<uint32_t> T;
      std::vector<int2> om;
      for (int t = 0; t < level + K; t++) {
        if (t >= lo && t < hi) continue;
        const int pi = c->ext_prime(level, t);
        const uint32_t p = pr[pi];
        for (int k = lo; k < hi; k++) {
          uint32_t prod = 1;
          for (int m = lo; m < hi; m++)
            if (m != k) prod = h_mul(prod, pr[m] % p, p);
          T.push_back(prod);
        }
        om.push_back(make_int2(t, pi));
      }
      (void)a;
      CUDA_OR_FAIL(upload(&c->modup_T[(size_t)(level - 1) * c->dnum + j], T));
      CUDA_OR_FAIL(upload(&c->modup_map[(size_t)(level - 1) * c->dnum + j], om));
      std::vector<uint32_t> pout;
      for (const int2 &m : om) pout.push_back(pr[m.y]);
      if (c->tabs.tc_k)  // tensor-core tables (digits of at most 8 limbs: K = 48; at most 12: K = 64)
        CUDA_OR_FAIL(upload(&c->modup_Btc[(size_t)(level - 1) * c->dnum + j],
                            fhe::bconv_tc_table(T, hi - lo, pout, c->tabs.tc_k)));
    }
  }
  CUDA_OR_FAIL(upload(&c->d_mu_scale, mu_scale));
  CUDA_OR_FAIL(upload(&c->d_mu_qhinv, mu_qhinv));

  // ModDown: pre-factor (P/p_k)^-1 mod p_k (with / without N^-1), table [P/p_k]_{q_i},
  // P^-1 mod q_i.
  std::vector<uint2> md_scale(K), md_phinv(K), pinv(L), pmod(L);
  std::vector<uint32_t> mdT((size_t)L * K);
  std::vector<int2> mdmap(L);
  for (int k = 0; k < K; k++) {
    const uint32_t p = pr[L + k];
    uint32_t prod = 1;
    for (int m = 0; m < K; m++)
      if (m != k) prod = h_mul(prod, pr[L + m] % p, p);
    const uint32_t ph = h_inv(prod, p);
    md_phinv[k] = h_pair(ph, p);
    md_scale[k] = h_pair(h_mul(ph, h_inv(N % p, p), p), p);
  }
  for (int i = 0; i < L; i++) {
    const uint32_t q = pr[i];
    uint32_t P = 1;
    for (int m = 0; m < K; m++) P = h_mul(P, pr[L + m] % q, q);
    pinv[i] = h_pair(h_inv(P, q), q);
    pmod[i] = h_pair(P, q);
    for (int k = 0; k < K; k++) {
      uint32_t prod = 1;
      for (int m = 0; m < K; m++)
        if (m != k) prod = h_mul(prod, pr[L + m] % q, q);
      mdT[(size_t)i * K + k] = prod;
    }
    mdmap[i] = make_int2(i, i);
  }
  CUDA_OR_FAIL(upload(&c->d_md_scale, md_scale));
  CUDA_OR_FAIL(upload(&c->d_md_phinv, md_phinv));
  CUDA_OR_FAIL(upload(&c->d_pinv, pinv));
  CUDA_OR_FAIL(upload(&c->d_pmod, pmod));
  CUDA_OR_FAIL(upload(&c->d_mdT, mdT));
  CUDA_OR_FAIL(upload(&c->d_mdmap, mdmap));
  if (c->tabs.tc_k)
    CUDA_OR_FAIL(upload(&c->d_md_Btc, fhe::bconv_tc_table(mdT, K, std::vector<uint32_t>(pr.begin(), pr.begin() + L),
                                                          c->tabs.tc_k)));
  CUDA_OR_FAIL(upload(&c->d_status, std::vector<unsigned int>(1, 0u)));
  c->tabs.status = c->d_status;
  CUDA_OR_FAIL(upload(&c->d_gbar, std::vector<unsigned int>((size_t)fhe::kGbarSlots * 8, 0u)));
  c->tabs.gbar = c->d_gbar;

  // rescale: q_{l-1}^-1 mod q_i for every level l and i < l-1
  std::vector<uint2> rs((size_t)L * L, make_uint2(0, 0));
  for (int level = 2; level <= L; level++)
    for (int i = 0; i < level - 1; i++) rs[(size_t)(level - 1) * L + i] = h_pair(h_inv(pr[level - 1] % pr[i], pr[i]), pr[i]);
  CUDA_OR_FAIL(upload(&c->d_rs_qinv, rs));

  c->table_bytes = sizeof(PrimeC) * NP + 2 * sizeof(uint2) * (size_t)NP * N + sizeof(uint2) * (size_t)(4 * L * L + 3 * K + 2 * L) +
                   sizeof(uint32_t) * (size_t)L * K;
  c->tabs.ntt.pc = c->d_pc;
  c->tabs.ntt.tw_fwd = c->d_tw;
  c->tabs.ntt.tw_inv = c->d_itw;
  c->tabs.ntt.ninv = c->d_ninv;
  c->tabs.pc = c->d_pc;
  c->tabs.logn = c->logn;
  c->tabs.tracer = nullptr;
  c->tabs.ip_ctas_per_sm = 2;
  c->tabs.ntt_otf = 0;
  c->tabs.ntt_single = 0;
  c->tabs.ntt_stream = 0;
  c->tabs.ntt_persist = 0;
  c->tabs.ntt_stream_stages = 3;
  c->tabs.ntt_stream_ctas = 3;
  c->tabs.bconv_tc_ctas = 4;
  c->tabs.bconv_tc_pipe = 0;
  c->tabs.ip_staged = 1;
  c->tabs.ip_staged_ctas = 2;
  c->tabs.ip_staged_depth = 0;
  c->tabs.status = c->d_status;
  return FHE_OK;
}

int ensure_lanes(fhe_ctx *c, int n) {
  while ((int)c->lanes.size() < n) {
    fhe_ctx::Lane l;
    if (c->lanes.empty()) {
      l.aux = c->aux;
      l.fork = c->ev_fork;
      l.join = c->ev_join;
    } else {
      CUDA_OR_FAIL(cudaStreamCreateWithFlags(&l.aux, cudaStreamNonBlocking));
      CUDA_OR_FAIL(cudaEventCreateWithFlags(&l.fork, cudaEventDisableTiming));
      CUDA_OR_FAIL(cudaEventCreateWithFlags(&l.join, cudaEventDisableTiming));
    }
    CUDA_OR_FAIL(cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking));
    CUDA_OR_FAIL(cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming));
    c->lanes.push_back(l);
  }
  return FHE_OK;
}

int fhe_ctx::reserve(size_t bytes, const char *what) {
  if (mem_limit && grown_bytes + bytes > mem_limit)
    return fhe_fail(FHE_ENOMEM, "%s: %zu more bytes exceed the context's memory limit (%zu of %zu in use)", what,
                    bytes, grown_bytes, mem_limit);
  return FHE_OK;
}

int ensure_slots(fhe_ctx *c, int n) {
  const size_t N = c->N;
  const int L = c->L, K = c->K, B = c->beta(L);
  const size_t limbs = (size_t)L + (size_t)B * (L + K) + 2 * (L + K) + 2 * K + 2 * L + 3 * L + 2 * L + 2;
  c->slot_bytes = limbs * N * sizeof(uint32_t);
  while ((int)c->slots.size() < n) {
    fhe_ctx::Slot s;
    const int rc = c->reserve(c->slot_bytes, "workspace slot");
    if (rc != FHE_OK) return rc;
    CUDA_OR_FAIL(cudaMalloc(&s.base, c->slot_bytes));
    c->grown_bytes += c->slot_bytes;
    uint32_t *p = s.base;
    auto take = [&](size_t l) {
      uint32_t *r = p;
      p += l * N;
      return r;
    };
    s.Y = take(L);
    s.EXT = take((size_t)B * (L + K));
    s.U = take(2 * (L + K));
    s.UC = take(2 * K);
    s.R = take(2 * L);
    s.D = take(3 * L);
    s.TMP = take(2 * L);
    s.V = take(2);
    c->slots.push_back(s);
    c->ws_bytes += c->slot_bytes;
  }
  return FHE_OK;
}

fhe_ctx::~fhe_ctx() {
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  cudaFree(d_pc);
  cudaFree(d_tw);
  cudaFree(d_itw);
  cudaFree(d_ninv);
  cudaFree(d_mu_scale);
  cudaFree(d_mu_qhinv);
  for (auto p : modup_T) cudaFree(p);
  for (auto p : modup_map) cudaFree(p);
  for (auto p : modup_Btc) cudaFree(p);
  cudaFree(d_md_Btc);
  cudaFree(d_status);
  cudaFree(d_md_scale);
  cudaFree(d_md_phinv);
  cudaFree(d_pinv);
  cudaFree(d_pmod);
  cudaFree(d_gbar);
  cudaFree(d_mdT);
  cudaFree(d_mdmap);
  cudaFree(d_rs_qinv);
  for (auto &s : slots) cudaFree(s.base);
  cudaFree(lt_scratch);
  cudaFree(relin_key);
  for (auto &kv : rot_keys) cudaFree(kv.second);
  for (auto &kv : bconv_prep) cudaFree(kv.second.block);
  cudaFree(bconv_y);
  if (order_ev) cudaEventDestroy(order_ev);
  for (size_t i = 0; i < lanes.size(); i++) {
    if (i > 0) {
      cudaStreamDestroy(lanes[i].aux);
      cudaEventDestroy(lanes[i].fork);
      cudaEventDestroy(lanes[i].join);
    }
    cudaStreamDestroy(lanes[i].stream);
    cudaEventDestroy(lanes[i].done);
  }
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
  if (aux) cudaStreamDestroy(aux);
  if (prev >= 0) cudaSetDevice(prev);
}

extern "C" int fhe_ctx_create(fhe_ctx **out, uint32_t N, const uint32_t *q, int L, const uint32_t *p, int K, int dnum,
                              int device) {
  if (!out) return fhe_fail(FHE_EINVAL, "fhe_ctx_create: out is null");
  *out = nullptr;
  if (!q || !p) return fhe_fail(FHE_EINVAL, "fhe_ctx_create: null prime list");
  if (N != 4096u && N != 65536u)
    return fhe_fail(FHE_EUNSUPPORTED, "fhe_ctx_create: N=%u (supported: 2^12, 2^16)", N);
  if (L < 1 || K < 1 || L + K > FHE_MAX_PRIMES)
    return fhe_fail(FHE_EINVAL, "fhe_ctx_create: L=%d K=%d (need L,K >= 1, L+K <= %d)", L, K, FHE_MAX_PRIMES);
  if (dnum < 1 || dnum > L) return fhe_fail(FHE_EINVAL, "fhe_ctx_create: dnum=%d outside [1, L=%d]", dnum, L);
  const int alpha = ceil_div(L, dnum);
  if (alpha > 16 || K > 16)
    return fhe_fail(FHE_EUNSUPPORTED, "fhe_ctx_create: alpha=%d, K=%d (base conversion supports <= 16 inputs)", alpha, K);
  if (ceil_div(L, alpha) > 4)
    return fhe_fail(FHE_EUNSUPPORTED, "fhe_ctx_create: beta=%d digits (inner product supports <= 4)", ceil_div(L, alpha));
  if (L + K - 1 > 64 || L > 64) return fhe_fail(FHE_EUNSUPPORTED, "fhe_ctx_create: too many limbs");
  std::vector<uint32_t> pr(q, q + L);
  pr.insert(pr.end(), p, p + K);
  for (int i = 0; i < L + K; i++) {
    const uint32_t x = pr[i];
    if (x >= (1u << 31) || x <= (1u << 20) || x % (2u * N) != 1 || !h_is_prime(x))
      return fhe_fail(FHE_EPRIME, "fhe_ctx_create: prime %d = %u is not a prime = 1 mod 2N in (2^20, 2^31)", i, x);
    for (int k = 0; k < i; k++)
      if (pr[k] == x) return fhe_fail(FHE_EPRIME, "fhe_ctx_create: prime %u repeated", x);
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return fhe_fail(FHE_ECUDA, "fhe_ctx_create: no CUDA device %d", device);
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return fhe_fail(FHE_ECUDA, "fhe_ctx_create: cudaSetDevice(%d)", device);
  fhe_ctx *c = new fhe_ctx();
  c->device = device;
  c->N = N;
  c->logn = N == 4096u ? 12 : 16;
  c->L = L;
  c->K = K;
  c->dnum = dnum;
  c->alpha = alpha;
  c->primes = pr;
  int rc = build_tables(c);
  if (rc == FHE_OK) rc = ensure_slots(c, 1);
  if (rc == FHE_OK && (cudaEventCreateWithFlags(&c->order_ev, cudaEventDisableTiming) != cudaSuccess ||
                       cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                       cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
                       cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) != cudaSuccess))
    rc = fhe_fail(FHE_ECUDA, "fhe_ctx_create: events / auxiliary stream");
  if (rc == FHE_OK) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = fhe_fail(FHE_ECUDA, "fhe_ctx_create: %s", cudaGetErrorString(e));
  }
  if (rc != FHE_OK) {
    delete c;
  } else {
    *out = c;
  }
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}

extern "C" int fhe_ctx_destroy(fhe_ctx *ctx) {
  if (!ctx) return fhe_fail(FHE_EINVAL, "fhe_ctx_destroy: null");
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  delete ctx;
  return FHE_OK;
}

extern "C" int fhe_ctx_info(const fhe_ctx *c, fhe_info *o) {
  if (!c || !o) return fhe_fail(FHE_EINVAL, "fhe_ctx_info: null");
  memset(o, 0, sizeof *o);
  o->N = c->N;
  o->L = c->L;
  o->K = c->K;
  o->dnum = c->dnum;
  o->alpha = c->alpha;
  o->device = c->device;
  o->limb_bytes = (size_t)4 * c->N;
  o->key_bytes = (size_t)c->dnum * 2 * (c->L + c->K) * o->limb_bytes;
  o->workspace_bytes = c->ws_bytes;
  o->table_bytes = c->table_bytes;
  o->n_rot_keys = (int)c->rot_keys.size();
  o->bconv_mode = c->bconv_mode;
  for (int i = 0; i < c->L + c->K; i++) o->psi[i] = c->psi[i];
  return FHE_OK;
}

extern "C" int fhe_ctx_set_bconv(fhe_ctx *c, int mode) {
  if (!c) return fhe_fail(FHE_EINVAL, "fhe_ctx_set_bconv: null");
  if (mode != FHE_BCONV_SCALAR && mode != FHE_BCONV_TC) return fhe_fail(FHE_EINVAL, "fhe_ctx_set_bconv: mode %d", mode);
  if (mode == FHE_BCONV_TC && !fhe_tc_available())
    return fhe_fail(FHE_EUNSUPPORTED, "fhe_ctx_set_bconv: tensor-core base conversion not built");
  if (mode == FHE_BCONV_TC && !c->tabs.tc_k)
    return fhe_fail(FHE_EUNSUPPORTED, "fhe_ctx_set_bconv: tensor-core base conversion needs alpha <= %d and K <= %d",
                    fhe::kTcMaxIn12, fhe::kTcMaxIn12);
  c->bconv_mode = mode;
  return FHE_OK;
}

extern "C" int fhe_trace_enable(fhe_ctx *c, int on) {
  if (!c) return fhe_fail(FHE_EINVAL, "fhe_trace_enable: null");
  if (c->capturing) return fhe_fail(FHE_EINVAL, "fhe_trace_enable: a plan is being captured");
  c->tabs.tracer = on ? &c->tracer : nullptr;
  return FHE_OK;
}

extern "C" int fhe_trace_read(fhe_ctx *c, fhe_kernel_stat *out, int max, int *n) {
  if (!c || !n || (max > 0 && !out)) return fhe_fail(FHE_EINVAL, "fhe_trace_read: bad arguments");
  cudaSetDevice(c->device);
  CUDA_OR_FAIL(cudaDeviceSynchronize());
  std::vector<fhe_kernel_stat> agg;
  for (const auto &r : c->tracer.recs) {
    float ms = 0.f;
    CUDA_OR_FAIL(cudaEventElapsedTime(&ms, r.a, r.b));
    size_t i = 0;
    for (; i < agg.size(); i++)
      if (!strncmp(agg[i].name, r.name, sizeof agg[i].name)) break;
    if (i == agg.size()) {
      fhe_kernel_stat z;
      memset(&z, 0, sizeof z);
      strncpy(z.name, r.name, sizeof z.name - 1);
      agg.push_back(z);
    }
    agg[i].launches++;
    agg[i].total_ms += ms;
  }
  c->tracer.reset();
  *n = (int)agg.size();
  for (int i = 0; i < max && i < (int)agg.size(); i++) out[i] = agg[i];
  return FHE_OK;
}

extern "C" int fhe_ctx_sync(fhe_ctx *c) {
  if (!c) return fhe_fail(FHE_EINVAL, "fhe_ctx_sync: null");
  cudaSetDevice(c->device);
  CUDA_OR_FAIL(cudaDeviceSynchronize());
  unsigned int st = 0;
  CUDA_OR_FAIL(cudaMemcpy(&st, c->d_status, sizeof st, cudaMemcpyDeviceToHost));
  if (st) {
    const unsigned int zero = 0;
    CUDA_OR_FAIL(cudaMemcpy(c->d_status, &zero, sizeof zero, cudaMemcpyHostToDevice));
    return fhe_fail(FHE_ETIMEOUT, "fhe_ctx_sync: a bounded device-side wait expired (status 0x%x)", st);
  }
  return FHE_OK;
}

extern "C" int fhe_ctx_set_pipelining(fhe_ctx *c, int on) {
  if (!c) return fhe_fail(FHE_EINVAL, "fhe_ctx_set_pipelining: null");
  c->comp_pipe = on ? 1 : 0;
  return FHE_OK;
}

extern "C" int fhe_ctx_set_ntt(fhe_ctx *c, int flags) {
  if (!c) return fhe_fail(FHE_EINVAL, "fhe_ctx_set_ntt: null");
  if (flags & ~(FHE_NTT_OTF | FHE_NTT_SINGLE_PASS | FHE_NTT_STREAM | FHE_NTT_PERSIST))
    return fhe_fail(FHE_EINVAL, "fhe_ctx_set_ntt: flags 0x%x", flags);
  if ((flags & FHE_NTT_PERSIST) && (flags & (FHE_NTT_OTF | FHE_NTT_SINGLE_PASS | FHE_NTT_STREAM)))
    return fhe_fail(FHE_EINVAL, "fhe_ctx_set_ntt: FHE_NTT_PERSIST combines with no other flag (0x%x)", flags);
  if ((flags & FHE_NTT_PERSIST) && c->logn != 16)
    return fhe_fail(FHE_EUNSUPPORTED, "fhe_ctx_set_ntt: the persistent NTT needs N = 2^16");
  if ((flags & FHE_NTT_STREAM) && c->logn != 16)
    return fhe_fail(FHE_EUNSUPPORTED, "fhe_ctx_set_ntt: the streaming NTT passes need N = 2^16");
  if (flags & FHE_NTT_SINGLE_PASS) {
    if (c->logn != 16) return fhe_fail(FHE_EUNSUPPORTED, "fhe_ctx_set_ntt: the single-pass NTT needs N = 2^16");
    cudaSetDevice(c->device);
    if (fhe::ntt_single_pass_clusters() < 1)
      return fhe_fail(FHE_EUNSUPPORTED, "fhe_ctx_set_ntt: no 16-CTA cluster of the single-pass NTT fits this device");
  }
  c->tabs.ntt_otf = (flags & FHE_NTT_OTF) ? 1 : 0;
  c->tabs.ntt_single = (flags & FHE_NTT_SINGLE_PASS) ? 1 : 0;
  c->tabs.ntt_stream = (flags & FHE_NTT_STREAM) ? 1 : 0;
  c->tabs.ntt_persist = (flags & FHE_NTT_PERSIST) ? 1 : 0;
  return FHE_OK;
}

extern "C" int fhe_ctx_set_kernel_shape(fhe_ctx *c, const fhe_kernel_shape *sh) {
  if (!c || !sh) return fhe_fail(FHE_EINVAL, "fhe_ctx_set_kernel_shape: null");
  if ((sh->fuse_ip_moddown != 0 && sh->fuse_ip_moddown != 1) || sh->bconv_tc_ctas < 1 || sh->bconv_tc_ctas > 4 ||
      sh->ntt_stream_stages < 2 || sh->ntt_stream_stages > 3 || sh->ntt_stream_ctas < 1 || sh->ntt_stream_ctas > 3 ||
      (sh->bconv_tc_pipeline != 0 && sh->bconv_tc_pipeline != 1) ||
      (sh->ip_staged_gather != 0 && sh->ip_staged_gather != 1) || sh->ip_staged_ctas < 1 || sh->ip_staged_ctas > 2 ||
      sh->ip_staged_depth < 0 || sh->ip_staged_depth == 1 || sh->ip_staged_depth > 4)
    return fhe_fail(FHE_EINVAL, "fhe_ctx_set_kernel_shape: fuse %d (0, 1), bconv_tc_ctas %d (1..4), stages %d (2..3), "
                    "stream ctas %d (1..3), pipeline %d (0, 1), staged gather %d (0, 1), staged ctas %d (1, 2), "
                    "staged depth %d (0, 2..4)", sh->fuse_ip_moddown, sh->bconv_tc_ctas, sh->ntt_stream_stages,
                    sh->ntt_stream_ctas, sh->bconv_tc_pipeline, sh->ip_staged_gather, sh->ip_staged_ctas,
                    sh->ip_staged_depth);
  if (sh->fuse_ip_moddown && c->logn != 16)
    return fhe_fail(FHE_EUNSUPPORTED, "fhe_ctx_set_kernel_shape: the fused inner product needs N = 2^16");
  c->fuse_ip_md = sh->fuse_ip_moddown;
  c->tabs.bconv_tc_ctas = sh->bconv_tc_ctas;
  c->tabs.ntt_stream_stages = sh->ntt_stream_stages;
  c->tabs.ntt_stream_ctas = sh->ntt_stream_ctas;
  c->tabs.bconv_tc_pipe = sh->bconv_tc_pipeline;
  c->tabs.ip_staged = sh->ip_staged_gather;
  c->tabs.ip_staged_ctas = sh->ip_staged_ctas;
  c->tabs.ip_staged_depth = sh->ip_staged_depth;
  return FHE_OK;
}

extern "C" int fhe_ctx_get_kernel_shape(const fhe_ctx *c, fhe_kernel_shape *out) {
  if (!c || !out) return fhe_fail(FHE_EINVAL, "fhe_ctx_get_kernel_shape: null");
  out->fuse_ip_moddown = c->fuse_ip_md;
  out->bconv_tc_ctas = c->tabs.bconv_tc_ctas;
  out->ntt_stream_stages = c->tabs.ntt_stream_stages;
  out->ntt_stream_ctas = c->tabs.ntt_stream_ctas;
  out->bconv_tc_pipeline = c->tabs.bconv_tc_pipe;
  out->ip_staged_gather = c->tabs.ip_staged;
  out->ip_staged_ctas = c->tabs.ip_staged_ctas;
  out->ip_staged_depth = c->tabs.ip_staged_depth;
  return FHE_OK;
}

extern "C" int fhe_ctx_set_memory_limit(fhe_ctx *c, size_t bytes) {
  if (!c) return fhe_fail(FHE_EINVAL, "fhe_ctx_set_memory_limit: null");
  c->mem_limit = bytes;
  return FHE_OK;
}

extern "C" int fhe_ctx_set_fused(fhe_ctx *c, int fused) {
  if (!c) return fhe_fail(FHE_EINVAL, "fhe_ctx_set_fused: null");
  c->fused = fused ? 1 : 0;
  return FHE_OK;
}

// ---------------------------------------------------------------- keys
uint32_t fhe_galois_elt(int32_t rot, uint32_t N) {
  const int64_t half = N / 2;
  int64_t r = rot % half;
  if (r < 0) r += half;
  return h_pow(5, (uint64_t)r, 2 * N);
}

static int set_key(fhe_ctx *c, uint32_t **slot, const uint32_t *key, cudaStream_t s) {
  const size_t bytes = (size_t)c->dnum * 2 * (c->L + c->K) * c->N * sizeof(uint32_t);
  if (!*slot) {
    const int rc = c->reserve(bytes, "switching key");
    if (rc != FHE_OK) return rc;
    CUDA_OR_FAIL(cudaMalloc(slot, bytes));
    c->grown_bytes += bytes;
  }
  c->order_stream(s);
  CUDA_OR_FAIL(cudaMemcpyAsync(*slot, key, bytes, cudaMemcpyDefault, s));
  return FHE_OK;
}

extern "C" int fhe_set_relin_key(fhe_ctx *c, const uint32_t *key, fhe_stream stream) {
  if (!c || !key) return fhe_fail(FHE_EINVAL, "fhe_set_relin_key: null argument");
  cudaSetDevice(c->device);
  return set_key(c, &c->relin_key, key, (cudaStream_t)stream);
}

extern "C" int fhe_set_rot_key(fhe_ctx *c, int32_t rot, const uint32_t *key, fhe_stream stream) {
  if (!c || !key) return fhe_fail(FHE_EINVAL, "fhe_set_rot_key: null argument");
  const uint32_t k = fhe_galois_elt(rot, c->N);
  if (k == 1) return fhe_fail(FHE_EINVAL, "fhe_set_rot_key: rotation %d is the identity", rot);
  cudaSetDevice(c->device);
  uint32_t *&slot = c->rot_keys[k];
  return set_key(c, &slot, key, (cudaStream_t)stream);
}

const uint32_t *fhe_ctx::find_key(int32_t key_id) const {
  if (key_id == FHE_RELIN_KEY) return relin_key;
  auto it = rot_keys.find(fhe_galois_elt(key_id, N));
  return it == rot_keys.end() ? nullptr : it->second;
}
