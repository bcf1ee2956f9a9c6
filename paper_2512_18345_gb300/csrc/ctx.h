// The context object behind the opaque fhe_ctx handle (host-side definition).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <vector>

#include "internal.h"

struct fhe_ctx {
  int device = 0;
  uint32_t N = 0;
  int logn = 0, L = 0, K = 0, dnum = 0, alpha = 0;
  std::vector<uint32_t> primes;  // q_0..q_{L-1}, p_0..p_{K-1}
  uint32_t psi[64] = {};
  int bconv_mode = 0;  // FHE_BCONV_SCALAR / FHE_BCONV_TC
  int fused = 1;

  // device tables
  fhe::PrimeC *d_pc = nullptr;
  uint2 *d_tw = nullptr, *d_itw = nullptr, *d_ninv = nullptr;
  uint2 *d_mu_scale = nullptr;  // [L][L]: N^-1 (D/q_t)^-1 mod q_t at level l (row l-1)
  uint2 *d_mu_qhinv = nullptr;  // [L][L]: (D/q_t)^-1 mod q_t
  std::vector<uint32_t *> modup_T;  // [(level-1)*dnum + j]: BConv table, rows in ext-limb order
  std::vector<int2 *> modup_map;    // same index: (ext limb, prime) per row
  uint2 *d_md_scale = nullptr, *d_md_phinv = nullptr;  // [K]
  uint2 *d_pinv = nullptr;                             // [L] P^-1 mod q_i
  uint32_t *d_mdT = nullptr;                           // [L][K] (P/p_k) mod q_i
  int2 *d_mdmap = nullptr;                             // [L] (i, i)
  uint2 *d_rs_qinv = nullptr;                          // [L][L]
  std::vector<void *> scratch_tabs;                    // tables built for fhe_bconv calls
  size_t table_bytes = 0;
  fhe::DevTables tabs{};
  fhe::Tracer tracer;

  // keys
  uint32_t *relin_key = nullptr;
  std::map<uint32_t, uint32_t *> rot_keys;  // by Galois element

  // workspace
  uint32_t *ws = nullptr;
  size_t ws_bytes = 0;
  uint32_t *wY = nullptr, *wEXT = nullptr, *wUC = nullptr, *wR = nullptr, *wD = nullptr, *wU = nullptr,
           *wTMP = nullptr, *wV = nullptr;

  // cross-stream ordering of calls on this context
  cudaStream_t last_stream = nullptr;
  bool have_last = false;
  bool capturing = false;  // a batched plan is being captured: no cross-stream ordering
  cudaEvent_t order_ev = nullptr;
  cudaStream_t aux = nullptr;  // concurrent branch of the fused pipeline
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  int beta(int level) const;
  int ext_prime(int level, int t) const;
  void order_stream(cudaStream_t s);
  const uint32_t *find_key(int32_t key_id) const;
  ~fhe_ctx();
};

int fhe_fail(int code, const char *fmt, ...);
uint32_t h_mulmod_pub(uint32_t a, uint32_t b, uint32_t q);
uint32_t h_invmod_pub(uint32_t a, uint32_t q);
// pipelines shared with the batched plans
int run_modup(fhe_ctx *c, const uint32_t *d, int level, uint32_t galois_d, uint32_t *ext, cudaStream_t s);
int run_moddown(fhe_ctx *c, fhe::KsArgs ks, int level, uint32_t *out, cudaStream_t s);
uint32_t fhe_galois_elt(int32_t rot, uint32_t N);
bool fhe_tc_available();
