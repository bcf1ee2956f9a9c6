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
  int comp_pipe = 1;  // complementary pipelining of the inner product (autotuned)
  int fuse_ip_md = 0; // special limbs' inner product fused with ModDown's first INTT pass (autotuned)
  size_t batch_budget = 0;  // L2 bytes per batched group (0: 3/4 of the L2 size)
  int batch_max_group = 0;  // items per batched group (0: 8)

  // device tables
  fhe::PrimeC *d_pc = nullptr;
  uint2 *d_tw = nullptr, *d_itw = nullptr, *d_ninv = nullptr;
  uint2 *d_mu_scale = nullptr;  // [L][L]: N^-1 (D/q_t)^-1 mod q_t at level l (row l-1)
  uint2 *d_mu_qhinv = nullptr;  // [L][L]: (D/q_t)^-1 mod q_t
  std::vector<uint32_t *> modup_T;  // [(level-1)*dnum + j]: BConv table, rows in ext-limb order
  std::vector<int2 *> modup_map;    // same index: (ext limb, prime) per row
  std::vector<uint16_t *> modup_Btc; // same index: byte-digit table of the tensor-core conversion
  uint2 *d_md_scale = nullptr, *d_md_phinv = nullptr;  // [K]
  uint2 *d_pinv = nullptr;                             // [L] P^-1 mod q_i
  uint32_t *d_mdT = nullptr;                           // [L][K] (P/p_k) mod q_i
  int2 *d_mdmap = nullptr;                             // [L] (i, i)
  uint16_t *d_md_Btc = nullptr;
  unsigned int *d_gbar = nullptr;                      // grid-barrier counters of the persistent NTT
  uint2 *d_pmod = nullptr;                             // [L] Shoup pairs of P mod q_i                        // tensor-core table of the ModDown conversion
  unsigned int *d_status = nullptr;                    // device status word (expired waits)
  uint2 *d_rs_qinv = nullptr;                          // [L][L]
  // fhe_bconv: the tables of each (input primes, output primes, kernel) combination, built and
  // uploaded by the first call that uses it and reused by later calls (one device block each)
  struct BconvPrep {
    void *block = nullptr;
    uint32_t *T = nullptr;
    int2 *om = nullptr;
    uint2 *pre = nullptr;
    uint16_t *Btc = nullptr;
  };
  std::map<std::vector<int>, BconvPrep> bconv_prep;
  uint32_t *bconv_y = nullptr;  // [16][N] fhe_bconv's pre-multiplied input
  size_t table_bytes = 0;
  fhe::DevTables tabs{};
  fhe::Tracer tracer;

  // keys
  uint32_t *relin_key = nullptr;
  std::map<uint32_t, uint32_t *> rot_keys;  // by Galois element

  // workspace: slots, each holding every scratch array of one key switch at level L
  struct Slot {
    uint32_t *base = nullptr;
    uint32_t *Y = nullptr;    // [L][N]        scaled INTT of the key-switched polynomial
    uint32_t *EXT = nullptr;  // [beta][L+K][N] ModUp outputs
    uint32_t *U = nullptr;    // [2][L+K][N]   inner product
    uint32_t *UC = nullptr;   // [2][K][N]     special limbs in coefficient form
    uint32_t *R = nullptr;    // [2][L][N]     ModDown base conversion
    uint32_t *D = nullptr;    // [3][L][N]     HMult tensor
    uint32_t *TMP = nullptr;  // [2][L][N]     plain-pipeline gather
    uint32_t *V = nullptr;    // [2][N]        rescale
  };
  std::vector<Slot> slots;
  size_t slot_bytes = 0;
  uint32_t *lt_scratch = nullptr;  // linear transform: baby / giant rotations and inner sums
  size_t lt_words = 0;
  size_t ws_bytes = 0;
  // growable device memory (workspace slots, transform scratch, key copies) and its cap
  // (0: none); growth past the cap fails with FHE_ENOMEM before any allocation
  size_t grown_bytes = 0, mem_limit = 0;
  int reserve(size_t bytes, const char *what);

  // cross-stream ordering of calls on this context
  cudaStream_t last_stream = nullptr;
  bool have_last = false;
  bool capturing = false;  // a batched plan is being captured: no cross-stream ordering
  cudaEvent_t order_ev = nullptr;
  cudaStream_t aux = nullptr;  // concurrent branch of the fused pipeline
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // batched plans run their item groups on several lanes; each lane has its own
  // stream, auxiliary stream and fork / join events (lane 0 reuses aux / ev_fork / ev_join)
  struct Lane {
    cudaStream_t stream = nullptr, aux = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, done = nullptr;
  };
  std::vector<Lane> lanes;
  int batch_lanes = 2;

  int beta(int level) const;
  int ext_prime(int level, int t) const;
  void order_stream(cudaStream_t s);
  const uint32_t *find_key(int32_t key_id) const;
  ~fhe_ctx();
};

int fhe_fail(int code, const char *fmt, ...);
uint32_t h_mulmod_pub(uint32_t a, uint32_t b, uint32_t q);
uint32_t h_invmod_pub(uint32_t a, uint32_t q);
int ensure_slots(fhe_ctx *c, int n);
int ensure_lanes(fhe_ctx *c, int n);
uint32_t fhe_galois_elt(int32_t rot, uint32_t N);
bool fhe_tc_available();
