// Allocation-free base conversion: fhe_bconv_noalloc.
//
// fhe_bconv keeps its tables and its pre-multiplied input in device memory
// that the context allocates on first use.  Some callers cannot allocate once
// they are running: a process whose framework has reserved all free device
// memory for its own pool (cudaMalloc then fails), or a real-time loop that
// must not take cudaMalloc's implicit device-wide synchronization.  This
// variant computes exactly the same conversion with no allocation: its
// scratch (the pre-multiplied input and the tables) lives in one fixed,
// file-scope device array that every GPU loading the library keeps until the
// process exits.  The tables reach the GPU as the argument of a small kernel
// that writes them into the array, so no host memory is read after the call
// returns.
#include <cstring>
#include <mutex>

#include "../../include/fhe.h"
#include "ctx.h"
#include "elementwise.cuh"
#include "internal.h"

using namespace fhe;

namespace {
constexpr int kMaxIn = FHE_BCONV_NOALLOC_MAX_IN;
constexpr int kMaxOut = FHE_BCONV_NOALLOC_MAX_OUT;
constexpr size_t kMaxN = FHE_BCONV_NOALLOC_MAX_N;
// scratch layout, in 32-bit words: y [kMaxIn][kMaxN] | T [kMaxOut][kMaxIn] | omap [kMaxOut] int2 | pre [kMaxIn] uint2
constexpr size_t kOffT = (size_t)kMaxIn * kMaxN;
constexpr size_t kOffMap = kOffT + (size_t)kMaxOut * kMaxIn;
constexpr size_t kOffPre = kOffMap + 2 * (size_t)kMaxOut;
constexpr size_t kWords = kOffPre + 2 * (size_t)kMaxIn;
constexpr int kMaxDevices = 64;
}  // namespace

// The shared scratch.  In host code this name is only a stand-in for the
// device symbol: the device address is obtained with cudaGetSymbolAddress.
static __device__ __align__(256) uint32_t g_bconv_scratch[kWords];

// The conversion tables of one call, passed by value to the kernel that stores them.
struct NoallocTables {
  uint32_t T[kMaxOut * kMaxIn];  // T[o][j] = (Qstar/q_j) mod p_o
  int2 om[kMaxOut];              // (output row, prime index)
  uint2 pre[kMaxIn];             // ((Qstar/q_j)^-1 mod q_j, Shoup companion)
  int n_in, n_out;
};

// Writes a call's tables into the shared scratch (device code names the array directly).
__global__ void k_noalloc_tables(const __grid_constant__ NoallocTables t) {
  const int nT = t.n_out * t.n_in;
  for (int i = threadIdx.x; i < nT; i += blockDim.x) g_bconv_scratch[kOffT + i] = t.T[i];
  for (int i = threadIdx.x; i < t.n_out; i += blockDim.x) {
    g_bconv_scratch[kOffMap + 2 * i] = (uint32_t)t.om[i].x;
    g_bconv_scratch[kOffMap + 2 * i + 1] = (uint32_t)t.om[i].y;
  }
  for (int i = threadIdx.x; i < t.n_in; i += blockDim.x) {
    g_bconv_scratch[kOffPre + 2 * i] = t.pre[i].x;
    g_bconv_scratch[kOffPre + 2 * i + 1] = t.pre[i].y;
  }
}

static uint32_t *g_scratch_addr[kMaxDevices];
static cudaError_t g_scratch_err[kMaxDevices];
static std::once_flag g_scratch_once[kMaxDevices];

// Device address of the scratch on `device` (which must be current); set up on first use.
static uint32_t *scratch_address(int device, cudaError_t &err) {
  std::call_once(g_scratch_once[device], [device]() {
    void *p = nullptr;
    g_scratch_err[device] = cudaGetSymbolAddress(&p, g_bconv_scratch);
    g_scratch_addr[device] = static_cast<uint32_t *>(p);
  });
  err = g_scratch_err[device];
  return g_scratch_addr[device];
}

extern "C" int fhe_bconv_noalloc(fhe_ctx *c, const uint32_t *in, const int *in_idx, int n_in, uint32_t *out,
                                 const int *out_idx, int n_out, fhe_stream stream) {
  if (!c) return fhe_fail(FHE_EINVAL, "fhe_bconv_noalloc: null ctx");
  if (!in || !out || !in_idx || !out_idx) return fhe_fail(FHE_EINVAL, "fhe_bconv_noalloc: null argument");
  if (((uintptr_t)in | (uintptr_t)out) & 15) return fhe_fail(FHE_EINVAL, "fhe_bconv_noalloc: buffers must be 16-byte aligned");
  if (n_in < 1 || n_in > kMaxIn || n_out < 1 || n_out > kMaxOut || c->N > kMaxN)
    return fhe_fail(FHE_EINVAL,
                    "fhe_bconv_noalloc: n_in=%d, n_out=%d, N=%u exceed the fixed scratch (n_in <= %d, n_out <= %d, "
                    "N <= %zu); use fhe_bconv",
                    n_in, n_out, c->N, kMaxIn, kMaxOut, kMaxN);
  if (c->device < 0 || c->device >= kMaxDevices) return fhe_fail(FHE_EINVAL, "fhe_bconv_noalloc: device %d", c->device);
  const int NP = c->L + c->K;
  for (int i = 0; i < n_in; i++)
    if (in_idx[i] < 0 || in_idx[i] >= NP) return fhe_fail(FHE_EINVAL, "fhe_bconv_noalloc: in prime index %d", in_idx[i]);
  for (int i = 0; i < n_out; i++)
    if (out_idx[i] < 0 || out_idx[i] >= NP) return fhe_fail(FHE_EINVAL, "fhe_bconv_noalloc: out prime index %d", out_idx[i]);
  const size_t N = c->N;
  const char *ib = (const char *)in, *ob = (const char *)out;
  if (ib < ob + 4 * N * n_out && ob < ib + 4 * N * n_in) return fhe_fail(FHE_EALIAS, "fhe_bconv_noalloc: out overlaps in");

  // the tables: pre-factor (Qstar/q_j)^-1 mod q_j, T[o][j] = (Qstar/q_j) mod p_o
  const std::vector<uint32_t> &pr = c->primes;
  NoallocTables tabs;
  memset(&tabs, 0, sizeof tabs);
  tabs.n_in = n_in;
  tabs.n_out = n_out;
  uint32_t *T = tabs.T;
  int2 *om = tabs.om;
  uint2 *pre = tabs.pre;
  for (int j = 0; j < n_in; j++) {
    const uint32_t q = pr[in_idx[j]];
    uint32_t prod = 1;
    for (int k = 0; k < n_in; k++)
      if (k != j) prod = h_mulmod_pub(prod, pr[in_idx[k]] % q, q);
    const uint32_t w = h_invmod_pub(prod, q);
    pre[j] = make_uint2(w, (uint32_t)(((uint64_t)w << 32) / q));
  }
  for (int o = 0; o < n_out; o++) {
    const uint32_t p = pr[out_idx[o]];
    for (int j = 0; j < n_in; j++) {
      uint32_t prod = 1;
      for (int k = 0; k < n_in; k++)
        if (k != j) prod = h_mulmod_pub(prod, pr[in_idx[k]] % p, p);
      T[o * n_in + j] = prod;
    }
    om[o] = make_int2(o, out_idx[o]);
  }

  if (cudaSetDevice(c->device) != cudaSuccess) return fhe_fail(FHE_ECUDA, "fhe_bconv_noalloc: cudaSetDevice");
  cudaError_t err;
  uint32_t *base = scratch_address(c->device, err);
  if (err != cudaSuccess || !base)
    return fhe_fail(FHE_ECUDA, "fhe_bconv_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(err));
  uint32_t *y = base, *dT = base + kOffT;
  int2 *dM = reinterpret_cast<int2 *>(base + kOffMap);
  uint2 *dPre = reinterpret_cast<uint2 *>(base + kOffPre);
  cudaStream_t s = (cudaStream_t)stream;
  c->order_stream(s);
  // every scratch word the kernels read is written first by this call: nothing needs clearing
  k_noalloc_tables<<<1, 256, 0, s>>>(tabs);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fhe_fail(FHE_ECUDA, "fhe_bconv_noalloc: tables: %s", cudaGetErrorString(e));
  SegList sl;
  memset(&sl, 0, sizeof sl);
  for (int j = 0; j < n_in; j++) {
    Seg &x = sl.seg[sl.nseg++];
    x.src = in + (size_t)j * N;
    x.dst = y + (size_t)j * N;
    x.n = 1;
    x.prime = in_idx[j];
    x.src_stride = 1;
    x.src_prime = -1;
    x.scale = dPre + j;
    x.galois = 1;
    sl.total += 1;
  }
  e = launch_ew(c->tabs, EW_SCALE, sl, s);
  if (e != cudaSuccess) return fhe_fail(FHE_ECUDA, "fhe_bconv_noalloc: scale: %s", cudaGetErrorString(e));
  BconvArgs ba;
  memset(&ba, 0, sizeof ba);
  BconvGroup &g = ba.g[ba.ngroups++];
  g.in = y;
  g.out = out;
  g.T = dT;
  g.omap = dM;
  g.n_in = n_in;
  g.n_out = n_out;
  e = launch_bconv(c->tabs, ba, n_in, n_out, s);
  if (e != cudaSuccess) return fhe_fail(FHE_ECUDA, "fhe_bconv_noalloc: %s", cudaGetErrorString(e));
  return FHE_OK;
}
