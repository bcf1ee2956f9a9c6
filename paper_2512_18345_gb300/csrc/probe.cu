// Probes (measurement support).
//
// Bandwidth: read, write and read+write copy of a block of `bytes` repeated
// `reps` times with 128-bit L2-cached accesses, timed with CUDA events.  A
// block smaller than the L2 gives the L2 bandwidth (the paper's method: a
// block smaller than the L2 read and written repeatedly); a larger one gives
// the DRAM bandwidth.
//
// Integer pipes: register-only chains of the instruction mixes the kernels are
// built from -- the forward Shoup butterfly of the NTT passes, the 32 x 32 ->
// 64-bit multiply-accumulate of the base conversion and inner product, and
// single IMAD / IMAD.HI / add+min chains -- at four 256-thread CTAs per SM, so
// that the rates are what the pipes sustain with no memory traffic.  They are
// the denominators of the transforms' and conversions' ALU roofline fractions.
#include <vector>

#include "../../include/fhe.h"
#include "ctx.h"

namespace {
__global__ void k_probe_read(const uint4 *__restrict__ p, size_t n, int reps, unsigned int *sink) {
  uint32_t acc = 0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; r++)
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      const uint4 v = __ldcg(p + i);
      acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
  if (acc == 0x9E3779B9u) sink[0] = acc;  // keeps the loads alive
}
__global__ void k_probe_write(uint4 *__restrict__ p, size_t n, int reps) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; r++)
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
      __stcg(p + i, make_uint4((uint32_t)r, (uint32_t)i, 0u, 1u));
}
__global__ void k_probe_copy(const uint4 *__restrict__ a, uint4 *__restrict__ b, size_t n, int reps) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; r++)
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      uint4 v = __ldcg(a + i);
      v.x += (uint32_t)r;
      __stcg(b + i, v);
    }
}

constexpr uint32_t kProbeQ = 2147352577u;  // a 31-bit prime = 1 mod 2^17
constexpr int kProbeThreads = 256, kProbeCtasPerSm = 4;

__device__ __forceinline__ uint32_t probe_red2(uint32_t x) { return min(x, x - kProbeQ); }

// OP 0: forward butterflies, 4 radix-2 stages over 16 register values per iteration (32 per
//       thread), each t = red2(x2 w - hi(x2 w') q), u = red2(x1), (u + t, u - t + q);
// OP 1: 64-bit multiply-accumulate, 16 per iteration into 8 accumulators;
// OP 2: IMAD chains, OP 3: IMAD.HI chains (16 per iteration);
// OP 4: add + min pairs (16 per iteration).
// Thread 0 of each CTA stores its SM cycle count, the other values feed a sink that is
// written only on an impossible match (keeps the chains alive).
template <int OP>
__global__ void __launch_bounds__(kProbeThreads, kProbeCtasPerSm) k_probe_int(uint32_t seed, int iters, unsigned long long *cycles,
                                                             unsigned int *sink) {
  const long long c0 = clock64();
  uint32_t x[16];
  uint32_t w[8], ws[8];
#pragma unroll
  for (int e = 0; e < 16; e++) x[e] = (threadIdx.x * 2654435761u + (uint32_t)e * 40503u + seed) % kProbeQ;
#pragma unroll
  for (int k = 0; k < 8; k++) {
    w[k] = (seed * (uint32_t)(k + 3) + threadIdx.x * 977u) % kProbeQ;
    ws[k] = (uint32_t)(((uint64_t)w[k] << 32) / kProbeQ);
  }
  uint64_t acc[8];
#pragma unroll
  for (int e = 0; e < 8; e++) acc[e] = x[e];
  for (int it = 0; it < iters; it++) {
    if (OP == 0) {
#pragma unroll
      for (int bit = 3; bit >= 0; bit--)
#pragma unroll
        for (int e = 0; e < 16; e++) {
          if (e & (1 << bit)) continue;
          const int e2 = e | (1 << bit), k = (e >> (bit + 1)) & 7;
          const uint32_t t = probe_red2(x[e2] * w[k] - __umulhi(x[e2], ws[k]) * kProbeQ);
          const uint32_t u = probe_red2(x[e]);
          x[e] = u + t;
          x[e2] = u - t + kProbeQ;
        }
    } else if (OP == 1) {
#pragma unroll
      for (int e = 0; e < 16; e++) acc[e & 7] += (uint64_t)x[e] * w[e & 7];
#pragma unroll
      for (int e = 0; e < 16; e++) x[e] ^= (uint32_t)acc[(e + 1) & 7];
    } else if (OP == 2) {
#pragma unroll
      for (int e = 0; e < 16; e++) x[e] = x[e] * w[e & 7] + x[(e + 1) & 15];
    } else if (OP == 3) {
#pragma unroll
      for (int e = 0; e < 16; e++) x[e] = __umulhi(x[e], w[e & 7]) ^ x[(e + 1) & 15];
    } else {
#pragma unroll
      for (int e = 0; e < 16; e++) x[e] = min(x[e] + x[(e + 1) & 15], x[e] - kProbeQ);
    }
  }
  uint32_t r = 0;
#pragma unroll
  for (int e = 0; e < 16; e++) r ^= x[e] ^ (uint32_t)acc[e & 7] ^ (uint32_t)(acc[e & 7] >> 32);
  if (r == 0x9E3779B9u) sink[0] = r;
  if (threadIdx.x == 0) cycles[blockIdx.x] = (unsigned long long)(clock64() - c0);
}
}  // namespace

extern "C" int fhe_probe_int(int device, fhe_int_peaks *out) {
  if (!out) return fhe_fail(FHE_EINVAL, "fhe_probe_int: null output");
  if (cudaSetDevice(device) != cudaSuccess) return fhe_fail(FHE_ECUDA, "fhe_probe_int: device %d", device);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int grid = sms * kProbeCtasPerSm;
  unsigned long long *cyc = nullptr;
  unsigned int *sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&cyc, sizeof(unsigned long long) * grid) != cudaSuccess || cudaMalloc(&sink, 4) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaFree(cyc);
    cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return fhe_fail(FHE_ENOMEM, "fhe_probe_int: buffers");
  }
  // units per thread per iteration of each chain
  const double per_iter[5] = {32.0, 16.0, 16.0, 16.0, 16.0};
  const int iters[5] = {2048, 4096, 8192, 8192, 8192};
  double rate[5] = {0, 0, 0, 0, 0}, mhz_sum = 0;
  int rc = FHE_OK;
  std::vector<unsigned long long> hc(grid);
  for (int op = 0; op < 5 && rc == FHE_OK; op++) {
    float ms = 0.f;
    for (int rep = 0; rep < 2; rep++) {  // the first run warms up
      cudaEventRecord(e0);
      switch (op) {
        case 0: k_probe_int<0><<<grid, kProbeThreads>>>(7u + rep, iters[op], cyc, sink); break;
        case 1: k_probe_int<1><<<grid, kProbeThreads>>>(7u + rep, iters[op], cyc, sink); break;
        case 2: k_probe_int<2><<<grid, kProbeThreads>>>(7u + rep, iters[op], cyc, sink); break;
        case 3: k_probe_int<3><<<grid, kProbeThreads>>>(7u + rep, iters[op], cyc, sink); break;
        default: k_probe_int<4><<<grid, kProbeThreads>>>(7u + rep, iters[op], cyc, sink); break;
      }
      cudaEventRecord(e1);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = fhe_fail(FHE_ECUDA, "fhe_probe_int: kernel");
        break;
      }
      cudaEventElapsedTime(&ms, e0, e1);
    }
    if (rc != FHE_OK) break;
    rate[op] = (double)grid * kProbeThreads * iters[op] * per_iter[op] / (ms * 1e-3);
    cudaMemcpy(hc.data(), cyc, sizeof(unsigned long long) * grid, cudaMemcpyDeviceToHost);
    unsigned long long mx = 0;
    for (int i = 0; i < grid; i++) mx = hc[i] > mx ? hc[i] : mx;
    mhz_sum += (double)mx / (ms * 1e3);  // one wave: the longest CTA spans the kernel
  }
  if (rc == FHE_OK && cudaGetLastError() != cudaSuccess) rc = fhe_fail(FHE_ECUDA, "fhe_probe_int: kernels");
  if (rc == FHE_OK) {
    out->clock_mhz = mhz_sum / 5.0;
    out->butterflies_per_s = rate[0];
    out->mac64_per_s = rate[1];
    out->imad_per_s = rate[2];
    out->imad_hi_per_s = rate[3];
    out->add_min_per_s = rate[4];
    out->sms = sms;
  }
  cudaFree(cyc);
  cudaFree(sink);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

extern "C" int fhe_probe_bandwidth(int device, size_t bytes, int reps, double *read_gbs, double *write_gbs,
                                   double *copy_gbs) {
  if (bytes < (1u << 20) || reps < 1 || !read_gbs || !write_gbs || !copy_gbs)
    return fhe_fail(FHE_EINVAL, "fhe_probe_bandwidth: bytes >= 1 MiB, reps >= 1, non-null outputs");
  if (cudaSetDevice(device) != cudaSuccess) return fhe_fail(FHE_ECUDA, "fhe_probe_bandwidth: device %d", device);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  uint4 *a = nullptr, *b = nullptr;
  unsigned int *sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = FHE_OK;
  if (cudaMalloc(&a, bytes) != cudaSuccess || cudaMalloc(&b, bytes) != cudaSuccess ||
      cudaMalloc(&sink, 4) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    rc = fhe_fail(FHE_ENOMEM, "fhe_probe_bandwidth: buffers");
  const size_t n = bytes / 16;
  const unsigned grid = (unsigned)(4 * sms);
  float ms = 0.f;
  if (rc == FHE_OK) {
    cudaMemset(a, 1, bytes);
    cudaMemset(b, 2, bytes);
    k_probe_read<<<grid, 512>>>(a, n, 1, sink);
    cudaEventRecord(e0);
    k_probe_read<<<grid, 512>>>(a, n, reps, sink);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    *read_gbs = (double)bytes * reps / (ms * 1e-3) / 1e9;
    k_probe_write<<<grid, 512>>>(b, n, 1);
    cudaEventRecord(e0);
    k_probe_write<<<grid, 512>>>(b, n, reps);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    *write_gbs = (double)bytes * reps / (ms * 1e-3) / 1e9;
    const size_t half = n / 2;  // copy half of a into half of b: the block stays `bytes`
    k_probe_copy<<<grid, 512>>>(a, b, half, 1);
    cudaEventRecord(e0);
    k_probe_copy<<<grid, 512>>>(a, b, half, reps);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    *copy_gbs = 2.0 * half * 16 * reps / (ms * 1e-3) / 1e9;
    if (cudaGetLastError() != cudaSuccess) rc = fhe_fail(FHE_ECUDA, "fhe_probe_bandwidth: kernels");
  }
  cudaFree(a);
  cudaFree(b);
  cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return rc;
}
