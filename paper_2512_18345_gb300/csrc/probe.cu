// Bandwidth probe (measurement support): read, write and read+write copy of a
// block of `bytes` repeated `reps` times with 128-bit L2-cached accesses, timed
// with CUDA events.  A block smaller than the L2 gives the L2 bandwidth (the
// paper's method: a block smaller than the L2 read and written repeatedly);
// a larger one gives the DRAM bandwidth.
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
}  // namespace

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
