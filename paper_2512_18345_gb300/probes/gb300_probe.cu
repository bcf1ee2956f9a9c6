// GB300 throughput probe (measurement support, not part of the library):
// integer multiply / multiply-high / add+min / wide multiply-add / Shoup
// modular multiply chains and FP32 FMA, L2 read / write / copy bandwidth on
// 32 and 64 MB blocks (smaller than L2, as in the paper's method), HBM on
// 4 GB, and legacy mma.sync u8 / f16 rates.  The numbers set the ALU and L2
// denominators of the roofline fractions.
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/gb300_probe \
//                paper_2512_18345_gb300/probes/gb300_probe.cu && /tmp/gb300_probe
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("CUDA %s at %d\n", cudaGetErrorString(e), __LINE__); return 1;}}while(0)

template<int OP>
__global__ void k_int(uint32_t* out, uint32_t seed, int iters) {
  uint32_t a0 = threadIdx.x ^ seed, a1 = a0 * 3 + 1, a2 = a0 * 5 + 7, a3 = a0 * 11 + 3;
  uint32_t a4 = a0 + 9, a5 = a0 + 13, a6 = a0 ^ 0x55, a7 = a0 ^ 0x77;
  const uint32_t m = seed | 1, q = 0x7fff0001u;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int r = 0; r < 16; r++) {
      if (OP == 0) { // mul.lo (IMAD)
        a0 = a0 * m + a1; a1 = a1 * m + a2; a2 = a2 * m + a3; a3 = a3 * m + a4;
        a4 = a4 * m + a5; a5 = a5 * m + a6; a6 = a6 * m + a7; a7 = a7 * m + a0;
      } else if (OP == 1) { // mul.hi
        a0 = __umulhi(a0, m) ^ a1; a1 = __umulhi(a1, m) ^ a2; a2 = __umulhi(a2, m) ^ a3; a3 = __umulhi(a3, m) ^ a4;
        a4 = __umulhi(a4, m) ^ a5; a5 = __umulhi(a5, m) ^ a6; a6 = __umulhi(a6, m) ^ a7; a7 = __umulhi(a7, m) ^ a0;
      } else if (OP == 2) { // add+min (ALU)
        a0 = min(a0 + a1, a0 - q); a1 = min(a1 + a2, a1 - q); a2 = min(a2 + a3, a2 - q); a3 = min(a3 + a4, a3 - q);
        a4 = min(a4 + a5, a4 - q); a5 = min(a5 + a6, a5 - q); a6 = min(a6 + a7, a6 - q); a7 = min(a7 + a0, a7 - q);
      } else if (OP == 3) { // wide mad
        uint64_t t0 = (uint64_t)a0 * m + a1, t1 = (uint64_t)a2 * m + a3, t2 = (uint64_t)a4 * m + a5, t3 = (uint64_t)a6 * m + a7;
        a0 = (uint32_t)t0; a1 = (uint32_t)(t0 >> 32); a2 = (uint32_t)t1; a3 = (uint32_t)(t1 >> 32);
        a4 = (uint32_t)t2; a5 = (uint32_t)(t2 >> 32); a6 = (uint32_t)t3; a7 = (uint32_t)(t3 >> 32);
      } else if (OP == 4) { // shoup modmul chain
        uint32_t w = m, ws = m ^ 0x1234567;
        a0 = a0 * w - __umulhi(a0, ws) * q; a1 = a1 * w - __umulhi(a1, ws) * q;
        a2 = a2 * w - __umulhi(a2, ws) * q; a3 = a3 * w - __umulhi(a3, ws) * q;
        a4 = a4 * w - __umulhi(a4, ws) * q; a5 = a5 * w - __umulhi(a5, ws) * q;
        a6 = a6 * w - __umulhi(a6, ws) * q; a7 = a7 * w - __umulhi(a7, ws) * q;
      } else if (OP == 5) { // fp32 fma
        float f0 = __uint_as_float(a0), f1 = __uint_as_float(a1), f2 = __uint_as_float(a2), f3 = __uint_as_float(a3);
        f0 = fmaf(f0, 1.0001f, f1); f1 = fmaf(f1, 1.0001f, f2); f2 = fmaf(f2, 1.0001f, f3); f3 = fmaf(f3, 1.0001f, f0);
        a0 = __float_as_uint(f0); a1 = __float_as_uint(f1); a2 = __float_as_uint(f2); a3 = __float_as_uint(f3);
        float g0 = __uint_as_float(a4), g1 = __uint_as_float(a5), g2 = __uint_as_float(a6), g3 = __uint_as_float(a7);
        g0 = fmaf(g0, 1.0001f, g1); g1 = fmaf(g1, 1.0001f, g2); g2 = fmaf(g2, 1.0001f, g3); g3 = fmaf(g3, 1.0001f, g0);
        a4 = __float_as_uint(g0); a5 = __float_as_uint(g1); a6 = __float_as_uint(g2); a7 = __float_as_uint(g3);
      }
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 ^ a1 ^ a2 ^ a3 ^ a4 ^ a5 ^ a6 ^ a7;
}

__global__ void k_read(const uint4* __restrict__ p, size_t n, int reps, uint32_t* out) {
  uint32_t acc = 0;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; r++)
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
      uint4 v = __ldcg(p + i); acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
  if (acc == 0x12345678u) out[0] = acc;
}
__global__ void k_write(uint4* __restrict__ p, size_t n, int reps) {
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; r++)
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride)
      __stcg(p + i, make_uint4(r, i, 0, 1));
}
__global__ void k_copy(const uint4* __restrict__ a, uint4* __restrict__ b, size_t n, int reps) {
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; r++)
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
      uint4 v = __ldcg(a + i); v.x += r; __stcg(b + i, v);
    }
}

__global__ void k_imma(int* c, int iters) {
  int a0 = threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, b0 = a0 * 7, b1 = a0 * 9;
  int d[4][4] = {};
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < 4; u++)
      asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+r"(d[u][0]),"+r"(d[u][1]),"+r"(d[u][2]),"+r"(d[u][3]) : "r"(a0),"r"(a1),"r"(a2),"r"(a3),"r"(b0),"r"(b1));
  }
  int s = 0;
  for (int u = 0; u < 4; u++) s += d[u][0] + d[u][1] + d[u][2] + d[u][3];
  c[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void k_hmma(float* c, int iters) {
  uint32_t a0 = threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, b0 = a0 * 7, b1 = a0 * 9;
  float d[4][4] = {};
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < 4; u++)
      asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[u][0]),"+f"(d[u][1]),"+f"(d[u][2]),"+f"(d[u][3]) : "r"(a0),"r"(a1),"r"(a2),"r"(a3),"r"(b0),"r"(b1));
  }
  float s = 0;
  for (int u = 0; u < 4; u++) s += d[u][0] + d[u][1] + d[u][2] + d[u][3];
  c[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int main() {
  cudaDeviceProp prop; CK(cudaGetDeviceProperties(&prop, 0));
  int clk_khz = 0; cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
  printf("device %s SMs %d L2 %d MB persistL2max %d MB smemOptin %zu clk %d MHz\n", prop.name, prop.multiProcessorCount,
         prop.l2CacheSize >> 20, prop.persistingL2CacheMaxSize >> 20, prop.sharedMemPerBlockOptin, clk_khz / 1000);
  int sms = prop.multiProcessorCount;
  uint32_t* out; CK(cudaMalloc(&out, 64 << 20));
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  const char* names[] = {"imad.lo", "umulhi", "iadd+imnmx(2 ops)", "mad.wide(4/iter)", "shoup(3imad+1)", "ffma"};
  int iters = 4096;
  for (int op = 0; op < 6; op++) {
    for (int rep = 0; rep < 2; rep++) {
      cudaEventRecord(e0);
      int blocks = sms * 4, threads = 512;
      switch (op) {
        case 0: k_int<0><<<blocks, threads>>>(out, 7, iters); break;
        case 1: k_int<1><<<blocks, threads>>>(out, 7, iters); break;
        case 2: k_int<2><<<blocks, threads>>>(out, 7, iters); break;
        case 3: k_int<3><<<blocks, threads>>>(out, 7, iters); break;
        case 4: k_int<4><<<blocks, threads>>>(out, 7, iters); break;
        case 5: k_int<5><<<blocks, threads>>>(out, 7, iters); break;
      }
      cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
      float ms; cudaEventElapsedTime(&ms, e0, e1);
      double ops = (double)blocks * threads * iters * 16 * 8;  // "op-chains" per thread
      if (rep) printf("%-20s %.3f ms  %.2f Tchain/s  %.1f chain/clk/SM (at %d MHz)\n", names[op], ms, ops / ms / 1e9,
                      ops / (ms * 1e-3) / sms / (clk_khz * 1e3), clk_khz / 1000);
    }
  }
  // L2 bandwidth on a block smaller than L2, and HBM on a block much larger
  size_t sizes[] = {(size_t)32 << 20, (size_t)64 << 20, (size_t)4 << 30};
  for (size_t bytes : sizes) {
    uint4 *a, *b; CK(cudaMalloc(&a, bytes)); CK(cudaMalloc(&b, bytes));
    cudaMemset(a, 1, bytes); cudaMemset(b, 2, bytes);
    size_t n = bytes / 16;
    int reps = bytes < ((size_t)1 << 30) ? 50 : 2;
    for (int blocksPerSM : {2, 4, 8}) {
      int blocks = sms * blocksPerSM, threads = 512;
      float ms;
      k_read<<<blocks, threads>>>(a, n, 1, out);
      cudaEventRecord(e0); k_read<<<blocks, threads>>>(a, n, reps, out); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
      cudaEventElapsedTime(&ms, e0, e1); double rd = bytes * (double)reps / ms / 1e6;
      k_write<<<blocks, threads>>>(b, n, 1);
      cudaEventRecord(e0); k_write<<<blocks, threads>>>(b, n, reps); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
      cudaEventElapsedTime(&ms, e0, e1); double wr = bytes * (double)reps / ms / 1e6;
      size_t half = n / 2;
      k_copy<<<blocks, threads>>>(a, b, half, 1);
      cudaEventRecord(e0); k_copy<<<blocks, threads>>>(a, b, half, reps); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
      cudaEventElapsedTime(&ms, e0, e1); double cp = 2.0 * half * 16 * (double)reps / ms / 1e6;
      printf("block %6zu MB  grid %d/SM: read %.0f GB/s  write %.0f GB/s  copy(r+w) %.0f GB/s\n", bytes >> 20, blocksPerSM, rd, wr, cp);
    }
    cudaFree(a); cudaFree(b);
  }
  // IMMA / HMMA legacy rates
  for (int rep = 0; rep < 2; rep++) {
    int blocks = sms * 4, threads = 256, it = 4096; float ms;
    cudaEventRecord(e0); k_imma<<<blocks, threads>>>((int*)out, it); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    double ops = (double)blocks * (threads / 32) * it * 4 * (16.0 * 8 * 32 * 2);
    if (rep) printf("mma.sync u8 m16n8k32: %.1f TOPS\n", ops / ms / 1e9);
    cudaEventRecord(e0); k_hmma<<<blocks, threads>>>((float*)out, it); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    ops = (double)blocks * (threads / 32) * it * 4 * (16.0 * 8 * 16 * 2);
    if (rep) printf("mma.sync f16 m16n8k16: %.1f TFLOPS\n", ops / ms / 1e9);
  }
  CK(cudaGetLastError());
  printf("done\n");
  return 0;
}
