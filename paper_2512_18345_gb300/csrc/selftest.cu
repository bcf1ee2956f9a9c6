// Failure-detection self-test: exercises the bounded-wait path of the
// tensor-core and streaming kernels without a fault.  One CTA initialises an
// mbarrier that nothing ever arrives on, waits on it with a short iteration
// limit, records the expiry in the context's status word exactly as the
// production kernels do, and returns; fhe_ctx_sync then reports FHE_ETIMEOUT
// and the context stays usable.
#include "../../include/fhe.h"
#include "async.cuh"
#include "ctx.h"
#include "internal.h"

namespace {
__global__ void k_unsatisfied_wait(unsigned int *status, unsigned int flag) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    fhe::mbar_init(&bar, 1);                                 // expects one arrival; none comes
    if (!fhe::mbar_wait_bounded(&bar, 0u, 4096u)) atomicOr(status, flag);
  }
}
}  // namespace

extern "C" int fhe_selftest_wait_timeout(fhe_ctx *c, fhe_stream stream) {
  if (!c) return fhe_fail(FHE_EINVAL, "fhe_selftest_wait_timeout: null");
  cudaSetDevice(c->device);
  k_unsatisfied_wait<<<1, 32, 0, (cudaStream_t)stream>>>(c->d_status, 0x80u);
  return cudaGetLastError() == cudaSuccess ? FHE_OK : fhe_fail(FHE_ECUDA, "fhe_selftest_wait_timeout: launch");
}
