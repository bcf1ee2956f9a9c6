// Host-side declarations shared by the translation units of the library.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <vector>

#include "bconv.cuh"
#include "common.cuh"
#include "ntt.cuh"

namespace fhe {

// A set-up step that applies to one device only (a kernel's function attributes:
// cudaFuncSetAttribute acts on the current device), run once per device.  Safe to
// call from several host threads: two may both run the step, which is idempotent.
class PerDeviceOnce {
 public:
  template <class F>
  cudaError_t run(F &&step) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = dev < 64 ? 1ull << dev : 0;  // devices beyond 64 repeat the step
    if (bit && (done_.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = step();
    if (e == cudaSuccess && bit) done_.fetch_or(bit, std::memory_order_acq_rel);
    return e;
  }

 private:
  std::atomic<uint64_t> done_{0};
};

// Optional per-launch timing: each kernel launch is bracketed by two CUDA events
// on its stream and recorded under the kernel's name.
struct TraceRec {
  const char *name;
  cudaEvent_t a, b;
};
struct Tracer {
  std::vector<TraceRec> recs;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  cudaEvent_t get();
  void begin(const char *name, cudaStream_t s);
  void end(cudaStream_t s);
  void reset() { recs.clear(); used = 0; }
  ~Tracer();
};

constexpr int kGbarSlots = 1024;  // grid-barrier counters of the persistent NTT per context

struct DevTables {
  NttTables ntt;
  const PrimeC *pc;
  int logn;
  Tracer *tracer;          // null: no tracing
  unsigned int *status;    // device word, nonzero once a bounded device-side wait expired: bit 0
                           // tensor-core BConv, bit 1 inner product, bit 2 diagonal pass,
                           // bit 3 streaming NTT, bit 4 persistent NTT's grid barrier,
                           // bit 7 the wait self-test
  unsigned int *gbar;      // kGbarSlots grid-barrier counters (8 words apart) of the persistent NTT
  int ip_ctas_per_sm;      // resident CTAs per SM of the streaming inner product (1 or 2; autotuned)
  int ntt_otf;             // block passes form their register twiddles on the fly
  int ntt_single;          // 2^16-point transforms in one cluster launch instead of two passes
  int ntt_stream;          // the passes as persistent kernels fed by a producer warp (ntt_bulk.cuh)
  int ntt_persist;         // both passes of a transform in one cooperative launch (k_nttp)
  int ntt_stream_stages;   // shared-memory stages per CTA of those kernels
  int ntt_stream_ctas;     // persistent CTAs per SM of those kernels (1..3)
  int bconv_tc_ctas;       // resident CTAs per SM of the tensor-core BConv (1..4)
  int bconv_tc_pipe;       // the tensor-core BConv with two accumulators per CTA (MMA beside epilogue)
  int ip_staged;           // hoisted inner product: digits' permuted blocks staged (ip_hoisted.cuh)
  int ip_staged_ctas;      // resident CTAs per SM of that kernel (1 or 2)
  int ip_staged_depth;     // its stages per warp (2..4; 0: 2)
  int tc_k;                // K of the context's tensor-core BConv tables (48 or 64; 0: none)
};

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
void note_launch();
// the byte-digit table of the tensor-core base conversion (host side)
// K = kt (48 for at most 8 inputs, 64 for at most 12)
std::vector<uint16_t> bconv_tc_table(const std::vector<uint32_t> &T, int n_in, const std::vector<uint32_t> &p_out,
                                     int kt);

// One NTT pass over every limb of `sl` (column or block pass, forward or inverse).
cudaError_t launch_ntt_pass(const DevTables &t, bool column, bool fwd, int pro, int epi, const SegList &sl,
                            cudaStream_t s);
// Both passes: forward = column (pro, lazy) then block (plain, epi);
// inverse = block (pro, lazy) then column (plain, epi).  In place after the first pass (dst of sl).
cudaError_t launch_ntt(const DevTables &t, bool fwd, int pro, int epi, const SegList &first, const SegList &second,
                       cudaStream_t s);
// Both passes in one cluster launch (first / second enumerate the same limbs); only for the
// (pro, epi) pairs ntt_single_pass_ok accepts, at N = 2^16.
bool ntt_single_pass_ok(const DevTables &t, int pro, int epi, bool fwd);
cudaError_t launch_ntt_single(const DevTables &t, bool fwd, int pro, int epi, const SegList &first,
                              const SegList &second, cudaStream_t s);
// how many 16-CTA clusters of the single-pass NTT the current device holds at once (0: none)
int ntt_single_pass_clusters();
cudaError_t launch_bconv(const DevTables &t, const BconvArgs &a, int max_in, int max_out, cudaStream_t s);
// kt: the K of the groups' tables (48: max_in <= 8; 64: max_in <= 12)
cudaError_t launch_bconv_tc(const DevTables &t, const BconvArgs &a, int max_in, int max_out, cudaStream_t s, int kt);
cudaError_t launch_ew(const DevTables &t, int op, const SegList &sl, cudaStream_t s);
// key inner product (both halves) for the ext limbs of sl; seg.dst = u_0[t0]
// beta_max: the largest digit count among the segments' items (sizes the stages)
cudaError_t launch_ip(const DevTables &t, const SegList &sl, bool gather_own, bool gather_ext, bool add_c1, int beta_max,
                      cudaStream_t s);
// the special limbs' inner product fused with ModDown's first inverse-NTT pass (ip_intt.cuh);
// sl: one segment per item over its K special limbs, dst = the item's UC [2][K][N]
cudaError_t launch_ip_intt(const DevTables &t, const SegList &sl, int beta_max, cudaStream_t s);

// number of kernels launched since the counter was last read (for the benchmark's launch count)
long long kernel_launches();

}  // namespace fhe
