// Tensor-core base conversion (placeholder until the tcgen05 kernel lands).
#include "ctx.h"
#include "internal.h"

namespace fhe {
cudaError_t launch_bconv_tc(const DevTables &, const BconvArgs &, int, int, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace fhe
bool fhe_tc_available() { return false; }
