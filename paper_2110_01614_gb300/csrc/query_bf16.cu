// BF16 tensor-core form of the fused collision query (placeholder until the
// tcgen05 kernel lands).
#include "nsdf_internal.h"

namespace nsdf {
bool query_bf16_supported(int, int, int) { return false; }
cudaError_t launch_query_bf16(const QueryParams &, int, cudaStream_t) { return cudaErrorNotSupported; }
size_t query_bf16_scratch_bytes(int, int, int) { return 0; }
int query_bf16_grid(int, int64_t, int) { return 1; }
}  // namespace nsdf
