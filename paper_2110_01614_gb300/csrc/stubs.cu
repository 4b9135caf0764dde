// Entry points whose kernels are not built yet.
#include "nsdf_internal.h"

extern "C" nsdf_status nsdf_query_grouped(nsdf_ctx *, const float *, const int64_t *,
                                          const int64_t *, int64_t, float, float *, float *,
                                          nsdf_stream) {
  return NSDF_ERR_UNSUPPORTED;
}
