// Separable tensor-core path (placeholder until the tcgen05 kernels land).
#include "cgh_internal.h"

int tc_progressive(const cgh_plan*, const int32_t*, const int32_t* const*, const int32_t*, float2*, int,
                   int, cudaStream_t) {
  return cgh_fail(CGH_ERR_UNSUPPORTED, "tensor-core form not built");
}
int tc_reconstruct(const cgh_plan*, const float2*, float2*, const uint8_t*, float*, cudaStream_t) {
  return cgh_fail(CGH_ERR_UNSUPPORTED, "reconstruction not built");
}
void tc_destroy(cgh_plan*) {}
