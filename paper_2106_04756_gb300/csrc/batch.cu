// Batched persistent solve (pdlp_solve_batch).
#include <string>

#include "common.cuh"

extern "C" int pdlp_solve_batch(int32_t, const int32_t *, const int32_t *, const int64_t *, const int64_t *,
                                const int64_t *, const int32_t *, const int32_t *, const double *, const double *,
                                const double *, const double *, const double *, const uint8_t *,
                                const pdlp_options *, double *, double *, pdlp_result *) {
  return PDLP_ERR_STATE;
}
