// Entry points whose implementation is not in this build yet.
#include "api_internal.h"

extern "C" {
rf_status rf_fit(const rf_model*, const rf_data*, const double*, const rf_fit_opts*, double*, double*, double*,
                 int32_t*, int32_t*) {
  rf::set_error("rf_fit: not available in this build");
  return RF_E_INVALID;
}
rf_status rf_generate_toys(const rf_model*, const double*, int32_t, uint64_t, int32_t, const double*, int32_t,
                           const int32_t*, rf_data**) {
  rf::set_error("rf_generate_toys: not available in this build");
  return RF_E_INVALID;
}
rf_status rf_hist64(const rf_model*, const rf_data*, int32_t, float*, void*) {
  rf::set_error("rf_hist64: not available in this build");
  return RF_E_INVALID;
}
}
