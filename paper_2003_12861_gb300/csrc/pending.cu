// Entry points whose implementation is not in this build yet.
#include "api_internal.h"

extern "C" {
rf_status rf_fit(const rf_model*, const rf_data*, const double*, const rf_fit_opts*, double*, double*, double*,
                 int32_t*, int32_t*) {
  rf::set_error("rf_fit: not available in this build");
  return RF_E_INVALID;
}
}
