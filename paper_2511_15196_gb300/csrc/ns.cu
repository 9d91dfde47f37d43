// Nested sampling driver (Sec. 2 sampler (iv); App. A).
#include "run.h"

namespace phi4 {

phi4_status ns_replace(phi4_run* r, int32_t* done_out) {
  (void)r;
  (void)done_out;
  set_error("nested sampling is not built yet");
  return PHI4_ERR_UNSUPPORTED;
}

phi4_status ns_evidence(phi4_run* r, double* logz, double* logz_err) {
  (void)r;
  if (logz) *logz = NAN;
  if (logz_err) *logz_err = NAN;
  set_error("nested sampling is not built yet");
  return PHI4_ERR_UNSUPPORTED;
}

}  // namespace phi4
