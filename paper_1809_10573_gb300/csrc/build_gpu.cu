// Placeholder translation unit for the on-device construction (filled in next).
#include "idbf_internal.h"
extern "C" idbf_status idbf_build(const idbf_kernel*, const double*, const double*, int64_t, const idbf_params*, void*,
                                  idbf_plan* out) {
  if (out) *out = nullptr;
  return IDBF_EUNSUPPORTED;
}
