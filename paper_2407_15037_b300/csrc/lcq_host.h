// lcq_host.h -- host-side helpers shared between the library's translation
// units (not part of the C ABI).
#pragma once

#include <cstdint>

#include "../../include/lcq.h"

namespace lcq {

// ABS/REL constants of Sec. 2.2 and the REL reading, as the raw bits stored
// in lcq_header (ebT, scale, inv, chk), and the certainty bounds of the
// float64 REL check (0 otherwise); false if the bound is unusable.
bool host_consts(lcq_dtype dtype, lcq_bound_type bound, double eb, uint64_t bits[4],
                 uint64_t* cert_w = nullptr, uint32_t* cert_emin = nullptr);

// Validation shared by lcq_quantize and the batch planner.
lcq_status check_quantize_args(lcq_dtype dtype, lcq_bound_type bound_type, double eb, const void* d_in,
                               uint64_t n, const int32_t* d_bins, const uint32_t* d_mask,
                               const void* d_outliers, uint64_t outlier_capacity, const lcq_header* d_hdr);

int device_sm_count();

}  // namespace lcq
