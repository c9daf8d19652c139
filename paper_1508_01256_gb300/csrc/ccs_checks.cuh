// ccs_checks.cuh -- alignment rules for the device pointers the entry points
// take.  A misaligned binary64 or int64 access, or a bulk copy from an
// address off a 16-byte boundary, faults on the device; the entry points
// refuse such pointers on the host with CCS_EINVAL before any device work.
#pragma once

#include <cstdint>

namespace ccs {

// CCS_OK when p is a multiple of `align` bytes (null passes: null pointers
// are checked separately); else CCS_EINVAL with "<who>: <what> ..." recorded.
int check_aligned(const char *who, const char *what, const void *p, unsigned align);

// One problem's arrays: csc_rows on 16 bytes (bulk-copied), csr_ptr, y,
// x_hat, r and r0_hist on 8, csr_cols on 4.
int check_problem_arrays(const char *who, const int32_t *csc_rows, const int64_t *csr_ptr,
                         const int32_t *csr_cols, const double *y, const double *x_hat,
                         const double *r, const int64_t *r0_hist);

// Workspaces start on a 256-byte boundary (every region inside is laid out
// on 256-byte offsets from it).
constexpr unsigned kWorkspaceAlign = 256;

}  // namespace ccs
