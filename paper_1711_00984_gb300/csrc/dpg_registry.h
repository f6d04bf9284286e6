// dpg_registry.h -- internal route of the general path into caller-provided scratch.
#pragma once
#include <cstddef>
#include <cstdint>

namespace dpg {

// dpg_integrate for the general map with the metric-field workspace at `scratch`
// (scratch_bytes long) instead of a pool allocation: the same programs and kernels as
// dpg_integrate (FP64 and FP32 forms), the whole call in one chunk.  Looks up existing
// state only (DPG_ERR_NOT_INIT when dpg_tables_init has not run for the space and order
// on the current device), holds the library lock from the look-up to the last launch,
// allocates nothing.  DPG_ERR_SCRATCH when the call's metric fields do not fit; DPG_ERR_ARG
// for the affine, extruded and DPG_VEC3 flags.
int integrate_in_scratch(int space, int p_trial, int q_test, int64_t n_elem, const double *vertices,
                         const double *coeffs, void *out, void *scratch, size_t scratch_bytes, void *stream);

}  // namespace dpg
