// dpg_registry.h -- read-only access to an initialised general-path program (internal).
#pragma once
#include "dpg_kernels.h"
#include "dpg_setup.h"

namespace dpg {

struct ProgramView {
    const Program *prog;
    const BlockDesc *d_blocks;
    const Unit *d_units;
    const double *zeta, *w, *pp64;
    const float *pp32;
    DevStatus *status;
};

// Looks up the active program of (space, p_trial, q) on the current device without
// creating any state and without allocating: DPG_ERR_NOT_INIT when dpg_tables_init has
// not run for it on this device.  The pointers stay valid until dpg_tables_free.
int lookup_program_view(int space, int p_trial, int q, ProgramView *view);

}  // namespace dpg
