// Parameters of the adjoint right-hand-side launch, shared by the C-ABI file
// and the kernel files (the kernels are in teno7_adjoint.cuh).
#pragma once
#include <stdint.h>

#include "teno7_internal.h"

namespace t7 {
struct Adjoint1D {
    const void *U;         // state [3][n]
    const void *v;         // adjoint input [3][n]
    void *out;             // accumulates scale (dL/dU)^T v, [3][n] (atomically)
    const uint8_t *masks;  // nullable: forward Delta codes [2][3][n+1]; else recomputed
    int n, bc_lo, bc_hi;
    double dx, eps, CT, gamma;
    DevCtl *ctl;
    int slot_in;               // alpha of U (frozen) ...
    const double *alpha_ptr;   // ... or, if not null, read from here
    double scale;              // out += scale (dL/dU)^T v
};
}  // namespace t7
