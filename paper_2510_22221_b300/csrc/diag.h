// Diagnostics on the device state (diag.cu); not part of the public ABI.
#pragma once
#include "fdtd_llg_internal.h"

namespace fl {

// div(H + M_face) at every cell centre of instance dI (field buffer F) into
// out[nc] (FP64, device), with M the instance's magnetisation assembled from
// its ncomp magnet regions dcomps into the scratch array M[3 nc] (device).
cudaError_t launch_div_b(const Inst *dI, const MagComp *dcomps, int ncomp, int F, long long nc, double dx, double dy,
                         double dz, double *M, double *out, cudaStream_t s);

}  // namespace fl
