// mbs_setup_dev.h -- the device setup of the per-cell step operators of
// jittered two-level media (mbs_setup_dev.cu), called by the scenario
// creation (mbs_host.cpp).
#pragma once

#include <cstddef>
#include <cstdint>

namespace mbs {

// One medium slot's FP64 parts: the Liouvillian's H0 and dissipator parts
// (4 x 4 on the dipole-eigenbasis coordinates), the reference and initial
// states, the dipole eigenvalues, and the coupling factor dt/eps / (1 + k)
// x overlap x density (times each cell's density jitter).
struct SetupSlot2 {
  double MH[16], MD[16], yref[4], yinit[4], lambda[2], cpl0;
};

// One thread per cell: rows as the host setup writes them (pcell [16][ld],
// pcell2 [7][ld], dinit [3][ld], zero for vacuum cells, which the caller
// zeroes); counts[0] = cells with a non-finite operator, counts[1] = cells
// without the optical-Bloch pattern (zeroed by the caller).
int setup_cells2(const SetupSlot2 *slots, const uint8_t *mat, const int *qslot, const double *jitter, int nx, int off,
                 int ld, double dt, double *pcell, double *pcell2, double *dinit, int *counts, void *stream);

// y = (float)x, n values
int to_float(const double *x, float *y, size_t n, void *stream);

}  // namespace mbs
