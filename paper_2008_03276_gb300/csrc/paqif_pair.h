// paqif_pair.h -- the lane-pair PAQIF kernel (half-bands 1..4, modes 0 and 1, float64 in and out,
// double-float arithmetic): one lane per side of a block, r in {1, 2, 4, 8, 16} blocks per system.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "ehl_internal.h"

namespace ehl {

// Blocks per system the lane-pair kernel would use for a launch of this shape, 0 if it does not
// take it (beta > 4, mode 2, float32 sweeps or a stored factorization).
int paqif_pair_parts(int n_sys, int n, int beta, int mode, bool f32, bool factor_store);
// Bytes of its Z-stack for r blocks per system; 0 for an inadmissible r.
size_t paqif_pair_stack_bytes(int n_sys, int n, int beta, int r);
// One launch with r blocks per system (L.stack: paqif_pair_stack_bytes bytes, 16-byte aligned;
// L.band on a 16-byte boundary).
cudaError_t launch_paqif_pair(const PaqifLaunch& L, int r, cudaStream_t st);
// Its shared-memory attribute for half-band beta on the current device (nothing for beta > 4),
// set once per device; called by paqif_prepare, before any stream capture.
cudaError_t paqif_pair_prepare(int beta);

}  // namespace ehl
