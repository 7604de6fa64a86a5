// ehl_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/ehl.h"

namespace ehl {

constexpr int kSmCount = 152;  // GB300: grids are sized for its 152 SMs
constexpr int kPaqifMaxActiveSetSteps = 64;
// Newton steps of a coarse grid of the nested iteration at most (a coarse grid that
// cannot resolve the surface stalls rather than converges)
constexpr int kCoarseMaxIter = 40;
constexpr size_t kWorkspaceAlign = 256;

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Count of kernels this library has launched (observability; see ehl_kernel_launches).
void note_launch();
unsigned long long thread_launches();  // note_launch() calls of this host thread
void add_launches(long long d);
// set the kernels' shared-memory attributes for half-band beta on the current device (before
// any stream capture: the launches themselves then make no attribute call)
cudaError_t paqif_prepare(int beta);

struct PaqifLaunch {
  int n_sys, n, beta, mode;
  const double* band;
  const double* rhs;
  int* act;     // int32 flags [n_sys][n] or nullptr
  void* stack;  // paqif_stack_bytes() bytes, 16-byte aligned
  double* x;
  int* iters;
  int* info;
  bool f32 = false;  // float32 sweeps (modes 0 and 1): a preconditioner, not a solve to 1e-12
  int parts = 0;     // partitions per system (Sec. 2.2.4); 0: chosen by paqif_parts
};

// Partitions per system that a launch uses: `requested` if its geometry is valid
// (it divides the groups of a CTA; blocks of even order 2 ceil(n / 2r) with an
// interior level and a real row each), -1 if not; 0 asks for the automatic choice.
int paqif_parts(int n_sys, int n, int beta, int requested);
// Bytes of the per-block Z-stack (padded to whole CTAs); 0 for a bad beta or partition count.
size_t paqif_stack_bytes(int n_sys, int n, int beta, int parts = 0);
cudaError_t launch_paqif(const PaqifLaunch& L, cudaStream_t st);
// Factor once (also solving for L.rhs), then resolve for new right-hand sides
// with the same band: the stack (L.stack) and the factor store are kept.
size_t paqif_factor_store_bytes(int n_sys, int n, int beta, int parts = 0);
cudaError_t launch_paqif_factor(const PaqifLaunch& L, void* fstore, cudaStream_t st);
cudaError_t launch_paqif_resolve(const PaqifLaunch& L, void* fstore, cudaStream_t st);
cudaError_t launch_expand_active(const uint8_t* in, int* out, size_t total, cudaStream_t st);

}  // namespace ehl
