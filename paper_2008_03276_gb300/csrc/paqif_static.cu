// paqif_static.cu -- ehl_paqif_solve_static: the batched PAQIF solve with its
// scratch memory in a fixed, library-owned device array instead of a
// caller-provided or freshly allocated workspace.
//
// Who needs this: callers that must not allocate device memory while they
// solve.  Examples are a host program that has handed the whole GPU to its
// own memory pool and forbids any other allocation, a plug-in that runs inside
// another application's callback where allocating is not allowed, and a
// real-time loop that may neither block on the allocator nor fail with an
// out-of-memory error in the middle of a run.  They still pass their own
// input and output arrays.
//
// The scratch array below is reserved on every GPU that loads this library,
// for as long as the process lives.  Its name is a host-side stand-in, not a
// device address, so the host obtains the address with cudaGetSymbolAddress
// once per device (with that device current) and hands it to the kernel.
#include <cuda_runtime.h>

#include <mutex>

#include "ehl_internal.h"

using namespace ehl;

static __device__ __align__(256) unsigned char g_paqif_static_scratch[EHL_PAQIF_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up on the
// first call per device and cached.  The address belongs to the device's primary context (the
// one the CUDA runtime uses): it stays valid until that context is destroyed, so a process that
// calls cudaDeviceReset must not call this entry point afterwards.  Returns EHL_ECUDA if the
// lookup fails.
ehl_status scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return EHL_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_paqif_static_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return EHL_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return EHL_OK;
}

}  // namespace

extern "C" ehl_status ehl_paqif_solve_static(int n_sys, int n, int beta, const double* band, const double* rhs,
                                             const uint8_t* active, int mode, double* x, int* iters, int* info,
                                             void* stream) {
  if (!band || !rhs || !x) return EHL_EINVAL;
  if ((const void*)x == (const void*)band || (const void*)x == (const void*)rhs) return EHL_EINVAL;
  size_t need = 0;
  if (ehl_paqif_workspace_size(n_sys, n, beta, mode, &need) != EHL_OK) return EHL_EINVAL;
  if (need > (size_t)EHL_PAQIF_STATIC_SCRATCH_BYTES) return EHL_EINVAL;  // batch too large for the fixed array
  // the layout below is the one ehl_paqif_workspace_size() counts for partitions = 0: the stack,
  // then the int32 flags at the next aligned offset; both must lie inside `need`
  const size_t stack_end = align_up(paqif_stack_bytes(n_sys, n, beta, 0), kWorkspaceAlign);
  if (stack_end + (size_t)n_sys * (size_t)n * sizeof(int) > need) return EHL_EINVAL;
  void* base = nullptr;
  ehl_status st = scratch_address(&base);
  if (st != EHL_OK) return st;
  unsigned char* ws = (unsigned char*)base;
  cudaStream_t s = (cudaStream_t)stream;
  PaqifLaunch L;
  L.n_sys = n_sys;
  L.n = n;
  L.beta = beta;
  L.mode = mode;
  L.band = band;
  L.rhs = rhs;
  L.stack = ws;  // every level's stack entries are written before they are read
  L.act = nullptr;
  L.x = x;
  L.iters = iters;
  L.info = info;
  cudaError_t e = cudaSuccess;
  if (active || mode == 2) {
    // the flags left by the previous call are overwritten here, from `active` or with zeros
    L.act = (int*)(ws + align_up(paqif_stack_bytes(n_sys, n, beta), kWorkspaceAlign));
    e = launch_expand_active(active, L.act, (size_t)n_sys * (size_t)n, s);
  }
  if (e == cudaSuccess) e = launch_paqif(L, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return EHL_ECUDA;
  }
  return EHL_OK;
}
