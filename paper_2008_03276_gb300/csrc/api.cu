// api.cu -- the extern "C" entry points of include/ehl.h: argument checks,
// workspace carving and kernel launches.  No compute happens on the host.
#include <cuda_runtime.h>

#include <atomic>

#include "ehl_internal.h"

namespace ehl {
static std::atomic<unsigned long long> g_launches{0};
static thread_local unsigned long long t_launches = 0;
void note_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
}
unsigned long long thread_launches() { return t_launches; }
// graph capture: the captured launches did not run (d < 0); each replay runs them (d > 0)
void add_launches(long long d) { g_launches.fetch_add((unsigned long long)d, std::memory_order_relaxed); }
}  // namespace ehl

using namespace ehl;

extern "C" const char* ehl_status_string(ehl_status s) {
  switch (s) {
    case EHL_OK: return "EHL_OK";
    case EHL_EINVAL: return "EHL_EINVAL: invalid argument";
    case EHL_ENOMEM: return "EHL_ENOMEM: device allocation failed";
    case EHL_ECUDA: return "EHL_ECUDA: CUDA runtime error";
    case EHL_ENOCONV: return "EHL_ENOCONV: iteration limit reached";
    case EHL_ENONFINITE: return "EHL_ENONFINITE: NaN or Inf";
    case EHL_ESINGULAR: return "EHL_ESINGULAR: singular 2x2 pivot";
    case EHL_ETIMEOUT: return "EHL_ETIMEOUT: bounded device wait expired";
  }
  return "EHL_?: unknown status";
}

extern "C" int ehl_version(void) { return 100; }

extern "C" unsigned long long ehl_kernel_launches(void) { return ehl::g_launches.load(std::memory_order_relaxed); }

static bool paqif_args_ok(int n_sys, int n, int beta, int mode) {
  return n_sys >= 1 && n_sys <= (1 << 24) && n >= 1 && n <= (1 << 24) && beta >= 1 && beta <= 8 && mode >= 0 &&
         mode <= 2;
}

static size_t paqif_act_bytes(int n_sys, int n) { return (size_t)n_sys * (size_t)n * sizeof(int); }

extern "C" ehl_status ehl_paqif_workspace_size_partitioned(int n_sys, int n, int beta, int partitions, int mode,
                                                          size_t* bytes) {
  if (!bytes || !paqif_args_ok(n_sys, n, beta, mode) || partitions < 0) return EHL_EINVAL;
  if (paqif_parts(n_sys, n, beta, partitions) < 0) return EHL_EINVAL;
  *bytes = align_up(paqif_stack_bytes(n_sys, n, beta, partitions), kWorkspaceAlign) +
           align_up(paqif_act_bytes(n_sys, n), kWorkspaceAlign);
  return EHL_OK;
}

extern "C" ehl_status ehl_paqif_partitions(int n_sys, int n, int beta, int partitions, int* r) {
  if (!r || !paqif_args_ok(n_sys, n, beta, 0) || partitions < 0) return EHL_EINVAL;
  const int got = paqif_parts(n_sys, n, beta, partitions);
  if (got < 1) return EHL_EINVAL;
  *r = got;
  return EHL_OK;
}

extern "C" ehl_status ehl_paqif_workspace_size(int n_sys, int n, int beta, int mode, size_t* bytes) {
  return ehl_paqif_workspace_size_partitioned(n_sys, n, beta, 0, mode, bytes);
}

extern "C" ehl_status ehl_paqif_solve_partitioned(int n_sys, int n, int beta, int partitions, const double* band,
                                                  const double* rhs, const uint8_t* active, int mode, double* x,
                                                  int* iters, int* info, void* workspace, size_t workspace_bytes,
                                                  void* stream) {
  if (!band || !rhs || !x || !paqif_args_ok(n_sys, n, beta, mode)) return EHL_EINVAL;
  if ((const void*)x == (const void*)band || (const void*)x == (const void*)rhs) return EHL_EINVAL;
  size_t need = 0;
  if (ehl_paqif_workspace_size_partitioned(n_sys, n, beta, partitions, mode, &need) != EHL_OK) return EHL_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  bool owned = false;
  if (workspace) {
    if (workspace_bytes < need || ((uintptr_t)workspace % kWorkspaceAlign) != 0) return EHL_EINVAL;
  } else {
    if (cudaMallocAsync(&workspace, need, st) != cudaSuccess) {
      cudaGetLastError();
      return EHL_ENOMEM;
    }
    owned = true;
  }
  unsigned char* ws = (unsigned char*)workspace;
  PaqifLaunch L;
  L.n_sys = n_sys;
  L.n = n;
  L.beta = beta;
  L.mode = mode;
  L.band = band;
  L.rhs = rhs;
  L.stack = ws;
  L.act = nullptr;
  L.x = x;
  L.iters = iters;
  L.info = info;
  L.parts = partitions;
  cudaError_t e = cudaSuccess;
  if (active || mode == 2) {
    L.act = (int*)(ws + align_up(paqif_stack_bytes(n_sys, n, beta, partitions), kWorkspaceAlign));
    e = launch_expand_active(active, L.act, (size_t)n_sys * (size_t)n, st);
  }
  if (e == cudaSuccess) e = launch_paqif(L, st);
  if (owned) cudaFreeAsync(workspace, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return EHL_ECUDA;
  }
  return EHL_OK;
}

extern "C" ehl_status ehl_paqif_solve(int n_sys, int n, int beta, const double* band, const double* rhs,
                                      const uint8_t* active, int mode, double* x, int* iters, int* info,
                                      void* workspace, size_t workspace_bytes, void* stream) {
  return ehl_paqif_solve_partitioned(n_sys, n, beta, 0, band, rhs, active, mode, x, iters, info, workspace,
                                     workspace_bytes, stream);
}

// Autotuning of the partition count (Sec. 2.2.4: the partitioned method leaves r free): every
// admissible r is timed on the caller's batch with CUDA events (one untimed launch, then the best
// of `reps`), the fastest returned.  The workspace is allocated stream-ordered for the largest r
// and released; the stream is synchronised.
// factorization object: the Z-stack (the folded Z0 rows, and the rhs column a resolve rewrites),
// then the factor store (multipliers, Pi^-1 rows, reduced-system factors)
static size_t paqif_factor_stack_part(int n_sys, int n, int beta) {
  return align_up(paqif_stack_bytes(n_sys, n, beta, 0), kWorkspaceAlign);
}

extern "C" ehl_status ehl_paqif_factor_size(int n_sys, int n, int beta, size_t* bytes) {
  if (!bytes || !paqif_args_ok(n_sys, n, beta, 0) || paqif_parts(n_sys, n, beta, 0) < 1) return EHL_EINVAL;
  *bytes = paqif_factor_stack_part(n_sys, n, beta) + paqif_factor_store_bytes(n_sys, n, beta, 0);
  return EHL_OK;
}

static ehl_status paqif_factor_or_resolve(bool factor, int n_sys, int n, int beta, const double* band,
                                          const double* rhs, int mode, double* x, int* info, void* fac,
                                          size_t fac_bytes, void* stream) {
  if (!rhs || !x || !fac || (factor && !band) || mode < 0 || mode > 1 || !paqif_args_ok(n_sys, n, beta, mode))
    return EHL_EINVAL;
  if ((const void*)x == (const void*)rhs || (factor && (const void*)x == (const void*)band)) return EHL_EINVAL;
  size_t need = 0;
  if (ehl_paqif_factor_size(n_sys, n, beta, &need) != EHL_OK) return EHL_EINVAL;
  if (fac_bytes < need || ((uintptr_t)fac % kWorkspaceAlign) != 0) return EHL_EINVAL;
  unsigned char* f = (unsigned char*)fac;
  PaqifLaunch L;
  L.n_sys = n_sys;
  L.n = n;
  L.beta = beta;
  L.mode = mode;
  L.band = band;
  L.rhs = rhs;
  L.stack = f;
  L.act = nullptr;
  L.x = x;
  L.iters = nullptr;
  L.info = info;
  void* fstore = f + paqif_factor_stack_part(n_sys, n, beta);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  // the resolve kernel writes only the systems that report something
  if (!factor && info) e = cudaMemsetAsync(info, 0, sizeof(int) * (size_t)n_sys, st);
  if (e == cudaSuccess) e = factor ? launch_paqif_factor(L, fstore, st) : launch_paqif_resolve(L, fstore, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return EHL_ECUDA;
  }
  return EHL_OK;
}

extern "C" ehl_status ehl_paqif_factor(int n_sys, int n, int beta, const double* band, const double* rhs, int mode,
                                       double* x, int* info, void* factor, size_t factor_bytes, void* stream) {
  return paqif_factor_or_resolve(true, n_sys, n, beta, band, rhs, mode, x, info, factor, factor_bytes, stream);
}

extern "C" ehl_status ehl_paqif_resolve(int n_sys, int n, int beta, const double* rhs, int mode, double* x, int* info,
                                        void* factor, size_t factor_bytes, void* stream) {
  return paqif_factor_or_resolve(false, n_sys, n, beta, nullptr, rhs, mode, x, info, factor, factor_bytes, stream);
}

extern "C" ehl_status ehl_paqif_autotune(int n_sys, int n, int beta, int mode, const double* band, const double* rhs,
                                         double* x, int reps, void* stream, int* best_r, float* ms_per_r) {
  if (!band || !rhs || !x || !best_r || !paqif_args_ok(n_sys, n, beta, mode) || reps < 1 || reps > 100)
    return EHL_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int gpc = 32;  // partition counts tried: the admissible ones up to the lane groups of a CTA
  size_t need = 0;
  for (int r = 1; r <= gpc; ++r) {
    size_t b = 0;
    if (paqif_parts(n_sys, n, beta, r) == r &&
        ehl_paqif_workspace_size_partitioned(n_sys, n, beta, r, mode, &b) == EHL_OK && b > need)
      need = b;
  }
  if (need == 0) return EHL_EINVAL;
  void* ws = nullptr;
  if (cudaMallocAsync(&ws, need, st) != cudaSuccess) {
    cudaGetLastError();
    return EHL_ENOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best_ms = 0.f;
  int best = -1;
  ehl_status status = EHL_OK;
  for (int r = 1; r <= gpc && e == cudaSuccess && status == EHL_OK; ++r) {
    if (ms_per_r) ms_per_r[r - 1] = -1.f;
    if (paqif_parts(n_sys, n, beta, r) != r) continue;
    status = ehl_paqif_solve_partitioned(n_sys, n, beta, r, band, rhs, nullptr, mode, x, nullptr, nullptr, ws, need,
                                         stream);
    float t_best = -1.f;
    for (int k = 0; k < reps && status == EHL_OK && e == cudaSuccess; ++k) {
      e = cudaEventRecord(e0, st);
      if (e != cudaSuccess) break;
      status = ehl_paqif_solve_partitioned(n_sys, n, beta, r, band, rhs, nullptr, mode, x, nullptr, nullptr, ws,
                                           need, stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float t = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
      if (e == cudaSuccess && (t_best < 0.f || t < t_best)) t_best = t;
    }
    if (ms_per_r) ms_per_r[r - 1] = t_best;
    if (t_best >= 0.f && (best < 0 || t_best < best_ms)) {
      best = r;
      best_ms = t_best;
    }
  }
  cudaFreeAsync(ws, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return EHL_ECUDA;
  }
  if (status != EHL_OK) return status;
  *best_r = best;
  return best > 0 ? EHL_OK : EHL_EINVAL;
}
