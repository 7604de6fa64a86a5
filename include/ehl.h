/*
 * ehl.h -- C ABI of the GB300 (sm_103a) hot path of the TVD / PAQIF
 * elastohydrodynamic-lubrication solver (arXiv 2008.03276).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Array arguments are DEVICE pointers into the current CUDA device's
 *    memory, owned by the caller (for example torch tensors' data_ptr()).
 *    They must be contiguous, float64 unless stated otherwise, and 8-byte
 *    aligned.  The library never frees or keeps them after the call returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every call enqueues its work on that stream and returns
 *    without synchronising unless its comment says otherwise.
 *  - Errors are returned as ehl_status codes, never as exceptions or aborts.
 *    Argument errors are detected on the host before anything is enqueued.
 *    Failures found by the kernels (a singular 2x2 pivot, a non-finite
 *    value, no convergence) are written to per-system / per-instance `info`
 *    words in device memory, which the caller reads when it needs them.
 *  - No entry point calls cudaDeviceSynchronize; none uses more than one GPU.
 */
#ifndef EHL_GB300_H
#define EHL_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EHL_OK = 0,
  EHL_EINVAL = 1,      /* an argument is out of range or a required pointer is NULL */
  EHL_ENOMEM = 2,      /* device memory could not be allocated                       */
  EHL_ECUDA = 3,       /* a CUDA runtime call failed (launch, copy, ...)             */
  EHL_ENOCONV = 4,     /* an iteration did not converge within its limit             */
  EHL_ENONFINITE = 5,  /* a NaN or Inf appeared                                      */
  EHL_ESINGULAR = 6,   /* a 2x2 pivot of the factorization was (numerically) singular */
  EHL_ETIMEOUT = 7     /* a bounded device-side wait ran out                         */
} ehl_status;

/* Per-system / per-instance device info words (int32). */
enum {
  EHL_INFO_OK = 0,
  EHL_INFO_SINGULAR = 1,   /* |det| of a 2x2 pivot below 1e-300 relative to the pivot block */
  EHL_INFO_NOCONV = 2,     /* mode 2 active-set loop or Newton loop hit its limit           */
  EHL_INFO_NONFINITE = 3   /* NaN / Inf in the input or the result                          */
};

/* Human-readable name of a status code (static string, never NULL). */
const char* ehl_status_string(ehl_status s);

/* Library version as major*10000 + minor*100 + patch. */
int ehl_version(void);

/* ------------------------------------------------------------------------
 * PAQIF: batched projected alternate quadrant interlocking factorization
 * ------------------------------------------------------------------------
 * Defines: Sec. 2.1 (the linear complementarity problem, Eq. eqn14),
 * Sec. 2.2.1-2.2.3 (the factorization L0 = W0 Z0 with 2x2 pivots taken
 * from the middle of the matrix outwards, W0 Y = F solved from the middle
 * outwards and Z0 U = Y from both ends towards the middle), Sec. 2.2.2 and
 * Sec. 2.2.4 Steps 5 and 7 (projection of the computed solution onto
 * U >= 0).  One system is one partition (r = 1): the projection follows the
 * full solve.
 *
 * Solves n_sys independent banded systems A_s x_s = b_s of order n with
 * half-bandwidth beta.
 *
 *   band  [n_sys][n][2*beta+1] float64, row-major:
 *         band[s][i][j] = A_s[i][i - beta + j]; entries whose column lies
 *         outside [0, n) are ignored.
 *   rhs   [n_sys][n] float64.
 *   active (nullable) [n_sys][n] uint8: rows with active != 0 are replaced
 *         by the identity row with zero right-hand side (x_i = 0).
 *   mode  0: x = A^{-1} b
 *         1: x = max(0, A^{-1} b)         (solve, then project onto x >= 0)
 *         2: the LCP  x >= 0, w = A x - b >= 0, x^T w = 0, by a primal-dual
 *            active-set loop whose every step is one PAQIF solve with the
 *            current active rows pinned to zero; at most 64 steps.
 *   x     [n_sys][n] float64 output (may not alias band or rhs).
 *   iters (nullable) [n_sys] int32 output: PAQIF solves used per system.
 *   info  (nullable) [n_sys] int32 output: EHL_INFO_* per system.
 *   workspace / workspace_bytes: device scratch of at least
 *         ehl_paqif_workspace_size() bytes, 256-byte aligned; if workspace is
 *         NULL the call allocates it with cudaMallocAsync on `stream` and
 *         releases it with cudaFreeAsync after the kernel (stream-ordered).
 *
 * Limits: 1 <= beta <= 8, 2 <= n <= 1<<24, 1 <= n_sys <= 1<<24.
 * Odd n is handled by one extra decoupled identity row (x_n = 0) at the end.
 * Arithmetic: pairs of float32 carrying a float64-class result (about 48
 * significant bits); inputs and outputs are float64.
 * Returns EHL_EINVAL for bad sizes/modes/NULL pointers, EHL_ENOMEM if the
 * internal allocation fails, EHL_ECUDA if the launch fails, else EHL_OK
 * (asynchronous: per-system failures are reported through `info`).
 */
ehl_status ehl_paqif_workspace_size(int n_sys, int n, int beta, int mode, size_t* bytes);

ehl_status ehl_paqif_solve(int n_sys, int n, int beta, const double* band, const double* rhs,
                           const uint8_t* active, int mode, double* x, int* iters, int* info,
                           void* workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------
 * PAQIF without any allocation
 * ------------------------------------------------------------------------
 * The paper has no counterpart to this entry point: it exists for callers
 * that cannot allocate device memory while they solve -- for example a host
 * program whose own pool owns the whole GPU and forbids other allocations, a
 * plug-in running inside another application's callback where allocation is
 * not allowed, or a real-time loop that may neither wait on the allocator nor
 * fail with out-of-memory halfway through a run.
 *
 * Same arguments, semantics and results as ehl_paqif_solve, without the
 * workspace arguments: the scratch lives in one fixed device array of
 * EHL_PAQIF_STATIC_SCRATCH_BYTES that the library reserves on every GPU that
 * loads it, until the process exits.  The call allocates and frees nothing.
 *
 *  - Size limit: returns EHL_EINVAL when ehl_paqif_workspace_size() for the
 *    batch exceeds EHL_PAQIF_STATIC_SCRATCH_BYTES (for example n_sys = 128,
 *    n = 1024, beta = 4 needs about 10 MB and fits; 4096 such systems do not).
 *  - Set-up: the first call on each device looks up the array's device
 *    address (cudaGetSymbolAddress) with that device current and caches it;
 *    make that first call before any stream capture.  A failed lookup returns
 *    EHL_ECUDA.
 *  - Sharing: all calls on a device use the same array and it keeps the last
 *    call's contents.  Each call overwrites every scratch word it reads, so no
 *    clearing is needed, but calls whose GPU work overlaps in time (different
 *    streams, or other host threads) race on the array: serialise them.
 */
#define EHL_PAQIF_STATIC_SCRATCH_BYTES (16u << 20)

ehl_status ehl_paqif_solve_static(int n_sys, int n, int beta, const double* band, const double* rhs,
                                  const uint8_t* active, int mode, double* x, int* iters, int* info,
                                  void* stream);

#ifdef __cplusplus
}
#endif

#endif /* EHL_GB300_H */
