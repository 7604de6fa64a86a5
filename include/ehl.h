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
  EHL_ENOMEM = 2,      /* device or host memory (or a host thread) not available      */
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

/* Number of CUDA kernels this library has launched in this process so far
 * (all devices, all streams; a monotone counter for instrumentation). */
unsigned long long ehl_kernel_launches(void);

/* ------------------------------------------------------------------------
 * PAQIF: batched projected alternate quadrant interlocking factorization
 * ------------------------------------------------------------------------
 * Defines: Sec. 2.1 (the linear complementarity problem, Eq. eqn14),
 * Sec. 2.2.1-2.2.3 (the factorization L0 = W0 Z0 with 2x2 pivots taken
 * from the middle of the matrix outwards, W0 Y = F solved from the middle
 * outwards and Z0 U = Y from both ends towards the middle), Sec. 2.2.2 and
 * Sec. 2.2.4 Steps 5 and 7 (projection of the computed solution onto
 * U >= 0).  The library picks the partition count r of Sec. 2.2.4 from the
 * batch shape (ehl_paqif_partitions); every r gives the same solution up to
 * rounding, and the projection follows the full solve.  For beta <= 4 in
 * modes 0 and 1 the solve runs a kernel with one lane per block side and
 * r in {1, 2, 4, 8, 16}, chosen by the same measure (elimination levels
 * plus 2 beta r for the reduced system) among the r whose blocks fit in
 * one round of its resident lanes; ehl_paqif_partitions reports the count
 * of the general kernel, which the other cases and the factor-once entry
 * points use.
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
 * Partitioned PAQIF
 * ------------------------------------------------------------------------
 * Defines: Sec. 2.1 (Eqs. eqn15, eqnn16: the system cut into r diagonal
 * blocks L0^(m) coupled through their first and last beta unknowns) and
 * Sec. 2.2.4 Steps 1-7 (each block factored and swept over its interior, a
 * reduced system of order 2 beta r for the blocks' outer unknowns, the
 * interiors solved from them).  The reduced system is solved by block
 * elimination without pivoting (not by the normal equations of Step 4), and
 * the projection of modes 1 and 2 (Steps 5, 7) is applied after the full
 * solve, so every admissible r gives the result of ehl_paqif_solve up to
 * rounding.
 *
 * Same arguments and semantics as ehl_paqif_solve, plus
 *   partitions  r >= 1 blocks per system; 0 chooses r from the batch shape
 *               (what ehl_paqif_solve does).  The blocks have the even order
 *               n_p = 2 ceil(n / 2r); an admissible r divides the lane groups
 *               of one CTA (4 warps, 8 at beta = 8, of 32 / (2 beta + 2)
 *               groups each: 32, 20, 16, 12, 8, 8, 8, 8 for beta = 1..8),
 *               and for r > 1 each block
 *               has n_p >= 2 beta + 2 and at least one row below n.
 * Returns EHL_EINVAL for an inadmissible r, otherwise as ehl_paqif_solve.
 * The workspace size depends on r (ehl_paqif_workspace_size_partitioned).
 */
ehl_status ehl_paqif_workspace_size_partitioned(int n_sys, int n, int beta, int partitions, int mode,
                                                size_t* bytes);

ehl_status ehl_paqif_solve_partitioned(int n_sys, int n, int beta, int partitions, const double* band,
                                       const double* rhs, const uint8_t* active, int mode, double* x,
                                       int* iters, int* info, void* workspace, size_t workspace_bytes,
                                       void* stream);

/* The partition count a batch is solved with (host only, no CUDA call).
 *   partitions  0: the automatic choice of ehl_paqif_solve (among the
 *               admissible r whose n_sys r lane groups fit in two rounds of
 *               the resident groups of the GPU, the one with the shortest
 *               chain per group: its sweep levels n_p/2 - beta plus 2 beta r
 *               for the reduced system; on a tie the larger r if it fits in
 *               one round); r >= 1: r itself if admissible
 *   *r          output
 * Returns EHL_EINVAL for bad sizes, a NULL r or an inadmissible r. */
ehl_status ehl_paqif_partitions(int n_sys, int n, int beta, int partitions, int* r);

/* Autotuning of the partition count for a batch shape (Sec. 2.2.4 leaves r
 * free; the best r depends on the batch size, the order and the GPU).  Times
 * every admissible r (1..32) on the caller's band / rhs (device arrays as for
 * ehl_paqif_solve; x receives a solution) with CUDA events: one untimed call,
 * then the best of `reps` (1..100).  best_r receives the fastest r, to pass to
 * ehl_paqif_solve_partitioned with a workspace of
 * ehl_paqif_workspace_size_partitioned(..., r, ...); ms_per_r (nullable, 32
 * floats) the best time of each r, -1 where r is not admissible.  Allocates
 * its workspace stream-ordered and synchronises the stream.  Returns
 * EHL_EINVAL, EHL_ENOMEM, EHL_ECUDA or a status of the timed solves. */
ehl_status ehl_paqif_autotune(int n_sys, int n, int beta, int mode, const double* band, const double* rhs,
                              double* x, int reps, void* stream, int* best_r, float* ms_per_r);

/* Factor once, resolve many (Sec. 2.2.1-2.2.3: the factorization L0 = W0 Z0
 * does not depend on the right-hand side; a new F runs the W0 Y = F sweep
 * with the stored multipliers and the Z0 U = Y sweep with the stored folded
 * pivot rows, and the partitioned reduced system of Sec. 2.2.4 with its
 * stored block factors).  This is what a Newton iteration's preconditioner
 * does between two Jacobian updates.
 *
 * ehl_paqif_factor_size: bytes of the factorization object of a batch
 *   (the per-level multipliers and Pi^-1 rows, the folded Z0 rows and the
 *   reduced-system factors, double-float), for the automatic partition
 *   count of ehl_paqif_partitions(..., 0, ...).
 * ehl_paqif_factor: factors the n_sys systems (band as for ehl_paqif_solve)
 *   into `factor` (device, >= ehl_paqif_factor_size bytes, 256-byte
 *   aligned, owned by the caller and kept unchanged until the next factor
 *   call on it) and solves them for `rhs` into x.
 * ehl_paqif_resolve: solves the factored systems for a new rhs into x; reads
 *   `factor` (and writes the rhs part of its folded rows: two resolves on
 *   one factorization must not overlap on the GPU).  band is not needed.
 *   mode  0 or 1 as for ehl_paqif_solve (no active rows, no LCP loop).
 *   info  (nullable) [n_sys] int32: EHL_INFO_* (the factor call reports a
 *         singular pivot; a resolve reports non-finite results).
 * Same limits as ehl_paqif_solve; stream-ordered, nothing is allocated.
 * Returns EHL_EINVAL for bad sizes, modes, NULL or misaligned pointers or a
 * factor_bytes below the size; EHL_ECUDA if a launch fails; else EHL_OK. */
ehl_status ehl_paqif_factor_size(int n_sys, int n, int beta, size_t* bytes);
ehl_status ehl_paqif_factor(int n_sys, int n, int beta, const double* band, const double* rhs, int mode, double* x,
                            int* info, void* factor, size_t factor_bytes, void* stream);
ehl_status ehl_paqif_resolve(int n_sys, int n, int beta, const double* rhs, int mode, double* x, int* info,
                             void* factor, size_t factor_bytes, void* stream);

/* ------------------------------------------------------------------------
 * EHL problem: context, residual, band Jacobian, solve
 * ------------------------------------------------------------------------
 * The problem statement is the paper's: given load and lubricant parameters
 * and a grid, find P >= 0 and the film H satisfying the Reynolds
 * complementarity problem with force balance (Sec. 3.3, Examples 5 and 6;
 * Sec. 3.3.4, Eq. eqn75).  Line contact (dim = 1), in Hertzian units:
 *   H_i = H0 + X_i^2/2 - sum_k K_{|i-k|} P_k + rough_i,  K_d = G_d / pi with
 *   the closed-form cell integral G_d of log|x - x'| (Sec. 3.3.1);
 *   R_i = (F_{i+1/2} - F_{i-1/2})/h - [eps_{i+1/2}(P_{i+1}-P_i)
 *         - eps_{i-1/2}(P_i-P_{i-1})]/h^2, F the limited face value of rho H
 *   (Sec. 3.3.3), eps = rho H^3 / (eta lambda) with Roelands eta and
 *   Dowson-Higginson rho;  P_i >= 0, R_i >= 0, P_i R_i = 0;  h sum P = pi/2.
 * lambda and alpha_bar = alpha p_H come from the Moes parameters:
 *   lambda = 3 pi^2 / (8 M^2), alpha_bar = L sqrt(M / (2 pi)).
 *
 * Arrays of one context are [n_inst][nx_max] with nx_max the largest nx of
 * its instances (nodal, including the two boundary nodes where P = 0): the
 * row of instance k holds its own nx_k nodes first; entries past nx_k are
 * neither read nor written.  H0 is [n_inst].  Band arrays are
 * [n_inst][nx_max - 2][2 beta + 1] and active [n_inst][nx_max - 2], padded
 * the same way.  A batch may mix grid sizes (ragged batch): instances are
 * grouped by nx and each group runs on its own stream, forked from and
 * joined back to the context's stream; with a single grid size the kernels
 * work on the caller's arrays in place.
 */
typedef struct ehl_ctx ehl_ctx;

typedef struct {
  int dim;              /* 1: line contact                                              */
  int nx, ny;           /* nodes incl. boundary nodes (ny = 1 for line contact)         */
  double xa, xb, ya, yb;/* domain                                                        */
  double M, L;          /* Moes load and lubricant parameters                           */
  double alpha;         /* pressure-viscosity coefficient [1/Pa] (1.7e-8)               */
  double p0, z;         /* Roelands constants (1.98e8, 0.68)                            */
  int compressible;     /* 1: Roelands + Dowson-Higginson; 0: rho = eta = 1             */
  int elastic;          /* 1: elastic deformation; 0: rigid surfaces                    */
  int limiter;          /* 0: minmod, 1: van Leer (limited, TVD); 2: the unlimited       */
                        /*   kappa-scheme of van Leer (Sec. 3.1, Eq. eqn41; Sec. 3.3.2,  */
                        /*   Eq. eqn56): psi = ((1 - kappa) a + (1 + kappa) b) / 2       */
  int halfband;         /* half-bandwidth beta of the band Jacobian, 1..8               */
  double switch_eps_h;  /* eps/h threshold of the hybrid splitting (0.6)                */
  double dist_weight;   /* weighted-change share per neighbour (line 0.5)               */
  double c_h0;          /* relaxation c of the force-balance H0 update (0.05)           */
  double omega;         /* relaxation of the pressure change (1.0)                      */
  int method;           /* 0: the paper's band Newton relaxation                        */
                        /* 1: Newton-Krylov, PAQIF band preconditioner (default)         */
  double tol;           /* converged when ||min(P,R)||_inf <= tol and |h sum P - pi/2| <= tol */
  int max_iter;         /* cap on outer iterations                                      */
  int krylov_dim;       /* GMRES basis size per Newton step (method 1; 40 line, 200 point) */
  double h_init;        /* Hertzian start: H0 chosen so that min H = h_init             */
  int levels;           /* nested iteration: coarse grids solved first (init = 0 only);  */
                        /*   -1 as many as allowed (default), 0 none                     */
  int coarse_min_nodes; /* coarsest grid keeps at least this many nodes (65)             */
  double coarse_tol;    /* tolerance of the coarse-grid solves, max(tol, coarse_tol) (1e-4) */
  int precond_blocks;   /* line contact, method 1: the band preconditioner is PAQIF on r  */
                        /*   diagonal blocks of each band (block Jacobi: couplings between */
                        /*   blocks dropped), r the largest divisor of nx - 2 not above    */
                        /*   precond_blocks with blocks of at least 32 rows; 1: one system */
  int precision;        /* method 1: arithmetic of the Krylov products K v (line and point) */
                        /*   and, in line contact, of the PAQIF preconditioner (>= 1:       */
                        /*   float32 sweeps)                                               */
                        /*   (the residual stays float64, so the converged answer does     */
                        /*   not depend on it): 0 double-float Toeplitz kernel; with one   */
                        /*   grid spacing per grid size, a float32-output GEMM of all     */
                        /*   instances: 1 float32, 2 float32 with cuBLAS's BF16x9        */
                        /*   emulation requested (cuBLAS may still choose a SIMT SGEMM),   */
                        /*   3 TF32 tensor cores, 4 BF16 tensor cores; point contact: one */
                        /*   GEMM [nx x nx ny] . [nx ny x ny] per instance from the        */
                        /*   block-Toeplitz structure of the 2-D kernel; 5 (line contact)   */
                        /*   the library's own tensor-core product: K and the vectors split */
                        /*   into TF32 hi + lo parts, three tcgen05 TF32 products with     */
                        /*   float32 accumulation (about 2^-21 relative)                   */
  int graph;            /* line contact, method 1: 1 = each Newton step is one CUDA graph  */
                        /*   launch (captured once, replayed; one host check per step);    */
                        /*   2 = the whole iteration of each grid is one graph launch: the  */
                        /*   Newton, GMRES and line-search loops run as device-side while   */
                        /*   loops whose conditions the kernels set from the instances'     */
                        /*   flags (no host round trip inside a grid; precision 0 or 5);  */
                        /*   line contact, method 0: 2 = the paper's iterations of each    */
                        /*   grid as one device-side while loop (same kernels, same        */
                        /*   iterates as 0), 1 is ignored;                                  */
                        /*   0 = launched kernel by kernel with early exits (default)      */
  double kappa;         /* kappa of limiter 2, -1..1 (0: Fromm, 1/3: third-order upwind    */
                        /*   biased, -1: second-order upwind)                              */
  int splitting;        /* Couette part of the kind-0 Newton matrix (method 0):             */
                        /*   0: the limiter frozen at the current iterate (Sec. 3.3.3);    */
                        /*   1: L_hs1, 2: L_hs2 (Sec. 3.3.2, Eqs. eqn57-eqn61): the upwind  */
                        /*   difference c (rho_i dH_i - rho_{i-1} dH_{i-1}) / h with        */
                        /*   c = (2 - kappa)/2 (L_hs1) or (2 - kappa)/2 + (1 - kappa)/4    */
                        /*   (L_hs2); the weighted-change distribution where eps/h is at   */
                        /*   most switch_eps_h in every case                               */
  int deform;           /* point contact: evaluation of the deformation sum (Sec. 3.3.1   */
                        /*   Case 2) in the film and the Krylov products:                   */
                        /*   0: the direct sum over all cells (the paper's);               */
                        /*   1: the same discrete convolution through a float64 FFT of     */
                        /*   cyclic length 2^ceil(log2(2 n - 3)) per direction (nx, ny up  */
                        /*   to 2049); the adjoint's products keep the direct sum          */
  int autotune;         /* method 1: 1 = at ehl_create, time every admissible PAQIF      */
                        /*   partition count on the shape of each grid's Krylov             */
                        /*   preconditioner (line: the bands; point: the x-line systems)   */
                        /*   with ehl_paqif_autotune on identity bands of that shape       */
                        /*   and keep the fastest for the context's life; 0 = the          */
                        /*   library's rule (ehl_paqif_partitions with 0)                  */
  int yline;            /* point contact: 1 adds the y-line stage to the preconditioner:    */
                        /*   z1 = M_x^-1 v, z = z1 + M_y^-1 (v - J z1), M_x and M_y the     */
                        /*   bordered PAQIF solves on the x- and y-line bands of the exact  */
                        /*   Jacobian (the alternating directions of Sec. 3.3.2-3.3.4); one */
                        /*   more Jacobian product and y-line solve per Krylov vector; 0   */
                        /*   x-lines only                                                  */
} ehl_params;

/* Fill *p with the defaults above for dimension `dim` (1). */
void ehl_params_default(ehl_params* p, int dim);

/* Create a context for n_inst instances.  `p` gives the shared settings; if
 * per_inst is not NULL it gives per-instance parameters (n_inst entries; dim,
 * halfband and method must equal p's, nx may differ: nx_max is the largest
 * of p->nx and the per-instance nx).  The context owns its device
 * workspace (allocated here with cudaMalloc) and enqueues on `stream`.
 * Returns EHL_EINVAL for invalid parameters (n_inst outside 1..65535, nx < 5
 * or > 65536, beta outside 1..8, M <= 0, xb <= xa, ...), EHL_ENOMEM,
 * EHL_ECUDA.  With levels != 0 the context also holds the coarse grids of
 * the nested iteration (nx_l - 1 = (nx - 1) / 2^l while that is an integer
 * and nx_l >= coarse_min_nodes), about as much memory again as the finest.
 * Two environment variables are read here, for line contact: EHL_TRACE=k
 * prints one line per Newton step of the first k instances to stderr;
 * EHL_FUSE=0 runs small instances through the stage kernels instead of the
 * one-CTA kernels (state for nx <= 256, Krylov step for nx <= 257), which
 * compute the same stages (to check the two against each other). */
ehl_status ehl_create(const ehl_params* p, int n_inst, const ehl_params* per_inst, void* stream, ehl_ctx** out);

/* Release the context and its device memory (synchronises its stream). */
ehl_status ehl_destroy(ehl_ctx* ctx);

/* Residual at (P, H0): R [n_inst][nx_max] (0 at boundary nodes), H (nullable)
 * [n_inst][nx_max] film thickness, comp_res (nullable) [n_inst][2] =
 * (||min(P,R)||_inf over interior nodes, h sum P - pi/2).  rough nullable.
 * Asynchronous. */
ehl_status ehl_residual(ehl_ctx* ctx, const double* P, const double* H0, const double* rough, double* R,
                        double* H, double* comp_res);

/* Band Jacobian at (P, H0), rows/columns = interior nodes (n = nx - 2),
 * band [n_inst][nx_max - 2][2 beta + 1] in the PAQIF row-major layout
 * (instance k fills its first n_k = nx_k - 2 rows), active
 * [n_inst][nx_max - 2] uint8.
 *  kind 0: the paper's limiter-based Newton matrix (Sec. 3.3.3-3.3.4):
 *          eps, rho and the limiter factor frozen, the film change through
 *          the kernel, the weighted-change distribution on the subregion
 *          eps/h <= switch_eps_h, truncated to the band; cavitated rows
 *          (P = 0, R > 0) are identity rows (active = 1).
 *  kind 1: the band of the exact Jacobian dR/dP; rows with P_i <= R_i / d_i
 *          are identity rows (active = 1), d_i = max(|dR_i/dP_i|, m_i / 10)
 *          with m_i the largest |entry| of the row's band (the Newton
 *          row scale; the diagonal alone can pass through zero).
 *  kind 2 (point contact only): the y-line bands of the exact Jacobian,
 *          band [n_inst][nx-2][ny-2][2 beta + 1] (one system per interior grid
 *          column, rows along y; the alternating direction of Sec. 3.3.2-3.3.4),
 *          with the identity rows and active flags of kind 1.
 * Point contact (dim = 2): kind 1 gives the x-line bands
 * [n_inst][ny-2][nx-2][2 beta + 1] (one system per interior grid row); kind 0
 * is line contact only.
 * Asynchronous. */
ehl_status ehl_jacobian_band(ehl_ctx* ctx, const double* P, const double* H0, const double* rough, int kind,
                             double* band, uint8_t* active);

/* Exact directional derivative of the residual at (P, H0):
 *   out = (dR/dP) v + (dR/dH0) v_h0,
 * every dependence on P included (the film through the kernel, rho, eta and
 * eps, the limiter on its current branch).  v [n_inst][nx_max] nodal with
 * zeros at the boundary nodes, v_h0 [n_inst], out [n_inst][nx_max] (0 at the
 * boundary).
 * This is the operator the Newton-Krylov method (method 1) iterates on; the
 * deformation of v uses the arithmetic the context's `precision` selects.
 * Asynchronous. */
ehl_status ehl_jacobian_apply(ehl_ctx* ctx, const double* P, const double* H0, const double* rough, const double* v,
                              const double* v_h0, double* out);

/* Solve every instance.  init = 0: start from the Hertzian pressure with
 * H0 chosen so that min H = h_init -- on the coarsest grid of the nested
 * iteration when the context has coarse grids, each finer grid then starting
 * from the linear interpolation of the solution below it where that solve
 * converged, else again from the Hertzian start (coarse grids solved to
 * max(tol, coarse_tol) in at most 40 Newton steps, the roughness sampled at
 * their nodes); init = 1:
 * start from the given P, H0 on the target grid.
 * On return P, H0 hold the last iterate, iters (nullable, [n_inst] int32)
 * the outer iterations on the target grid and final_res (nullable, [n_inst][2]) the residuals
 * as in ehl_residual.  Synchronises the stream (to test convergence); in a
 * ragged batch each grid-size group iterates on its own host thread and
 * stream, so groups with different iteration counts overlap on the GPU.
 * An instance has converged when ||min(P,R)||_inf <= tol and
 * |h sum P - pi/2| <= tol, or when the first has not halved for five outer
 * iterations and lies within 1e3 roundoff units of the largest term of R
 * (its rounding floor) with the force balance met.
 * Returns EHL_OK if every instance converged, EHL_ENOCONV if some reached
 * max_iter, EHL_ENONFINITE if some produced NaN/Inf. */
ehl_status ehl_solve(ehl_ctx* ctx, double* P, double* H0, const double* rough, int init, int* iters,
                     double* final_res);

/* Sensitivities of converged solutions (the paper stops at the solution;
 * these follow from its discrete problem by the implicit-function theorem).
 * At a converged (P, H0) -- as ehl_solve returns it -- for an objective
 * J(P, H, H0) with partial derivatives gP, gH ([n_inst][nx_max], nullable
 * = 0) and gH0 ([n_inst], nullable), P, H and H0 taken as independent:
 *   grad_rough [n_inst][nx_max] (nullable)  dJ/d rough at every node,
 *   grad_ML    [n_inst][2]      (nullable)  (dJ/dM, dJ/dL),
 *   relres     [n_inst]         (nullable)  relative residual reached by
 *              the transposed solve.
 * The rows with P_i > R_i / d_i (d_i as for ehl_jacobian_band kind 1) carry
 * the equation R_i = 0, the
 * others keep P_i = 0; the transposed bordered system of these equations is
 * solved by GMRES (a basis of max(krylov_dim, 120) vectors, restarted up to
 * max_cycles times) on the exact
 * transposed Jacobian, preconditioned by PAQIF on the transposed band, to
 * the relative residual tol.  H_c, H_min and integrals of P are functions of
 * (P, H) whose partials the caller supplies (e.g. through autograd).
 * Synchronises the stream.  Returns EHL_OK, EHL_ENOCONV if some instance
 * stayed above tol, EHL_ENONFINITE. */
ehl_status ehl_adjoint(ehl_ctx* ctx, const double* P, const double* H0, const double* rough, const double* gP,
                       const double* gH, const double* gH0, double* grad_rough, double* grad_ML, double* relres,
                       double tol, int max_cycles);

/* ------------------------------------------------------------------------
 * Linear convection-diffusion workload of the line splittings
 * ------------------------------------------------------------------------
 * Defines: Sec. 3.1, Examples 1 and 2 (L u = (a u)_x + (b u)_y - eps Lap u = f,
 * Dirichlet data), Eq. eqn41 (van Leer's kappa-scheme for the convective
 * term), Eqs. eqn48-eqn49 (the x-line splittings Ls0 and Ls1), solved by AQIF
 * line by line (Sec. 6 runs it with u = x^4 + y^4, eps = 1e-6).
 *
 * Grid: n x n nodes on [lo, hi]^2, h = (hi - lo) / (n - 1).  Arrays are
 * [n_inst][n][n] float64 with x fastest (index [z][j][i] for node (x_i, y_j));
 * every instance shares the parameters.  u carries the Dirichlet values on
 * its boundary nodes (never written); f is read at the interior nodes.
 * Convective face value F_{k+1/2} = u_k + (1-kappa)/4 (u_k - u_{k-1})
 * + (1+kappa)/4 (u_{k+1} - u_k), the node before the inflow boundary being the
 * linear extrapolation 2 u_0 - u_1; diffusion by the 5-point Laplacian.
 */
typedef struct {
  int n;            /* nodes per direction incl. the boundary, 5..16385             */
  double lo, hi;    /* the square [lo, hi]^2                                        */
  double a, b;      /* constant convection coefficients, a > 0, b >= 0             */
  double eps;       /* diffusion coefficient, >= 0                                  */
  double kappa;     /* kappa of the scheme, -1..1                                   */
  int splitting;    /* 0: Ls0 (line operator c = (2-kappa)/2 + (1-kappa)/4),       */
                    /* 1: Ls1 (c = (2-kappa)/2); the line operator is the upwind   */
                    /*    difference c a (u_i - u_{i-1}) / h plus the diffusion's    */
                    /*    x part and diagonal: tridiagonal                          */
  int order;        /* 0: x-lines one after another in increasing y, each from the */
                    /*    iterate its predecessors left (the paper's order);        */
                    /* 1: all x-lines of a sweep from the same iterate              */
  double omega;     /* relaxation of the change, > 0 (1)                           */
} ehl_cd_params;

/* r = f - L u at the interior nodes (r nullable, [n_inst][n][n], 0 on the
 * boundary) and rmax (nullable, [n_inst]) = max |r| per instance (NaN if any r
 * is NaN).  Asynchronous.  EHL_EINVAL for bad parameters or NULL u / f. */
ehl_status ehl_cd_residual(const ehl_cd_params* p, int n_inst, const double* u, const double* f, double* r,
                           double* rmax, void* stream);

/* Bytes of device workspace ehl_cd_relax needs (line matrices, right-hand
 * sides, changes and the PAQIF factors of the line operator). */
ehl_status ehl_cd_workspace_size(const ehl_cd_params* p, int n_inst, size_t* bytes);

/* `sweeps` x-line relaxation sweeps in place on u: for each x-line, the change
 * sigma solves L^0 sigma = f - L u (the current residual of the line) by
 * PAQIF (the line operator is factored once per call and resolved for every
 * line), then u += omega sigma.
 *   rmax_hist (nullable) [sweeps][n_inst]: max |f - L u| after each sweep.
 *   info (nullable) [n_inst] int32: EHL_INFO_* of the line solves.
 *   workspace: at least ehl_cd_workspace_size() bytes, 256-byte aligned, or
 *   NULL to allocate it stream-ordered (cudaMallocAsync / cudaFreeAsync).
 * Asynchronous.  EHL_EINVAL for bad parameters, u == f or a short workspace,
 * EHL_ENOMEM, EHL_ECUDA. */
ehl_status ehl_cd_relax(const ehl_cd_params* p, int n_inst, double* u, const double* f, int sweeps,
                        double* rmax_hist, int* info, void* workspace, size_t workspace_bytes, void* stream);

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
 *    EHL_ECUDA.  The address belongs to the device's primary context (the
 *    CUDA runtime's): after a cudaDeviceReset the cached address is stale,
 *    so do not call this entry point in a process that has reset the device.
 *  - Partitions: the solve always uses the automatic partition count of
 *    ehl_paqif_solve (partitions = 0); the size limit is checked against
 *    ehl_paqif_workspace_size() for that count.
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
