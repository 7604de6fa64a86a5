// line.h -- host-side state and stage launchers of the line-contact path.
#pragma once
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "ehl_internal.h"
#include "line_kernels.cuh"

namespace ehl {

// kernels a device-driven solve graph holds outside its loops and in each loop body
struct SolveGraphCounts {
  long long fixed = 0, newton = 0, krylov = 0, trial = 0;
};

struct LineCtx {
  int n_inst = 0, N = 0, n = 0, beta = 2, method = 0, max_iter = 0, krylov_dim = 30;
  cudaStream_t st = nullptr;
  std::vector<LineInst> h_inst;
  LineInst* inst = nullptr;
  float2* gtab = nullptr;    // K_d / pi as double-float (Krylov products)
  double* gtab64 = nullptr;  // K_d / pi in float64 (the residual)
  int ksplit = 1, nblk = 1;
  float2* partial = nullptr;
  double *H = nullptr, *rho = nullptr, *drho = nullptr, *deta_rel = nullptr, *eps = nullptr, *u = nullptr;
  double *F = nullptr, *psi = nullptr, *psia = nullptr, *psib = nullptr, *R = nullptr;
  double *blk = nullptr, *red = nullptr;
  double *band = nullptr, *rhs = nullptr, *sigma = nullptr, *jh = nullptr, *dg = nullptr;
  uint8_t* act = nullptr;
  void* pq_ws = nullptr;
  size_t pq_ws_bytes = 0;
  int* pq_info = nullptr;
  int pq_parts = 1;  // Krylov preconditioner: PAQIF blocks per band (block Jacobi)
  int pq_r = 0;      // its partitions per system (Sec. 2.2.4): 0 the library's rule, else autotuned
  // mixed-precision Krylov products (precision > 0): dense float32 K, vectors, products
  int precision = 0;
  cublasHandle_t blas = nullptr;
  float *Kf = nullptr, *Vf = nullptr, *Df = nullptr;
  // precision 5: the hand-written TF32x3 tcgen05 product (tc_gemm.cu): tf32 hi / lo parts of K
  // and of the vectors, the plan (a TcGemm), its K-splits and its bounded-wait error flag
  float *Khi = nullptr, *Klo = nullptr, *Vhi = nullptr, *Vlo = nullptr;
  void* tc = nullptr;
  int tc_splits = 1;
  int* tc_err = nullptr;
  double *Pw = nullptr, *H0w = nullptr, *dH = nullptr;
  int *done = nullptr, *iters = nullptr;
  double* best = nullptr;  // smallest ||min(P,R)||_inf seen (stall test of the rounding-floor stop)
  int* stall = nullptr;    // outer iterations since it last halved
  int* loop0 = nullptr;    // graph mode 2 of the paper's iteration: pass counter of its while-loop
  std::vector<void*> allocs;
  // Newton-Krylov buffers (line_newton.cu)
  void* nk = nullptr;
  // adjoint buffers (line_adjoint.cu), allocated on first use
  void* adj = nullptr;
  // EHL_TRACE=k in the environment: one line per Newton step for the first k instances (stderr)
  int trace = 0;
  // small instances (N <= 256 for the state, N <= kNkSmallN for a Krylov step) run the stages of
  // one instance in one CTA, with the same arithmetic as the multi-kernel stages;
  // EHL_FUSE=0 in the environment turns this off (to check the two against each other)
  bool fuse = true;
  // graph mode: one Newton step captured as a CUDA graph (no host checks inside; the first
  // kGraphTrials line-search trials), replayed each outer iteration
  bool use_graph = false, capturing = false;
  // the state arrays (H, R, rho, eps, ...) hold the state at (Pw, H0w) of every instance: the
  // line search of the last Newton step evaluated and accepted it there
  bool state_current = false;
  cudaGraphExec_t graph = nullptr;
  int graph_mode = 0;                    // 0 host-driven, 1 one Newton step per graph, 2 the whole solve
  cudaStream_t gs1 = nullptr, gs2 = nullptr;  // mode 2: streams the loop bodies are captured on
  SolveGraphCounts gcounts;
  const double *g_P = nullptr, *g_H0 = nullptr, *g_rough = nullptr;  // pointers the graph was captured with
  long long graph_launches = 0;
};

cudaError_t ctx_alloc(LineCtx* c, void** p, size_t bytes);
cudaError_t line_deform(LineCtx* c, const double* V, int vstride, const int* skip);
cudaError_t line_state(LineCtx* c, const double* P, const double* H0, const double* rough, const int* skip,
                       int* unused);
cudaError_t line_finalize(LineCtx* c, int* done, int* iters);
// kind 0 (the paper's matrix) can also write the paper iteration's right-hand side (rhs_out) and
// PAQIF's int32 row flags (act32); kind 1 (exact) ignores them.
cudaError_t line_jac_band(LineCtx* c, const double* P, int kind, double* band, uint8_t* act, double* jh,
                          double* dg, const int* skip, double* rhs_out = nullptr, int* act32 = nullptr);
cudaError_t line_start(LineCtx* c, double* P, double* H0, const double* rough);
cudaError_t line_paper_iteration(LineCtx* c, double* P, double* H0, const double* rough);
// Graph mode 2 of the paper's iteration: the iterations of one grid as a device-side while-loop
// (the kernels of line_paper_iteration, done instances skipped) captured on c->st, which must be
// capturing; s1 is a stream of the same device for the loop body.  n.newton counts the kernels
// of one pass, n.fixed those outside the loop; c->loop0[0] holds the passes a replay ran.
cudaError_t line_paper_capture_solve(LineCtx* c, double* P, double* H0, const double* rough, cudaStream_t s1,
                                     SolveGraphCounts& n);
cudaError_t line_init_tables(LineCtx* c);
// The same sums in float64 (the residual's deformation; also the adjoint's products)
cudaError_t line_deform64(LineCtx* c, const double* V, int vstride, const int* skip);
// dH = -K v + zh0: the film's directional derivative (v in c->partial from line_deform, or
// from line_deform64 with p64)
cudaError_t line_film_dir(LineCtx* c, const double* zh0, const int* skip, bool p64 = false);
// (dR/dP) v + (dR/dH0) v_h0 at (P, H0); v nodal (zero at the boundary nodes)
cudaError_t line_jacobian_apply(LineCtx* c, const double* P, const double* H0, const double* rough, const double* v,
                                const double* v_h0, double* out);
// Grid sequence: dst[z][i] = src[z][i * (Nf - 1) / (Nc - 1)] (coarse values of a fine nodal array)
cudaError_t line_inject(const double* src, int Nf, double* dst, int Nc, int n_inst, cudaStream_t st);
// Linear prolongation of (P, H0) from a grid of Nc nodes to one of 2 Nc - 1; instances with
// cdone = 2 (non-finite on the coarse grid) keep their fine values.
cudaError_t line_prolong(const double* Pc, const double* H0c, const int* cdone, int Nc, double* Pf, double* H0f,
                         int n_inst, cudaStream_t st);
// Newton-Krylov method (line_newton.cu)
cudaError_t line_nk_alloc(LineCtx* c);
void line_nk_free(LineCtx* c);
cudaError_t line_nk_step(LineCtx* c, double* P, double* H0, const double* rough);
// line-search trials first_trial.. after a graph replay, for instances still searching
cudaError_t line_nk_finish(LineCtx* c, double* P, double* H0, const double* rough, int first_trial);
constexpr int kGraphTrials = 6;
// Graph mode 2: the whole iteration of one grid (Newton steps, their GMRES and line-search loops)
// captured as one graph with device-side while-loops.  Captured on c->st (which must be capturing
// when called); s1, s2 are streams of the same device for the loop bodies.  Counts hold the kernels
// captured outside the loops and in each loop body, to count the kernels a replay runs.
cudaError_t line_nk_capture_solve(LineCtx* c, double* P, double* H0, const double* rough, cudaStream_t s1,
                                  cudaStream_t s2, SolveGraphCounts& n);
long long line_nk_graph_launches(const SolveGraphCounts& n, const int* loop_host);
const int* line_nk_loop_counters(LineCtx* c);
// Adjoint of a converged state (line_adjoint.cu): gradients of an objective J(P, H, H0) given
// its partials gP, gH ([n_inst][N], nullable) and gH0 ([n_inst], nullable) with respect to the
// roughness (grad_rough [n_inst][N], nullable) and the Moes parameters (grad_ML [n_inst][2],
// nullable); relres [n_inst] (nullable) the relative residual of the transposed solve.
cudaError_t line_adjoint(LineCtx* c, const double* P, const double* H0, const double* rough, const double* gP,
                         const double* gH, const double* gH0, double* grad_rough, double* grad_ML, double* relres,
                         double tol, int max_cycles, int* cycles);
void line_adj_free(LineCtx* c);
// Krylov products dH = -K v + zh0 (double-float, or a float32-output GEMM with precision > 0)
cudaError_t line_mixed_init(LineCtx* c, int precision);
cudaError_t line_tc_init(LineCtx* c);
void line_mixed_free(LineCtx* c);
cudaError_t line_krylov_deform(LineCtx* c, const double* V, const double* zh0, const int* skip);

}  // namespace ehl
