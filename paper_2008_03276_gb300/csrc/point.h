// point.h -- host-side state and stage launchers of the point-contact path.
#pragma once
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "ehl_internal.h"
#include "fft.h"
#include "line_kernels.cuh"

namespace ehl {

// One point-contact instance: the lubricant constants (in the line record, whose
// fields line_material reads) and the grid.
struct PointInst {
  LineInst m;  // lam, abar, alpha, p0, z, pH, compressible, elastic, limiter, tol, h_init, M, L
  int nx, ny;
  double xa, ya, h;
};

// kernels a device-driven solve graph holds outside its loops and in each loop body
struct PtGraphCounts {
  long long fixed = 0, newton = 0, krylov = 0, trial = 0;
};

struct PtCtx {
  int n_inst = 0, nx = 0, ny = 0, NN = 0, n = 0, lines = 0, beta = 2, max_iter = 0, m = 30;
  cudaStream_t st = nullptr;
  std::vector<PointInst> h_inst;
  PointInst* inst = nullptr;
  float2* gtab = nullptr;    // (2/pi^2) G(a, b) as double-float, [n_inst][ny][nx] (b = y offset)
  double* gtab64 = nullptr;  // the same in float64
  int ksplit = 1, nblk = 1, nvb = 1;
  void* partial = nullptr;   // [ksplit][n_inst][NN] double or float2
  double *H = nullptr, *rho = nullptr, *drho = nullptr, *deta_rel = nullptr, *eps = nullptr, *u = nullptr;
  double *F = nullptr, *psia = nullptr, *psib = nullptr, *R = nullptr, *Pw = nullptr, *dH = nullptr;
  double *blk = nullptr, *red = nullptr, *H0w = nullptr, *best = nullptr;
  int *done = nullptr, *iters = nullptr, *stall = nullptr;
  double *band = nullptr, *jh = nullptr, *dg = nullptr, *rhs = nullptr, *sigma = nullptr;
  uint8_t* act = nullptr;
  void* pq_ws = nullptr;
  int pq_r = 0;  // partitions per x-line system of the Krylov preconditioner: 0 the rule, else autotuned
  // graph mode 2: the grid's iteration as one graph with device-side loops
  int graph_mode = 0;
  int* loop = nullptr;  // [8] loop counters and totals (newton, krylov, trial, krylov total, trial total)
  double* jc = nullptr; // [n_inst][NN][4] Jacobian-product factors of the current Newton step
  cudaStream_t gs0 = nullptr, gs1 = nullptr, gs2 = nullptr;
  cudaEvent_t gev = nullptr;
  cudaGraphExec_t graph = nullptr;
  const double *g_P = nullptr, *g_H0 = nullptr, *g_rough = nullptr;
  PtGraphCounts gcounts;
  int* pq_info = nullptr;
  void* fstore = nullptr;
  // Newton-Krylov
  double *V = nullptr, *Z = nullptr, *Hh = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *w = nullptr;
  double *phinorm = nullptr, *zH = nullptr, *den = nullptr, *delta = nullptr, *Pt = nullptr, *H0t = nullptr;
  double *tstep = nullptr, *rtol = nullptr, *beta0 = nullptr, *znode = nullptr, *dots = nullptr, *hcol = nullptr;
  double* zh0 = nullptr;  // border component of the current preconditioned vector, per instance
  int *gm_k = nullptr, *gm_conv = nullptr, *lsdone = nullptr, *lsphase = nullptr, *skip = nullptr;
  int* acc = nullptr;     // line search: trial accepted in this pass
  void* adj = nullptr;    // adjoint buffers (point_newton.cu), allocated on first use
  // mixed-precision Krylov products (precision > 0): the deformation as one GEMM per instance,
  // T_all [nx][nx*ny] (the x-Toeplitz blocks of every y offset) times the shifted sums of the rows
  int precision = 0;
  cublasHandle_t blas = nullptr;
  float *Tall = nullptr, *Qf = nullptr, *Df = nullptr;
  int trace = 0;
  // deformation by the float64 FFT convolution (fft.cu) instead of the direct sum: the film of the
  // residual and the Krylov products (their inputs vanish on the boundary nodes); the adjoint's
  // transposed products, whose weights do not, keep the direct sum
  bool use_fft = false;
  Fft2 fft;
  // y-line stage of the preconditioner (yline = 1): after the bordered x-line solve z1 = M_x^-1 v,
  // z = z1 + M_y^-1 (v - J z1) with M_y the bordered solve on the y-line bands (grid columns)
  int yline = 0, ylines = 0;
  double *band_y = nullptr, *rhs_y = nullptr, *sig_y = nullptr, *zHy = nullptr, *deny = nullptr, *xiy = nullptr;
  void* pq_ws_y = nullptr;
  void* fstore_y = nullptr;
  int* pq_info_y = nullptr;
  std::vector<void*> allocs;
};

cudaError_t pt_alloc(PtCtx* c, void** p, size_t bytes);
ehl_status pt_init(PtCtx* c, const std::vector<PointInst>& insts, int beta, int max_iter, int krylov_dim,
                   int precision = 0, int deform = 0, int yline = 0, int autotune = 0);
void pt_free(PtCtx* c);
// state (film, lubricant, faces, residual, block partials) at (P, H0); all [n_inst][ny][nx]
cudaError_t pt_state(PtCtx* c, const double* P, const double* H0, const double* rough, const int* skip);
cudaError_t pt_finalize(PtCtx* c, int* done, int* iters);
// exact x-line band Jacobian: band [n_inst][ny-2][nx-2][2 beta + 1], act [n_inst][n]
cudaError_t pt_jac_band(PtCtx* c, const double* P, double* band, uint8_t* act, double* jh, double* dg,
                        const int* skip);
// exact y-line band Jacobian: band [n_inst][nx-2][ny-2][2 beta + 1] (one system per grid column),
// rows active in `act` (from pt_jac_band) identity, the others divided by dg when scale != 0
cudaError_t pt_jac_yband(PtCtx* c, const double* P, const uint8_t* act, const double* dg, double* band, int scale,
                         const int* skip);
cudaError_t pt_jacobian_apply(PtCtx* c, const double* P, const double* H0, const double* rough, const double* v,
                              const double* v_h0, double* out);
cudaError_t pt_start(PtCtx* c, double* P, double* H0, const double* rough);
// grid sequence: coarse values of a fine nodal array; bilinear prolongation of (Pw, H0w)
cudaError_t pt_inject(const PtCtx* fine, const double* src, PtCtx* coarse, double* dst);
cudaError_t pt_prolong(const PtCtx* coarse, PtCtx* fine);
// dH = K zn + zh0 (double-float deformation; the Krylov products)
cudaError_t pt_deform_dir(PtCtx* c, const double* zn, const double* zh0, const int* skip);
// dH = K v in float64 (the adjoint's products)
cudaError_t pt_deform_dir64(PtCtx* c, const double* v, const int* skip);
// Adjoint of a converged point-contact state (point_newton.cu): gradients of J(P, H, H0) from its
// partials gP, gH ([n_inst][ny][nx], nullable) and gH0 ([n_inst], nullable) with respect to the
// roughness (grad_rough, nullable) and (M, L) (grad_ML [n_inst][2], nullable); relres [n_inst]
cudaError_t pt_adjoint(PtCtx* c, const double* P, const double* H0, const double* rough, const double* gP,
                       const double* gH, const double* gH0, double* grad_rough, double* grad_ML, double* relres,
                       double tol, int max_cycles);
void pt_adj_free(PtCtx* c);
cudaError_t pt_nk_step(PtCtx* c, double* P, double* H0, const double* rough);
// graph mode 2: the Newton / GMRES / line-search loops of this grid captured on c->st (capturing)
cudaError_t pt_nk_capture_solve(PtCtx* c, double* P, double* H0, const double* rough, cudaStream_t s1, cudaStream_t s2,
                                PtGraphCounts& n);

}  // namespace ehl
