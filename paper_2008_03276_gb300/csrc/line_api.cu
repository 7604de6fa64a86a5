// line_api.cu -- extern "C" context API of include/ehl.h for line contact.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "ehl_internal.h"
#include "line.h"

using namespace ehl;

struct ehl_ctx {
  int dim;
  LineCtx line;
};

extern "C" void ehl_params_default(ehl_params* p, int dim) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->dim = dim;
  p->nx = 129;
  p->ny = 1;
  p->xa = -4.5;
  p->xb = 1.5;
  p->ya = -3.0;
  p->yb = 3.0;
  p->M = 20.0;
  p->L = 10.0;
  p->alpha = 1.7e-8;
  p->p0 = 1.98e8;
  p->z = 0.68;
  p->compressible = 1;
  p->elastic = 1;
  p->limiter = 0;
  p->halfband = 2;
  p->switch_eps_h = 0.6;
  p->dist_weight = 0.5;
  p->c_h0 = 0.05;
  p->omega = 1.0;
  p->method = 1;
  p->tol = 1e-8;
  p->max_iter = 200;
  p->krylov_dim = 40;
  p->h_init = 0.05;
}

static bool params_ok(const ehl_params& p) {
  return p.dim == 1 && p.nx >= 5 && p.nx <= 65536 && p.halfband >= 1 && p.halfband <= 8 && p.M > 0.0 &&
         p.L >= 0.0 && p.xb > p.xa && p.alpha > 0.0 && p.p0 > 0.0 && p.z > 0.0 && (p.limiter == 0 || p.limiter == 1) &&
         (p.method == 0 || p.method == 1) && p.max_iter >= 1 && p.krylov_dim >= 1 && p.krylov_dim <= 200 &&
         p.tol > 0.0 && isfinite(p.h_init) && isfinite(p.c_h0) && isfinite(p.omega) && isfinite(p.dist_weight) &&
         isfinite(p.switch_eps_h);
}

static LineInst make_inst(const ehl_params& p) {
  LineInst q;
  memset(&q, 0, sizeof(q));
  q.N = p.nx;
  q.beta = p.halfband;
  q.limiter = p.limiter;
  q.compressible = p.compressible ? 1 : 0;
  q.elastic = p.elastic ? 1 : 0;
  q.xa = p.xa;
  q.h = (p.xb - p.xa) / (p.nx - 1);
  q.lam = 3.0 * M_PI * M_PI / (8.0 * p.M * p.M);
  q.abar = p.L * sqrt(p.M / (2.0 * M_PI));
  q.alpha = p.alpha;
  q.p0 = p.p0;
  q.z = p.z;
  q.pH = q.abar / p.alpha;
  q.switch_eps_h = p.switch_eps_h;
  q.dist_w = p.dist_weight;
  q.c_h0 = p.c_h0;
  q.omega = p.omega;
  q.tol = p.tol;
  q.h_init = p.h_init;
  return q;
}

static void free_all(LineCtx* c) {
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  if (c->nk) line_nk_free(c);
}

extern "C" ehl_status ehl_create(const ehl_params* p, int n_inst, const ehl_params* per_inst, void* stream,
                                 ehl_ctx** out) {
  if (!p || !out || n_inst < 1 || n_inst > (1 << 20) || !params_ok(*p)) return EHL_EINVAL;
  if (per_inst) {
    for (int k = 0; k < n_inst; ++k) {
      const ehl_params& q = per_inst[k];
      if (!params_ok(q) || q.nx != p->nx || q.dim != p->dim || q.halfband != p->halfband || q.method != p->method)
        return EHL_EINVAL;
    }
  }
  ehl_ctx* ctx = new ehl_ctx();
  ctx->dim = p->dim;
  LineCtx* c = &ctx->line;
  c->n_inst = n_inst;
  c->N = p->nx;
  c->n = p->nx - 2;
  c->beta = p->halfband;
  c->method = p->method;
  c->max_iter = p->max_iter;
  c->krylov_dim = p->krylov_dim;
  c->st = (cudaStream_t)stream;
  c->h_inst.resize(n_inst);
  for (int k = 0; k < n_inst; ++k) c->h_inst[k] = make_inst(per_inst ? per_inst[k] : *p);
  c->ksplit = (c->N + 127) / 128;
  c->nblk = (c->N + 255) / 256;
  const size_t NN = (size_t)n_inst * c->N, nn = (size_t)n_inst * c->n;
  const size_t bw = 2 * c->beta + 1;
  bool ok = true;
  auto A = [&](void** ptr, size_t bytes) {
    if (ok && ctx_alloc(c, ptr, bytes) != cudaSuccess) ok = false;
  };
  A((void**)&c->inst, sizeof(LineInst) * n_inst);
  A((void**)&c->gtab, sizeof(float2) * NN);
  A((void**)&c->partial, sizeof(float2) * NN * c->ksplit);
  double** nodal[] = {&c->H, &c->rho, &c->drho, &c->deta_rel, &c->eps, &c->u, &c->F, &c->psi, &c->psia, &c->psib,
                      &c->R, &c->Pw, &c->dH};
  for (double** q : nodal) A((void**)q, sizeof(double) * NN);
  A((void**)&c->blk, sizeof(double) * n_inst * c->nblk * 4);
  A((void**)&c->red, sizeof(double) * n_inst * 4);
  A((void**)&c->band, sizeof(double) * nn * bw);
  A((void**)&c->rhs, sizeof(double) * nn);
  A((void**)&c->sigma, sizeof(double) * nn);
  A((void**)&c->jh, sizeof(double) * nn);
  A((void**)&c->dg, sizeof(double) * nn);
  A((void**)&c->act, nn);
  A((void**)&c->H0w, sizeof(double) * n_inst);
  A((void**)&c->done, sizeof(int) * n_inst);
  A((void**)&c->iters, sizeof(int) * n_inst);
  A((void**)&c->pq_info, sizeof(int) * n_inst);
  if (ok) {
    size_t wb = 0;
    ehl_paqif_workspace_size(n_inst, c->n, c->beta, 0, &wb);
    c->pq_ws_bytes = wb;
    A(&c->pq_ws, wb);
  }
  if (ok && c->method == 1 && line_nk_alloc(c) != cudaSuccess) ok = false;
  if (!ok) {
    cudaGetLastError();
    free_all(c);
    delete ctx;
    return EHL_ENOMEM;
  }
  cudaError_t e = cudaMemcpyAsync(c->inst, c->h_inst.data(), sizeof(LineInst) * n_inst, cudaMemcpyHostToDevice,
                                  c->st);
  if (e == cudaSuccess) e = line_init_tables(c);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_all(c);
    delete ctx;
    return EHL_ECUDA;
  }
  *out = ctx;
  return EHL_OK;
}

extern "C" ehl_status ehl_destroy(ehl_ctx* ctx) {
  if (!ctx) return EHL_EINVAL;
  cudaStreamSynchronize(ctx->line.st);
  free_all(&ctx->line);
  delete ctx;
  return EHL_OK;
}

static ehl_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return EHL_OK;
  cudaGetLastError();
  return EHL_ECUDA;
}

// (red [n_inst][4]) -> (comp_res [n_inst][2])
static cudaError_t copy_comp(LineCtx* c, double* comp_res) {
  return cudaMemcpy2DAsync(comp_res, 2 * sizeof(double), c->red, 4 * sizeof(double), 2 * sizeof(double), c->n_inst,
                           cudaMemcpyDeviceToDevice, c->st);
}

extern "C" ehl_status ehl_residual(ehl_ctx* ctx, const double* P, const double* H0, const double* rough, double* R,
                                   double* H, double* comp_res) {
  if (!ctx || !P || !H0 || !R) return EHL_EINVAL;
  LineCtx* c = &ctx->line;
  cudaError_t e = line_state(c, P, H0, rough, nullptr, nullptr);
  if (e == cudaSuccess) e = line_finalize(c, nullptr, nullptr);
  const size_t NN = (size_t)c->n_inst * c->N;
  if (e == cudaSuccess) e = cudaMemcpyAsync(R, c->R, sizeof(double) * NN, cudaMemcpyDeviceToDevice, c->st);
  if (e == cudaSuccess && H) e = cudaMemcpyAsync(H, c->H, sizeof(double) * NN, cudaMemcpyDeviceToDevice, c->st);
  if (e == cudaSuccess && comp_res) e = copy_comp(c, comp_res);
  return cuda_status(e);
}

extern "C" ehl_status ehl_jacobian_band(ehl_ctx* ctx, const double* P, const double* H0, const double* rough,
                                        int kind, double* band, uint8_t* active) {
  if (!ctx || !P || !H0 || !band || !active || (kind != 0 && kind != 1)) return EHL_EINVAL;
  LineCtx* c = &ctx->line;
  cudaError_t e = line_state(c, P, H0, rough, nullptr, nullptr);
  if (e == cudaSuccess) e = line_jac_band(c, P, kind, band, active, nullptr, nullptr, nullptr);
  return cuda_status(e);
}

extern "C" ehl_status ehl_jacobian_apply(ehl_ctx* ctx, const double* P, const double* H0, const double* rough,
                                         const double* v, const double* v_h0, double* out) {
  if (!ctx || !P || !H0 || !v || !v_h0 || !out) return EHL_EINVAL;
  return cuda_status(line_jacobian_apply(&ctx->line, P, H0, rough, v, v_h0, out));
}

extern "C" ehl_status ehl_solve(ehl_ctx* ctx, double* P, double* H0, const double* rough, int init, int* iters,
                                double* final_res) {
  if (!ctx || !P || !H0 || (init != 0 && init != 1)) return EHL_EINVAL;
  LineCtx* c = &ctx->line;
  const size_t NN = (size_t)c->n_inst * c->N;
  cudaError_t e = cudaSuccess;
  if (init == 1) {
    e = cudaMemcpyAsync(c->Pw, P, sizeof(double) * NN, cudaMemcpyDeviceToDevice, c->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->H0w, H0, sizeof(double) * c->n_inst, cudaMemcpyDeviceToDevice, c->st);
  } else {
    e = line_start(c, c->Pw, c->H0w, rough);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(c->done, 0, sizeof(int) * c->n_inst, c->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->iters, 0, sizeof(int) * c->n_inst, c->st);
  std::vector<int> hdone(c->n_inst, 0);
  const int check_every = 8;
  for (int it = 0; it < c->max_iter && e == cudaSuccess; ++it) {
    e = (c->method == 0) ? line_paper_iteration(c, c->Pw, c->H0w, rough) : line_nk_step(c, c->Pw, c->H0w, rough);
    if (e != cudaSuccess) break;
    if ((it + 1) % check_every == 0 || it + 1 == c->max_iter) {
      e = cudaMemcpyAsync(hdone.data(), c->done, sizeof(int) * c->n_inst, cudaMemcpyDeviceToHost, c->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
      bool all = true;
      for (int v : hdone) all = all && (v != 0);
      if (all) break;
    }
  }
  // final residual at the returned iterate
  if (e == cudaSuccess) e = line_state(c, c->Pw, c->H0w, rough, nullptr, nullptr);
  if (e == cudaSuccess) e = line_finalize(c, nullptr, nullptr);
  if (e == cudaSuccess) e = cudaMemcpyAsync(P, c->Pw, sizeof(double) * NN, cudaMemcpyDeviceToDevice, c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(H0, c->H0w, sizeof(double) * c->n_inst, cudaMemcpyDeviceToDevice, c->st);
  if (e == cudaSuccess && iters)
    e = cudaMemcpyAsync(iters, c->iters, sizeof(int) * c->n_inst, cudaMemcpyDeviceToDevice, c->st);
  if (e == cudaSuccess && final_res) e = copy_comp(c, final_res);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hdone.data(), c->done, sizeof(int) * c->n_inst, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return cuda_status(e);
  bool nonfinite = false, noconv = false;
  for (int v : hdone) {
    nonfinite = nonfinite || v == 2;
    noconv = noconv || v == 0;
  }
  return nonfinite ? EHL_ENONFINITE : (noconv ? EHL_ENOCONV : EHL_OK);
}
