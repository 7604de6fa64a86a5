// line_api.cu -- extern "C" context API of include/ehl.h for line contact.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <thread>
#include <vector>

#include "ehl_internal.h"
#include "line.h"
#include "point.h"

using namespace ehl;

// A context holds one bucket (an internal LineCtx on its own stream) per
// distinct grid size.  Caller arrays are [n_inst][nx_max] (rows padded to the
// largest grid); each bucket works on compact [n_b][N_b] copies, gathered from
// and scattered back to the caller's rows.  When every instance has the same
// grid the single bucket works on the caller's arrays directly.
struct Bucket {
  LineCtx c;
  std::vector<LineCtx*> lv;  // coarse grids of the nested iteration, coarsest first
  std::vector<double*> lrough;  // roughness injected on each coarse grid
  std::vector<int> idx;      // caller instance of each bucket instance
  int* d_idx = nullptr;      // the same on the device
  double *Pb = nullptr, *H0b = nullptr, *rb = nullptr, *vb = nullptr, *vhb = nullptr, *ob = nullptr;
  double *gPb = nullptr, *gHb = nullptr, *gH0b = nullptr, *grb = nullptr, *gmlb = nullptr;  // adjoint I/O
  double* relw = nullptr;  // adjoint relative residuals [n_b]
  cudaEvent_t ev = nullptr;  // completion of the bucket's work on its stream
  bool own_stream = false;
};

struct ehl_ctx {
  int dim = 1;
  int n_inst = 0, nx_max = 0, beta = 0;
  bool direct = true;  // single bucket in caller order: no gather/scatter
  bool own_streams = false;  // buckets run on streams of their own (several buckets, or graphs)
  cudaStream_t st = nullptr;
  std::vector<Bucket*> buckets;
  PtCtx* pt = nullptr;  // point contact (dim 2): one grid for every instance
  std::vector<PtCtx*> ptlv;       // its coarse grids (nested iteration), coarsest first
  std::vector<double*> ptrough;   // roughness injected on each coarse grid
};

// dst[r][0:len] = src[idx[r]][0:len]  (gather, forward) or the reverse (scatter)
template <typename T>
__global__ void k_rows(const T* __restrict__ src, int sstride, T* __restrict__ dst, int dstride,
                       const int* __restrict__ idx, int rows, int len, int scatter) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    if (!scatter)
      dst[(size_t)r * dstride + i] = src[(size_t)idx[r] * sstride + i];
    else
      dst[(size_t)idx[r] * dstride + i] = src[(size_t)r * sstride + i];
  }
}

template <typename T>
static cudaError_t rows(cudaStream_t st, const T* src, int sstride, T* dst, int dstride, const int* idx,
                        int nrows, int len, bool scatter) {
  if (nrows <= 0 || len <= 0) return cudaSuccess;
  dim3 g((len + 255) / 256, nrows < 65535 ? nrows : 65535);
  k_rows<T><<<g, 256, 0, st>>>(src, sstride, dst, dstride, idx, nrows, len, scatter ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

extern "C" void ehl_params_default(ehl_params* p, int dim) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->dim = dim;
  p->nx = 129;
  p->ny = dim == 2 ? 129 : 1;
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
  p->krylov_dim = dim == 2 ? 200 : 40;  // the x-line preconditioner leaves the y-coupling to GMRES
  p->h_init = 0.05;
  p->levels = -1;
  p->coarse_min_nodes = 65;
  p->coarse_tol = 1e-4;
  p->precond_blocks = 1;
  p->precision = 0;
  p->graph = 0;
  p->kappa = 0.0;
  p->splitting = 0;
  p->deform = 0;
  p->autotune = 0;
  p->yline = 0;
}

// band rows of the identity matrix (the other entries already zero): the autotuner's input
__global__ void k_unit_diagonal(double* __restrict__ band, size_t rows, int bw, int beta) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < rows) band[t * bw + beta] = 1.0;
}

static bool point_grid_ok(const ehl_params& p) {
  if (p.dim != 2) return true;
  const double hx = (p.xb - p.xa) / (p.nx - 1), hy = (p.yb - p.ya) / (p.ny - 1);
  // graph mode 2 captures the Krylov products too: the cuBLAS GEMMs of precision 1-4 stay out
  return p.ny >= 5 && p.ny <= 4097 && p.nx <= 4097 && p.yb > p.ya && fabs(hx - hy) <= 1e-12 * hx && p.method == 1 &&
         p.graph != 1 && (p.graph != 2 || p.precision == 0 || p.deform == 1);
}

static bool params_ok(const ehl_params& p) {
  return (p.dim == 1 || p.dim == 2) && point_grid_ok(p) && p.nx >= 5 && p.nx <= 65536 && p.halfband >= 1 && p.halfband <= 8 && p.M > 0.0 &&
         p.L >= 0.0 && p.xb > p.xa && p.alpha > 0.0 && p.p0 > 0.0 && p.z > 0.0 && (p.limiter >= 0 && p.limiter <= 2) &&
         p.kappa >= -1.0 && p.kappa <= 1.0 && p.splitting >= 0 && p.splitting <= 2 &&
         (p.deform == 0 || (p.deform == 1 && p.dim == 2 && fft2_size_ok(p.nx, p.ny))) &&
         (p.yline == 0 || (p.yline == 1 && p.dim == 2)) && (p.autotune == 0 || p.autotune == 1) &&
         (p.method == 0 || p.method == 1) && p.max_iter >= 1 && p.krylov_dim >= 1 && p.krylov_dim <= 200 &&
         p.tol > 0.0 && isfinite(p.h_init) && isfinite(p.c_h0) && isfinite(p.omega) && isfinite(p.dist_weight) &&
         isfinite(p.switch_eps_h) && p.levels >= -1 && p.coarse_min_nodes >= 5 && p.coarse_tol > 0.0 &&
         p.precond_blocks >= 1 && p.precond_blocks <= 4096 && p.precision >= 0 && p.precision <= 5 &&
         (p.graph == 0 || p.graph == 1 || (p.graph == 2 && (p.precision == 0 || p.precision == 5))) &&
         (p.precision != 5 || p.dim == 1);
}

static LineInst make_inst(const ehl_params& p) {
  LineInst q;
  memset(&q, 0, sizeof(q));
  q.N = p.nx;
  q.beta = p.halfband;
  q.limiter = p.limiter;
  q.kappa = p.kappa;
  q.splitting = p.splitting;
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
  q.M = p.M;
  q.L = p.L;
  return q;
}

static void free_all(LineCtx* c) {
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  if (c->nk) line_nk_free(c);
  if (c->adj) line_adj_free(c);
  line_mixed_free(c);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  if (c->gs1) cudaStreamDestroy(c->gs1);
  if (c->gs2) cudaStreamDestroy(c->gs2);
  c->gs1 = c->gs2 = nullptr;
}

static void free_bucket(Bucket* b) {
  if (!b) return;
  if (b->c.st) cudaStreamSynchronize(b->c.st);
  for (LineCtx* l : b->lv) {
    free_all(l);
    delete l;
  }
  b->lv.clear();
  free_all(&b->c);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->own_stream && b->c.st) cudaStreamDestroy(b->c.st);
  delete b;
}

static void free_ctx(ehl_ctx* ctx) {
  for (Bucket* b : ctx->buckets) free_bucket(b);
  ctx->buckets.clear();
  delete ctx;
}

// Workspace and tables of one LineCtx for the given instances (all on grid N).
static ehl_status init_line(LineCtx* c, const std::vector<LineInst>& insts, int N, const ehl_params& p) {
  const int n_inst = (int)insts.size();
  if (const char* tr = getenv("EHL_TRACE")) c->trace = atoi(tr) > 0 ? atoi(tr) : 0;
  if (const char* fu = getenv("EHL_FUSE")) c->fuse = atoi(fu) != 0;
  c->n_inst = n_inst;
  c->N = N;
  c->n = N - 2;
  c->beta = p.halfband;
  c->method = p.method;
  c->max_iter = p.max_iter;
  c->krylov_dim = p.krylov_dim;
  c->h_inst = insts;
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
  A((void**)&c->gtab64, sizeof(double) * NN);
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
  A((void**)&c->best, sizeof(double) * n_inst);
  A((void**)&c->stall, sizeof(int) * n_inst);
  A((void**)&c->loop0, sizeof(int) * 8);
  // preconditioner blocks: the largest divisor r of n with r <= precond_blocks and n / r >= 32
  c->pq_parts = 1;
  if (p.method == 1)
    for (int r = p.precond_blocks; r > 1; --r)
      if (c->n % r == 0 && c->n / r >= 32) {
        c->pq_parts = r;
        break;
      }
  A((void**)&c->pq_info, sizeof(int) * n_inst * c->pq_parts);
  c->pq_r = 0;
  if (ok && p.method == 1 && p.autotune == 1) {
    // the fastest partition count for the preconditioner's shape, timed on identity bands
    const int ns = n_inst * c->pq_parts, nb = c->n / c->pq_parts, bw = 2 * c->beta + 1;
    double *tb = nullptr, *tr = nullptr, *tx = nullptr;
    cudaError_t e = cudaMalloc(&tb, sizeof(double) * (size_t)ns * nb * bw);
    if (e == cudaSuccess) e = cudaMalloc(&tr, sizeof(double) * (size_t)ns * nb);
    if (e == cudaSuccess) e = cudaMalloc(&tx, sizeof(double) * (size_t)ns * nb);
    if (e == cudaSuccess) e = cudaMemsetAsync(tb, 0, sizeof(double) * (size_t)ns * nb * bw, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(tr, 0, sizeof(double) * (size_t)ns * nb, c->st);
    if (e == cudaSuccess) {
      k_unit_diagonal<<<(unsigned)(((size_t)ns * nb + 255) / 256), 256, 0, c->st>>>(tb, (size_t)ns * nb, bw,
                                                                                     c->beta);
      note_launch();
      e = cudaGetLastError();
    }
    int r = 0;
    if (e == cudaSuccess &&
        ehl_paqif_autotune(ns, nb, c->beta, 0, tb, tr, tx, 3, c->st, &r, nullptr) == EHL_OK && r > 0)
      c->pq_r = r;
    if (tb) cudaFree(tb);
    if (tr) cudaFree(tr);
    if (tx) cudaFree(tx);
    cudaGetLastError();
  }
  if (ok) {
    size_t wb = 0, wb2 = 0;
    ehl_paqif_workspace_size(n_inst, c->n, c->beta, 0, &wb);
    ehl_paqif_workspace_size_partitioned(n_inst * c->pq_parts, c->n / c->pq_parts, c->beta, c->pq_r, 0, &wb2);
    c->pq_ws_bytes = wb > wb2 ? wb : wb2;
    A(&c->pq_ws, c->pq_ws_bytes);
  }
  if (ok && c->method == 1 && line_nk_alloc(c) != cudaSuccess) ok = false;
  if (!ok) {
    cudaGetLastError();
    return EHL_ENOMEM;
  }
  cudaError_t e = cudaMemcpyAsync(c->inst, c->h_inst.data(), sizeof(LineInst) * n_inst, cudaMemcpyHostToDevice,
                                  c->st);
  if (e == cudaSuccess) e = line_init_tables(c);
  if (e == cudaSuccess && c->method == 1) e = line_mixed_init(c, p.precision);
  if (e == cudaSuccess) e = paqif_prepare(c->beta);  // no attribute calls inside a graph capture
  c->use_graph = c->method == 1 && p.graph == 1;
  c->graph_mode = (c->method == 1 || p.graph == 2) ? p.graph : 0;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return EHL_ECUDA;
  }
  return EHL_OK;
}

// Grids of the nested iteration below N (finest excluded), coarsest first:
// halve the intervals while their number stays even and the coarse grid
// keeps at least `min_nodes` nodes, at most `levels` times (-1: no cap).
static std::vector<int> coarse_grids(int N, int levels, int min_nodes) {
  std::vector<int> g;
  int n = N;
  while ((n - 1) % 2 == 0 && (n - 1) / 2 + 1 >= min_nodes && (levels < 0 || (int)g.size() < levels)) {
    n = (n - 1) / 2 + 1;
    g.push_back(n);
  }
  return std::vector<int>(g.rbegin(), g.rend());
}

// One bucket: the finest-grid LineCtx, its coarse grids and the gather buffers.
static ehl_status init_bucket(Bucket* b, const ehl_params& p0, const std::vector<const ehl_params*>& ps,
                              bool gather) {
  const int n_inst = (int)ps.size();
  std::vector<LineInst> insts(n_inst);
  for (int k = 0; k < n_inst; ++k) insts[k] = make_inst(*ps[k]);
  ehl_status st = init_line(&b->c, insts, p0.nx, p0);
  if (st != EHL_OK) return st;
  for (int Nl : coarse_grids(p0.nx, p0.levels, p0.coarse_min_nodes)) {
    LineCtx* l = new LineCtx();
    l->st = b->c.st;
    b->lv.push_back(l);
    std::vector<LineInst> ci(n_inst);
    for (int k = 0; k < n_inst; ++k) {
      ehl_params q = *ps[k];
      q.nx = Nl;
      q.tol = q.tol > q.coarse_tol ? q.tol : q.coarse_tol;
      ci[k] = make_inst(q);
    }
    st = init_line(l, ci, Nl, p0);
    if (st != EHL_OK) return st;
    l->max_iter = std::min(p0.max_iter, kCoarseMaxIter);
    double* r = nullptr;
    if (ctx_alloc(l, (void**)&r, sizeof(double) * n_inst * (size_t)Nl) != cudaSuccess) {
      cudaGetLastError();
      return EHL_ENOMEM;
    }
    b->lrough.push_back(r);
  }
  LineCtx* c = &b->c;
  const size_t NN = (size_t)n_inst * c->N;
  bool ok = true;
  auto A = [&](void** ptr, size_t bytes) {
    if (ok && ctx_alloc(c, ptr, bytes) != cudaSuccess) ok = false;
  };
  if (gather) {
    A((void**)&b->d_idx, sizeof(int) * n_inst);
    A((void**)&b->Pb, sizeof(double) * NN);
    A((void**)&b->H0b, sizeof(double) * n_inst);
    A((void**)&b->rb, sizeof(double) * NN);
    A((void**)&b->vb, sizeof(double) * NN);
    A((void**)&b->vhb, sizeof(double) * n_inst);
    A((void**)&b->ob, sizeof(double) * NN);
    A((void**)&b->gPb, sizeof(double) * NN);
    A((void**)&b->gHb, sizeof(double) * NN);
    A((void**)&b->gH0b, sizeof(double) * n_inst);
    A((void**)&b->grb, sizeof(double) * NN);
    A((void**)&b->gmlb, sizeof(double) * 2 * n_inst);
  }
  A((void**)&b->relw, sizeof(double) * n_inst);
  if (ok && cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) ok = false;
  if (!ok) {
    cudaGetLastError();
    return EHL_ENOMEM;
  }
  cudaError_t e = cudaSuccess;
  if (gather) e = cudaMemcpyAsync(b->d_idx, b->idx.data(), sizeof(int) * n_inst, cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return EHL_ECUDA;
  }
  return EHL_OK;
}

static PointInst make_point(const ehl_params& p) {
  PointInst q;
  memset(&q, 0, sizeof(q));
  q.m = make_inst(p);
  // point-contact Moes conversion: lambda = (128 pi^3 / (3 M^4))^(1/3), alpha_bar = (L/pi)(3M/2)^(1/3)
  q.m.lam = cbrt(128.0 * M_PI * M_PI * M_PI / (3.0 * p.M * p.M * p.M * p.M));
  q.m.abar = (p.L / M_PI) * cbrt(1.5 * p.M);
  q.m.pH = q.m.abar / p.alpha;
  q.nx = p.nx;
  q.ny = p.ny;
  q.xa = p.xa;
  q.ya = p.ya;
  q.h = (p.xb - p.xa) / (p.nx - 1);
  return q;
}

static ehl_status create_point(const ehl_params* p, int n_inst, const ehl_params* per_inst, cudaStream_t stream,
                               ehl_ctx** out) {
  std::vector<PointInst> insts(n_inst);
  for (int k = 0; k < n_inst; ++k) {
    const ehl_params& q = per_inst ? per_inst[k] : *p;
    if (q.nx != p->nx || q.ny != p->ny || q.xa != p->xa || q.xb != p->xb || q.ya != p->ya || q.yb != p->yb)
      return EHL_EINVAL;
    insts[k] = make_point(q);
  }
  ehl_ctx* ctx = new ehl_ctx();
  ctx->dim = 2;
  ctx->n_inst = n_inst;
  ctx->nx_max = p->nx;
  ctx->beta = p->halfband;
  ctx->st = stream;
  ctx->pt = new PtCtx();
  ctx->pt->st = stream;
  if (const char* tr = getenv("EHL_TRACE")) ctx->pt->trace = atoi(tr) > 0 ? atoi(tr) : 0;
  ehl_status st = pt_init(ctx->pt, insts, p->halfband, p->max_iter, p->krylov_dim, p->precision, p->deform, p->yline, p->autotune);
  ctx->pt->graph_mode = p->graph;
  // coarse grids: halve the intervals in both directions while both stay even and
  // the coarse grid keeps coarse_min_nodes nodes per direction
  int gx = p->nx, gy = p->ny;
  std::vector<std::pair<int, int>> grids;
  while (st == EHL_OK && (gx - 1) % 2 == 0 && (gy - 1) % 2 == 0 && (gx - 1) / 2 + 1 >= p->coarse_min_nodes &&
         (gy - 1) / 2 + 1 >= p->coarse_min_nodes && (p->levels < 0 || (int)grids.size() < p->levels)) {
    gx = (gx - 1) / 2 + 1;
    gy = (gy - 1) / 2 + 1;
    grids.insert(grids.begin(), {gx, gy});
  }
  for (auto& gxy : grids) {
    if (st != EHL_OK) break;
    std::vector<PointInst> ci(n_inst);
    for (int k = 0; k < n_inst; ++k) {
      ehl_params q = per_inst ? per_inst[k] : *p;
      q.nx = gxy.first;
      q.ny = gxy.second;
      q.tol = q.tol > q.coarse_tol ? q.tol : q.coarse_tol;
      ci[k] = make_point(q);
    }
    PtCtx* l = new PtCtx();
    l->st = stream;
    l->trace = ctx->pt->trace;
    ctx->ptlv.push_back(l);
    st = pt_init(l, ci, p->halfband, std::min(p->max_iter, kCoarseMaxIter), p->krylov_dim, p->precision, p->deform, p->yline, p->autotune);
    l->graph_mode = p->graph;
    double* r = nullptr;
    if (st == EHL_OK && pt_alloc(l, (void**)&r, sizeof(double) * n_inst * (size_t)l->NN) != cudaSuccess) {
      cudaGetLastError();
      st = EHL_ENOMEM;
    }
    ctx->ptrough.push_back(r);
  }
  if (st != EHL_OK) {
    for (PtCtx* l : ctx->ptlv) {
      pt_free(l);
      delete l;
    }
    pt_free(ctx->pt);
    delete ctx->pt;
    delete ctx;
    return st;
  }
  *out = ctx;
  return EHL_OK;
}

static ehl_status ehl_create_impl(const ehl_params* p, int n_inst, const ehl_params* per_inst, void* stream,
                                 ehl_ctx** out) {
  if (!p || !out || n_inst < 1 || n_inst > 65535 || !params_ok(*p)) return EHL_EINVAL;
  if (p->dim == 2) {
    if (per_inst)
      for (int k = 0; k < n_inst; ++k)
        if (!params_ok(per_inst[k]) || per_inst[k].dim != 2 || per_inst[k].halfband != p->halfband)
          return EHL_EINVAL;
    return create_point(p, n_inst, per_inst, (cudaStream_t)stream, out);
  }
  int nx_max = p->nx;
  if (per_inst) {
    for (int k = 0; k < n_inst; ++k) {
      const ehl_params& q = per_inst[k];
      if (!params_ok(q) || q.dim != p->dim || q.halfband != p->halfband || q.method != p->method) return EHL_EINVAL;
      nx_max = q.nx > nx_max ? q.nx : nx_max;
    }
  }
  // buckets by grid size, in order of first appearance
  std::vector<int> sizes;
  std::vector<std::vector<int>> members;
  for (int k = 0; k < n_inst; ++k) {
    const int nx = per_inst ? per_inst[k].nx : p->nx;
    size_t q = 0;
    while (q < sizes.size() && sizes[q] != nx) ++q;
    if (q == sizes.size()) {
      sizes.push_back(nx);
      members.emplace_back();
    }
    members[q].push_back(k);
  }
  ehl_ctx* ctx = new ehl_ctx();
  ctx->dim = p->dim;
  ctx->n_inst = n_inst;
  ctx->nx_max = nx_max;
  ctx->beta = p->halfband;
  ctx->st = (cudaStream_t)stream;
  ctx->direct = sizes.size() == 1;
  // a graph cannot be captured on the legacy default stream the caller may pass
  ctx->own_streams = !ctx->direct || (p->graph >= 1 && p->method == 1) || p->graph == 2;
  for (size_t q = 0; q < sizes.size(); ++q) {
    Bucket* b = new Bucket();
    ctx->buckets.push_back(b);
    b->idx = members[q];
    if (!ctx->own_streams) {
      b->c.st = ctx->st;
    } else {
      if (cudaStreamCreateWithFlags(&b->c.st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        free_ctx(ctx);
        return EHL_ECUDA;
      }
      b->own_stream = true;
    }
    std::vector<const ehl_params*> ps;
    for (int k : b->idx) ps.push_back(per_inst ? &per_inst[k] : p);
    ehl_params p0 = *ps[0];
    p0.halfband = p->halfband;
    p0.method = p->method;
    p0.levels = p->levels;
    p0.coarse_min_nodes = p->coarse_min_nodes;
    p0.precision = p->precision;
    p0.graph = p->graph;
    const ehl_status st = init_bucket(b, p0, ps, !ctx->direct);
    if (st != EHL_OK) {
      free_ctx(ctx);
      return st;
    }
  }
  *out = ctx;
  return EHL_OK;
}

extern "C" ehl_status ehl_destroy(ehl_ctx* ctx) {
  if (!ctx) return EHL_EINVAL;
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  if (ctx->pt) {
    for (PtCtx* l : ctx->ptlv) {
      pt_free(l);
      delete l;
    }
    ctx->ptlv.clear();
    pt_free(ctx->pt);
    delete ctx->pt;
    ctx->pt = nullptr;
  }
  free_ctx(ctx);
  return EHL_OK;
}

static ehl_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return EHL_OK;
  cudaGetLastError();
  return EHL_ECUDA;
}

// bucket streams wait for the caller's stream (fork) and the caller's stream for them (join)
static cudaError_t fork(ehl_ctx* ctx) {
  if (!ctx->own_streams) return cudaSuccess;
  cudaEvent_t e0;
  cudaError_t e = cudaEventCreateWithFlags(&e0, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->st);
  for (Bucket* b : ctx->buckets)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->c.st, e0, 0);
  cudaEventDestroy(e0);
  return e;
}
static cudaError_t join(ehl_ctx* ctx) {
  if (!ctx->own_streams) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  for (Bucket* b : ctx->buckets) {
    if (e == cudaSuccess) e = cudaEventRecord(b->ev, b->c.st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->st, b->ev, 0);
  }
  return e;
}

// caller [n_inst][stride] rows -> bucket compact rows (or the caller pointer when direct)
static const double* gin(ehl_ctx* ctx, Bucket* b, const double* src, int stride, int len, double* buf,
                         cudaError_t& e) {
  if (!src) return nullptr;
  if (ctx->direct) return src;
  if (e == cudaSuccess) e = rows(b->c.st, src, stride, buf, len, b->d_idx, (int)b->idx.size(), len, false);
  return buf;
}

static cudaError_t bucket_state(ehl_ctx* ctx, Bucket* b, const double* P, const double* H0, const double* rough) {
  LineCtx* c = &b->c;
  cudaError_t e = cudaSuccess;
  const double* Pb = gin(ctx, b, P, ctx->nx_max, c->N, b->Pb, e);
  const double* H0b = gin(ctx, b, H0, 1, 1, b->H0b, e);
  const double* rb = gin(ctx, b, rough, ctx->nx_max, c->N, b->rb, e);
  if (e == cudaSuccess) e = line_state(c, Pb, H0b, rb, nullptr, nullptr);
  if (e == cudaSuccess) e = line_finalize(c, nullptr, nullptr);
  return e;
}

// (red [n][4]) -> (comp_res rows of 2)
static cudaError_t put_comp(ehl_ctx* ctx, Bucket* b, double* comp_res) {
  LineCtx* c = &b->c;
  if (ctx->direct)
    return cudaMemcpy2DAsync(comp_res, 2 * sizeof(double), c->red, 4 * sizeof(double), 2 * sizeof(double),
                             c->n_inst, cudaMemcpyDeviceToDevice, c->st);
  return rows(c->st, (const double*)c->red, 4, comp_res, 2, b->d_idx, c->n_inst, 2, true);
}

template <typename T>
static cudaError_t put_rows(ehl_ctx* ctx, Bucket* b, const T* src, int len, T* dst, int dstride) {
  LineCtx* c = &b->c;
  if (ctx->direct) return cudaMemcpyAsync(dst, src, sizeof(T) * len * c->n_inst, cudaMemcpyDeviceToDevice, c->st);
  return rows(c->st, src, len, dst, dstride, b->d_idx, c->n_inst, len, true);
}

// ------------------------------------------------------------ point contact
static cudaError_t pt_put_comp(PtCtx* c, double* comp_res) {
  return cudaMemcpy2DAsync(comp_res, 2 * sizeof(double), c->red, 4 * sizeof(double), 2 * sizeof(double), c->n_inst,
                           cudaMemcpyDeviceToDevice, c->st);
}

static ehl_status pt_residual_api(ehl_ctx* ctx, const double* P, const double* H0, const double* rough, double* R,
                                  double* H, double* comp_res) {
  PtCtx* c = ctx->pt;
  const size_t NNt = (size_t)c->n_inst * c->NN;
  cudaError_t e = pt_state(c, P, H0, rough, nullptr);
  if (e == cudaSuccess) e = pt_finalize(c, nullptr, nullptr);
  if (e == cudaSuccess) e = cudaMemcpyAsync(R, c->R, sizeof(double) * NNt, cudaMemcpyDeviceToDevice, c->st);
  if (e == cudaSuccess && H) e = cudaMemcpyAsync(H, c->H, sizeof(double) * NNt, cudaMemcpyDeviceToDevice, c->st);
  if (e == cudaSuccess && comp_res) e = pt_put_comp(c, comp_res);
  return cuda_status(e);
}

// outer iterations of one point-contact grid from (Pw, H0w); done flags in hdone
// Graph mode 2 for point contact: the grid's iteration is one graph with device-side loops,
// captured on a private stream (a capture needs one; the caller's may be the legacy stream)
// forked from and joined back to the context's stream.
static cudaError_t pt_iterate_device_graph(PtCtx* c, const double* rough, std::vector<int>& hdone) {
  cudaError_t e = cudaSuccess;
  if (!c->gs1) {
    e = cudaStreamCreateWithFlags(&c->gs0, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->gs1, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->gs2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->gev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  const cudaStream_t user = c->st;
  e = cudaEventRecord(c->gev, user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->gs0, c->gev, 0);
  if (e != cudaSuccess) return e;
  c->st = c->gs0;
  if (!c->graph || c->g_P != c->Pw || c->g_H0 != c->H0w || c->g_rough != rough) {
    if (c->graph) {
      cudaGraphExecDestroy(c->graph);
      c->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    const unsigned long long l0 = thread_launches();
    e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      PtGraphCounts n;
      const cudaError_t es = pt_nk_capture_solve(c, c->Pw, c->H0w, rough, c->gs1, c->gs2, n);
      e = cudaStreamEndCapture(c->st, &g);
      add_launches(-(long long)(thread_launches() - l0));  // captured, not run
      if (es != cudaSuccess) e = es;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e == cudaSuccess) {
        c->gcounts = n;
        c->g_P = c->Pw;
        c->g_H0 = c->H0w;
        c->g_rough = rough;
      } else {
        c->graph = nullptr;
        cudaGetLastError();
      }
    }
  }
  int loops[8] = {0};
  if (e == cudaSuccess) e = cudaGraphLaunch(c->graph, c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(loops, c->loop, sizeof(loops), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hdone.data(), c->done, sizeof(int) * c->n_inst, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e == cudaSuccess)
    add_launches(c->gcounts.fixed + (long long)loops[0] * c->gcounts.newton +
                 (long long)loops[3] * c->gcounts.krylov + (long long)loops[4] * c->gcounts.trial);
  c->st = user;
  return e;
}

static cudaError_t pt_iterate(PtCtx* c, const double* rough, std::vector<int>& hdone) {
  const int ni = c->n_inst;
  if (c->graph_mode == 2) {
    hdone.assign(ni, 0);
    return pt_iterate_device_graph(c, rough, hdone);
  }
  cudaError_t e = cudaMemsetAsync(c->done, 0, sizeof(int) * ni, c->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->iters, 0, sizeof(int) * ni, c->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->best, 0x7f, sizeof(double) * ni, c->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->stall, 0, sizeof(int) * ni, c->st);
  hdone.assign(ni, 0);
  for (int it = 0; it < c->max_iter && e == cudaSuccess; ++it) {
    e = pt_nk_step(c, c->Pw, c->H0w, rough);
    if (e != cudaSuccess) break;
    e = cudaMemcpyAsync(hdone.data(), c->done, sizeof(int) * ni, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    bool all = true;
    for (int v : hdone) all = all && (v != 0);
    if (all) break;
  }
  return e;
}

static ehl_status pt_solve_api(ehl_ctx* ctx, double* P, double* H0, const double* rough, int init, int* iters,
                               double* final_res) {
  PtCtx* c = ctx->pt;
  const int ni = c->n_inst;
  const size_t NNt = (size_t)ni * c->NN;
  cudaError_t e = cudaSuccess;
  std::vector<int> hdone(ni, 0);
  if (init == 1) {
    e = cudaMemcpyAsync(c->Pw, P, sizeof(double) * NNt, cudaMemcpyDeviceToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->H0w, H0, sizeof(double) * ni, cudaMemcpyDeviceToDevice, c->st);
  } else {
    PtCtx* prev = nullptr;
    for (size_t l = 0; l < ctx->ptlv.size() && e == cudaSuccess; ++l) {
      PtCtx* cl = ctx->ptlv[l];
      const double* rl = nullptr;
      if (rough) {
        e = pt_inject(c, rough, cl, ctx->ptrough[l]);
        rl = ctx->ptrough[l];
      }
      if (e == cudaSuccess) e = pt_start(cl, cl->Pw, cl->H0w, rl);
      if (e == cudaSuccess && prev) e = pt_prolong(prev, cl);
      if (e == cudaSuccess) e = pt_iterate(cl, rl, hdone);
      prev = cl;
    }
    if (e == cudaSuccess) e = pt_start(c, c->Pw, c->H0w, rough);
    if (e == cudaSuccess && prev) e = pt_prolong(prev, c);
  }
  if (e == cudaSuccess) e = pt_iterate(c, rough, hdone);
  if (e == cudaSuccess) e = pt_state(c, c->Pw, c->H0w, rough, nullptr);
  if (e == cudaSuccess) e = pt_finalize(c, nullptr, nullptr);
  if (e == cudaSuccess) e = cudaMemcpyAsync(P, c->Pw, sizeof(double) * NNt, cudaMemcpyDeviceToDevice, c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(H0, c->H0w, sizeof(double) * ni, cudaMemcpyDeviceToDevice, c->st);
  if (e == cudaSuccess && iters)
    e = cudaMemcpyAsync(iters, c->iters, sizeof(int) * ni, cudaMemcpyDeviceToDevice, c->st);
  if (e == cudaSuccess && final_res) e = pt_put_comp(c, final_res);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hdone.data(), c->done, sizeof(int) * ni, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return cuda_status(e);
  bool nonfinite = false, noconv = false;
  for (int v : hdone) {
    nonfinite = nonfinite || v == 2;
    noconv = noconv || v == 0;
  }
  return nonfinite ? EHL_ENONFINITE : (noconv ? EHL_ENOCONV : EHL_OK);
}

static ehl_status ehl_residual_impl(ehl_ctx* ctx, const double* P, const double* H0, const double* rough, double* R,
                                   double* H, double* comp_res) {
  if (!ctx || !P || !H0 || !R) return EHL_EINVAL;
  if (ctx->pt) return pt_residual_api(ctx, P, H0, rough, R, H, comp_res);
  cudaError_t e = fork(ctx);
  for (Bucket* b : ctx->buckets) {
    LineCtx* c = &b->c;
    if (e == cudaSuccess) e = bucket_state(ctx, b, P, H0, rough);
    if (e == cudaSuccess) e = put_rows(ctx, b, (const double*)c->R, c->N, R, ctx->nx_max);
    if (e == cudaSuccess && H) e = put_rows(ctx, b, (const double*)c->H, c->N, H, ctx->nx_max);
    if (e == cudaSuccess && comp_res) e = put_comp(ctx, b, comp_res);
  }
  if (e == cudaSuccess) e = join(ctx);
  return cuda_status(e);
}

static ehl_status ehl_jacobian_band_impl(ehl_ctx* ctx, const double* P, const double* H0, const double* rough,
                                        int kind, double* band, uint8_t* active) {
  if (!ctx || !P || !H0 || !band || !active || kind < 0 || kind > 2) return EHL_EINVAL;
  if (ctx->pt) {
    if (kind == 0) return EHL_EINVAL;
    PtCtx* c = ctx->pt;
    cudaError_t e = pt_state(c, P, H0, rough, nullptr);
    if (kind == 1) {
      if (e == cudaSuccess) e = pt_jac_band(c, P, band, active, nullptr, nullptr, nullptr);
    } else {
      // the y-line bands; the x-line bands (into the context's scratch) fix the row scale and the
      // identity rows
      if (e == cudaSuccess) e = pt_jac_band(c, P, c->band, active, nullptr, c->dg, nullptr);
      if (e == cudaSuccess) e = pt_jac_yband(c, P, active, c->dg, band, 0, nullptr);
    }
    return cuda_status(e);
  }
  if (kind == 2) return EHL_EINVAL;
  const int bw = 2 * ctx->beta + 1, nmax = ctx->nx_max - 2;
  cudaError_t e = fork(ctx);
  for (Bucket* b : ctx->buckets) {
    LineCtx* c = &b->c;
    if (e == cudaSuccess) e = bucket_state(ctx, b, P, H0, rough);
    const double* Pb = ctx->direct ? P : b->Pb;
    double* bo = ctx->direct ? band : c->band;
    uint8_t* ao = ctx->direct ? active : c->act;
    if (e == cudaSuccess) e = line_jac_band(c, Pb, kind, bo, ao, nullptr, nullptr, nullptr);
    if (!ctx->direct) {
      if (e == cudaSuccess) e = rows(c->st, (const double*)c->band, c->n * bw, band, nmax * bw, b->d_idx, c->n_inst,
                                     c->n * bw, true);
      if (e == cudaSuccess) e = rows(c->st, (const uint8_t*)c->act, c->n, active, nmax, b->d_idx, c->n_inst, c->n,
                                     true);
    }
  }
  if (e == cudaSuccess) e = join(ctx);
  return cuda_status(e);
}

static ehl_status ehl_jacobian_apply_impl(ehl_ctx* ctx, const double* P, const double* H0, const double* rough,
                                         const double* v, const double* v_h0, double* out) {
  if (!ctx || !P || !H0 || !v || !v_h0 || !out) return EHL_EINVAL;
  if (ctx->pt) return cuda_status(pt_jacobian_apply(ctx->pt, P, H0, rough, v, v_h0, out));
  cudaError_t e = fork(ctx);
  for (Bucket* b : ctx->buckets) {
    LineCtx* c = &b->c;
    const double* Pb = gin(ctx, b, P, ctx->nx_max, c->N, b->Pb, e);
    const double* H0b = gin(ctx, b, H0, 1, 1, b->H0b, e);
    const double* rb = gin(ctx, b, rough, ctx->nx_max, c->N, b->rb, e);
    const double* vb = gin(ctx, b, v, ctx->nx_max, c->N, b->vb, e);
    const double* vhb = gin(ctx, b, v_h0, 1, 1, b->vhb, e);
    double* ob = ctx->direct ? out : b->ob;
    if (e == cudaSuccess) e = line_jacobian_apply(c, Pb, H0b, rb, vb, vhb, ob);
    if (e == cudaSuccess && !ctx->direct) e = put_rows(ctx, b, (const double*)b->ob, c->N, out, ctx->nx_max);
  }
  if (e == cudaSuccess) e = join(ctx);
  return cuda_status(e);
}

// The final residual at the returned iterate and the done flags in hdone.
static cudaError_t iterate_end(LineCtx* c, const double* rough, std::vector<int>& hdone) {
  cudaError_t e = line_state(c, c->Pw, c->H0w, rough, nullptr, nullptr);
  if (e == cudaSuccess) e = line_finalize(c, nullptr, nullptr);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hdone.data(), c->done, sizeof(int) * c->n_inst, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  return e;
}

// Graph mode: the Newton step (without host checks, with the first kGraphTrials
// line-search trials) is captured once per (P, H0, rough) and replayed; after each
// replay one host check reads the done flags, and instances still searching get
// the remaining trials eagerly.
static cudaError_t iterate_graph(LineCtx* c, const double* rough, std::vector<int>& hdone) {
  cudaError_t e = cudaSuccess;
  if (!c->graph || c->g_P != c->Pw || c->g_H0 != c->H0w || c->g_rough != rough) {
    if (c->graph) {
      cudaGraphExecDestroy(c->graph);
      c->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    const unsigned long long l0 = thread_launches();
    e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    c->capturing = true;
    const cudaError_t es = line_nk_step(c, c->Pw, c->H0w, rough);
    c->capturing = false;
    e = cudaStreamEndCapture(c->st, &g);
    c->graph_launches = (long long)(thread_launches() - l0);
    add_launches(-c->graph_launches);  // captured, not run
    if (es != cudaSuccess) e = es;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      c->graph = nullptr;
      return e;
    }
    c->g_P = c->Pw;
    c->g_H0 = c->H0w;
    c->g_rough = rough;
  }
  for (int it = 0; it < c->max_iter && e == cudaSuccess; ++it) {
    e = cudaGraphLaunch(c->graph, c->st);
    if (e != cudaSuccess) break;
    add_launches(c->graph_launches);
    e = line_nk_finish(c, c->Pw, c->H0w, rough, kGraphTrials);
    if (e != cudaSuccess) break;
    e = cudaMemcpyAsync(hdone.data(), c->done, sizeof(int) * c->n_inst, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    bool all = true;
    for (int v : hdone) all = all && (v != 0);
    if (all) break;
  }
  if (e == cudaSuccess) e = iterate_end(c, rough, hdone);
  return e;
}

// Graph mode 2: the whole iteration of this grid as one graph with device-side loops (method 1:
// Newton steps, GMRES, line search; method 0: the paper's iteration), captured once per
// (P, H0, rough) and launched once per solve; the host reads the done flags and the loop totals
// afterwards.
static cudaError_t iterate_device_graph(LineCtx* c, const double* rough, std::vector<int>& hdone) {
  cudaError_t e = cudaSuccess;
  if (!c->gs1) {
    e = cudaStreamCreateWithFlags(&c->gs1, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->gs2, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
  }
  if (!c->graph || c->g_P != c->Pw || c->g_H0 != c->H0w || c->g_rough != rough) {
    if (c->graph) {
      cudaGraphExecDestroy(c->graph);
      c->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    const unsigned long long l0 = thread_launches();
    e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    SolveGraphCounts n;
    const cudaError_t es = c->method == 0 ? line_paper_capture_solve(c, c->Pw, c->H0w, rough, c->gs1, n)
                                          : line_nk_capture_solve(c, c->Pw, c->H0w, rough, c->gs1, c->gs2, n);
    e = cudaStreamEndCapture(c->st, &g);
    add_launches(-(long long)(thread_launches() - l0));  // captured, not run
    if (es != cudaSuccess) e = es;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      c->graph = nullptr;
      cudaGetLastError();
      return e;
    }
    c->gcounts = n;
    c->g_P = c->Pw;
    c->g_H0 = c->H0w;
    c->g_rough = rough;
  }
  int loops[8] = {0};
  e = cudaGraphLaunch(c->graph, c->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(loops, c->method == 0 ? c->loop0 : line_nk_loop_counters(c), sizeof(loops),
                        cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hdone.data(), c->done, sizeof(int) * c->n_inst, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e == cudaSuccess) add_launches(line_nk_graph_launches(c->gcounts, loops));
  return e;
}

// Outer iterations of one LineCtx from (c->Pw, c->H0w) until every instance is
// done or max_iter; ends with the residual at the returned iterate and the
// done flags in hdone.
static cudaError_t iterate(LineCtx* c, const double* rough, std::vector<int>& hdone) {
  c->state_current = false;
  cudaError_t e = cudaMemsetAsync(c->done, 0, sizeof(int) * c->n_inst, c->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->iters, 0, sizeof(int) * c->n_inst, c->st);
  // bytes 0x7f: best = 1.4e306 (no residual seen yet)
  if (e == cudaSuccess) e = cudaMemsetAsync(c->best, 0x7f, sizeof(double) * c->n_inst, c->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->stall, 0, sizeof(int) * c->n_inst, c->st);
  hdone.assign(c->n_inst, 0);
  if (e == cudaSuccess && c->graph_mode == 2) return iterate_device_graph(c, rough, hdone);
  if (e == cudaSuccess && c->method == 1 && c->use_graph) return iterate_graph(c, rough, hdone);
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
  if (e == cudaSuccess) e = line_state(c, c->Pw, c->H0w, rough, nullptr, nullptr);
  if (e == cudaSuccess) e = line_finalize(c, nullptr, nullptr);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hdone.data(), c->done, sizeof(int) * c->n_inst, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  return e;
}

// The solve of one bucket on its stream; the result stays in c->Pw, c->H0w.
// From the Hertzian start with coarse grids: nested iteration, each grid
// started from the prolonged solution of the one below.
static cudaError_t solve_bucket(ehl_ctx* ctx, Bucket* b, const double* P, const double* H0, const double* rough,
                                int init, std::vector<int>& hdone) {
  LineCtx* c = &b->c;
  const size_t NN = (size_t)c->n_inst * c->N;
  cudaError_t e = cudaSuccess;
  const double* rb = gin(ctx, b, rough, ctx->nx_max, c->N, b->rb, e);
  if (init == 1) {
    const double* Pb = gin(ctx, b, P, ctx->nx_max, c->N, b->Pb, e);
    const double* H0b = gin(ctx, b, H0, 1, 1, b->H0b, e);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->Pw, Pb, sizeof(double) * NN, cudaMemcpyDeviceToDevice, c->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->H0w, H0b, sizeof(double) * c->n_inst, cudaMemcpyDeviceToDevice, c->st);
  } else {
    LineCtx* prev = nullptr;
    std::vector<int> hd;
    for (size_t l = 0; l < b->lv.size() && e == cudaSuccess; ++l) {
      LineCtx* cl = b->lv[l];
      const double* rl = nullptr;
      if (rb) {
        e = line_inject(rb, c->N, b->lrough[l], cl->N, cl->n_inst, cl->st);
        rl = b->lrough[l];
      }
      if (e == cudaSuccess) e = line_start(cl, cl->Pw, cl->H0w, rl);
      if (e == cudaSuccess && prev)
        e = line_prolong(prev->Pw, prev->H0w, prev->done, prev->N, cl->Pw, cl->H0w, cl->n_inst, cl->st);
      if (e == cudaSuccess) e = iterate(cl, rl, hd);
      prev = cl;
    }
    if (e == cudaSuccess) e = line_start(c, c->Pw, c->H0w, rb);
    if (e == cudaSuccess && prev)
      e = line_prolong(prev->Pw, prev->H0w, prev->done, prev->N, c->Pw, c->H0w, c->n_inst, c->st);
  }
  if (e == cudaSuccess) e = iterate(c, rb, hdone);
  return e;
}

static ehl_status ehl_solve_impl(ehl_ctx* ctx, double* P, double* H0, const double* rough, int init, int* iters,
                                double* final_res) {
  if (!ctx || !P || !H0 || (init != 0 && init != 1)) return EHL_EINVAL;
  if (ctx->pt) return pt_solve_api(ctx, P, H0, rough, init, iters, final_res);
  cudaError_t e = fork(ctx);
  if (e != cudaSuccess) return cuda_status(e);
  const size_t nb = ctx->buckets.size();
  std::vector<cudaError_t> errs(nb, cudaSuccess);
  std::vector<std::vector<int>> dones(nb);
  if (nb == 1) {
    errs[0] = solve_bucket(ctx, ctx->buckets[0], P, H0, rough, init, dones[0]);
  } else {
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<std::thread> th;
    th.reserve(nb);
    bool spawned = true;
    for (size_t q = 0; q < nb && spawned; ++q) {
      try {
        th.emplace_back([&, q, dev]() {
          cudaSetDevice(dev);
          try {
            errs[q] = solve_bucket(ctx, ctx->buckets[q], P, H0, rough, init, dones[q]);
          } catch (...) {  // a host allocation failed inside the bucket's solve
            errs[q] = cudaErrorMemoryAllocation;
          }
        });
      } catch (...) {  // no thread for this bucket: the started ones finish, then the call fails
        spawned = false;
      }
    }
    for (auto& t : th) t.join();
    if (!spawned) {
      join(ctx);
      return EHL_ENOMEM;
    }
  }
  for (size_t q = 0; q < nb; ++q) {
    Bucket* b = ctx->buckets[q];
    LineCtx* c = &b->c;
    if (errs[q] != cudaSuccess) e = errs[q];
    if (e != cudaSuccess) break;
    e = put_rows(ctx, b, (const double*)c->Pw, c->N, P, ctx->nx_max);
    if (e == cudaSuccess) e = put_rows(ctx, b, (const double*)c->H0w, 1, H0, 1);
    if (e == cudaSuccess && iters) e = put_rows(ctx, b, (const int*)c->iters, 1, iters, 1);
    if (e == cudaSuccess && final_res) e = put_comp(ctx, b, final_res);
  }
  if (e == cudaSuccess) e = join(ctx);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
  if (e != cudaSuccess) return cuda_status(e);
  bool nonfinite = false, noconv = false;
  for (auto& hd : dones)
    for (int v : hd) {
      nonfinite = nonfinite || v == 2;
      noconv = noconv || v == 0;
    }
  return nonfinite ? EHL_ENONFINITE : (noconv ? EHL_ENOCONV : EHL_OK);
}

static ehl_status ehl_adjoint_impl(ehl_ctx* ctx, const double* P, const double* H0, const double* rough,
                                  const double* gP, const double* gH, const double* gH0, double* grad_rough,
                                  double* grad_ML, double* relres, double tol, int max_cycles) {
  if (!ctx || !P || !H0 || !(tol > 0.0) || max_cycles < 1 || max_cycles > 1000) return EHL_EINVAL;
  if (ctx->pt) {
    PtCtx* c = ctx->pt;
    std::vector<double> h(c->n_inst);
    double* rel = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&rel, sizeof(double) * c->n_inst, c->st);
    if (e == cudaSuccess)
      e = pt_adjoint(c, P, H0, rough, gP, gH, gH0, grad_rough, grad_ML, rel, tol, max_cycles);
    if (e == cudaSuccess && relres)
      e = cudaMemcpyAsync(relres, rel, sizeof(double) * c->n_inst, cudaMemcpyDeviceToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), rel, sizeof(double) * c->n_inst, cudaMemcpyDeviceToHost, c->st);
    if (rel) cudaFreeAsync(rel, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_status(e);
    bool nonfinite = false, noconv = false;
    for (double v : h) {
      nonfinite = nonfinite || !(v == v);
      noconv = noconv || v > tol;
    }
    return nonfinite ? EHL_ENONFINITE : (noconv ? EHL_ENOCONV : EHL_OK);
  }
  cudaError_t e = fork(ctx);
  for (Bucket* b : ctx->buckets) {
    LineCtx* c = &b->c;
    const double* Pb = gin(ctx, b, P, ctx->nx_max, c->N, b->Pb, e);
    const double* H0b = gin(ctx, b, H0, 1, 1, b->H0b, e);
    const double* rb = gin(ctx, b, rough, ctx->nx_max, c->N, b->rb, e);
    const double* gPb = gin(ctx, b, gP, ctx->nx_max, c->N, b->gPb, e);
    const double* gHb = gin(ctx, b, gH, ctx->nx_max, c->N, b->gHb, e);
    const double* gH0b = gin(ctx, b, gH0, 1, 1, b->gH0b, e);
    double* grb = grad_rough ? (ctx->direct ? grad_rough : b->grb) : nullptr;
    double* gml = grad_ML ? (ctx->direct ? grad_ML : b->gmlb) : nullptr;
    int cyc = 0;
    if (e == cudaSuccess)
      e = line_adjoint(c, Pb, H0b, rb, gPb, gHb, gH0b, grb, gml, b->relw, tol, max_cycles, &cyc);
    if (!ctx->direct) {
      if (e == cudaSuccess && grad_rough) e = put_rows(ctx, b, (const double*)b->grb, c->N, grad_rough, ctx->nx_max);
      if (e == cudaSuccess && grad_ML) e = put_rows(ctx, b, (const double*)b->gmlb, 2, grad_ML, 2);
    }
    if (e == cudaSuccess && relres) e = put_rows(ctx, b, (const double*)b->relw, 1, relres, 1);
  }
  if (e == cudaSuccess) e = join(ctx);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
  if (e != cudaSuccess) return cuda_status(e);
  bool nonfinite = false, noconv = false;
  for (Bucket* b : ctx->buckets) {
    std::vector<double> h(b->c.n_inst);
    if (cudaMemcpy(h.data(), b->relw, sizeof(double) * h.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
      return cuda_status(cudaGetLastError());
    for (double v : h) {
      nonfinite = nonfinite || !(v == v);
      noconv = noconv || v > tol;
    }
  }
  return nonfinite ? EHL_ENONFINITE : (noconv ? EHL_ENOCONV : EHL_OK);
}

// ---------------------------------------------------------------- C ABI
// No C++ exception leaves an entry point: a failed host allocation (or host
// thread) is reported as EHL_ENOMEM.
#define EHL_NOTHROW(call)           \
  try {                             \
    return call;                    \
  } catch (...) {                   \
    return EHL_ENOMEM;              \
  }

extern "C" ehl_status ehl_create(const ehl_params* p, int n_inst, const ehl_params* per_inst, void* stream,
                                 ehl_ctx** out) {
  EHL_NOTHROW(ehl_create_impl(p, n_inst, per_inst, stream, out))
}

extern "C" ehl_status ehl_residual(ehl_ctx* ctx, const double* P, const double* H0, const double* rough, double* R,
                                   double* H, double* comp_res) {
  EHL_NOTHROW(ehl_residual_impl(ctx, P, H0, rough, R, H, comp_res))
}

extern "C" ehl_status ehl_jacobian_band(ehl_ctx* ctx, const double* P, const double* H0, const double* rough,
                                        int kind, double* band, uint8_t* active) {
  EHL_NOTHROW(ehl_jacobian_band_impl(ctx, P, H0, rough, kind, band, active))
}

extern "C" ehl_status ehl_jacobian_apply(ehl_ctx* ctx, const double* P, const double* H0, const double* rough,
                                         const double* v, const double* v_h0, double* out) {
  EHL_NOTHROW(ehl_jacobian_apply_impl(ctx, P, H0, rough, v, v_h0, out))
}

extern "C" ehl_status ehl_solve(ehl_ctx* ctx, double* P, double* H0, const double* rough, int init, int* iters,
                                double* final_res) {
  EHL_NOTHROW(ehl_solve_impl(ctx, P, H0, rough, init, iters, final_res))
}

extern "C" ehl_status ehl_adjoint(ehl_ctx* ctx, const double* P, const double* H0, const double* rough,
                                  const double* gP, const double* gH, const double* gH0, double* grad_rough,
                                  double* grad_ML, double* relres, double tol, int max_cycles) {
  EHL_NOTHROW(ehl_adjoint_impl(ctx, P, H0, rough, gP, gH, gH0, grad_rough, grad_ML, relres, tol, max_cycles))
}

#undef EHL_NOTHROW
