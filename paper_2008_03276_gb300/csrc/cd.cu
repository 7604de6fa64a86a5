// cd.cu -- the linear convection-diffusion workload of the AQIF line splittings
// (Sec. 3.1, Examples 1 and 2; Sec. 6): residual of van Leer's kappa-scheme and the
// x-line relaxations Ls0 / Ls1 with every line system solved by PAQIF.
//
//   L u = (a u)_x + (b u)_y - eps (u_xx + u_yy) = f on an n x n grid, Dirichlet data in u.
//   Convective face value (Eq. eqn41):
//     F_{k+1/2} = u_k + (1 - kappa)/4 (u_k - u_{k-1}) + (1 + kappa)/4 (u_{k+1} - u_k),
//   with the node before the inflow boundary taken as the linear extrapolation
//   2 u_0 - u_1.  Line operator L^0 of the splittings (Eqs. eqn48, eqn49): the
//   upwind difference c (u_i - u_{i-1}) a / h, c = (2 - kappa)/2 (Ls1) or
//   (2 - kappa)/2 + (1 - kappa)/4 (Ls0), and the diffusion's x part and diagonal.
//   A sweep solves L^0 sigma = f - L u for the x-lines (in increasing y, each line
//   from the iterate its predecessors left, or all lines from one iterate) and
//   adds omega sigma.
//
// GB300 mapping: the residual is a streaming 5-point (plus two upwind nodes) stencil,
// one thread per node, float64, rows of x contiguous; the line matrix is the same
// for every line, so its PAQIF factorization is computed once per call and every
// line's change is a PAQIF resolve (Sec. 2.2.2 sweeps with the stored factors).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ehl_internal.h"

namespace ehl {

namespace {

constexpr int kCdBlock = 256;

struct CdCoef {
  int n;
  double h, a, b, eps, kappa;
  double c;  // upwind coefficient of L^0
};

// F_{k+1/2} along one direction from the values at k-1, k, k+1 (k-1 < 0: extrapolated)
__device__ __forceinline__ double cd_face(double vm, double v0, double vp, double kappa) {
  return v0 + 0.25 * (1.0 - kappa) * (v0 - vm) + 0.25 * (1.0 + kappa) * (vp - v0);
}

// f - L u at interior node (i, j) of one instance (u, f: [n][n], x fastest)
__device__ __forceinline__ double cd_node_residual(const CdCoef& q, const double* __restrict__ u,
                                                   const double* __restrict__ f, int i, int j) {
  const int n = q.n;
  const double* row = u + (size_t)j * n;
  const double uc = row[i], ue = row[i + 1], uw = row[i - 1];
  const double uww = (i >= 2) ? row[i - 2] : 2.0 * uw - uc;  // i = 1: ghost 2 u_0 - u_1
  const double un = u[(size_t)(j + 1) * n + i], us = u[(size_t)(j - 1) * n + i];
  double conv = q.a * (cd_face(uw, uc, ue, q.kappa) - cd_face(uww, uw, uc, q.kappa)) / q.h;
  if (q.b != 0.0) {
    const double uss = (j >= 2) ? u[(size_t)(j - 2) * n + i] : 2.0 * us - uc;
    conv += q.b * (cd_face(us, uc, un, q.kappa) - cd_face(uss, us, uc, q.kappa)) / q.h;
  }
  const double lap = (ue + uw + un + us - 4.0 * uc) / (q.h * q.h);
  return f[(size_t)j * n + i] - conv + q.eps * lap;
}

// order-preserving bits of a non-negative double (NaN above +Inf)
__device__ __forceinline__ unsigned long long cd_bits(double x) { return (unsigned long long)__double_as_longlong(x); }

__device__ __forceinline__ void cd_block_max(double v, unsigned long long* out) {
  __shared__ double red[kCdBlock / 32];
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = (w > v || w != w) ? w : v;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_xor_sync(0xffffffffu, v, o);
      v = (w > v || w != w) ? w : v;
    }
    if (lane == 0 && v > 0.0) atomicMax(out, cd_bits(v));
    if (lane == 0 && v != v) atomicMax(out, cd_bits(__longlong_as_double(0x7ff8000000000000ll)));
  }
}

// r = f - L u on interior nodes (0 on the boundary), rmax[z] = max |r| (bits, pre-zeroed)
__global__ void __launch_bounds__(kCdBlock) k_cd_residual(CdCoef q, const double* __restrict__ u,
                                                          const double* __restrict__ f, double* __restrict__ r,
                                                          unsigned long long* __restrict__ rmax) {
  const int z = blockIdx.y;
  const int n = q.n;
  const size_t nn = (size_t)n * n;
  const double* uz = u + z * nn;
  const double* fz = f + z * nn;
  double m = 0.0;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)(t / n);
    double v = 0.0;
    if (i > 0 && i < n - 1 && j > 0 && j < n - 1) {
      v = cd_node_residual(q, uz, fz, i, j);
      const double av = fabs(v);
      m = (av > m || av != av) ? av : m;
    }
    if (r) r[z * nn + t] = v;
  }
  if (rmax) cd_block_max(m, rmax + z);
}

// the line matrix L^0 (n - 2 rows, half-band 1) for n_sys systems
__global__ void k_cd_band(CdCoef q, double* __restrict__ band, size_t rows) {
  const double c = q.c * q.a / q.h, d = q.eps / (q.h * q.h);
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < rows; t += (size_t)gridDim.x * blockDim.x) {
    band[3 * t + 0] = -c - d;
    band[3 * t + 1] = c + 4.0 * d;
    band[3 * t + 2] = -d;
  }
}

// right-hand sides f - L u of the x-lines j0 .. j0 + nl - 1 of every instance:
// rhs[(z * nl + l)][i - 1]
__global__ void k_cd_rhs(CdCoef q, const double* __restrict__ u, const double* __restrict__ f, int j0, int nl,
                         double* __restrict__ rhs) {
  const int z = blockIdx.y;
  const int n = q.n, m = n - 2;
  const size_t nn = (size_t)n * n;
  const size_t total = (size_t)nl * m;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int l = (int)(t / m), i = (int)(t % m) + 1;
    rhs[(size_t)z * total + t] = cd_node_residual(q, u + z * nn, f + z * nn, i, j0 + l);
  }
}

// u += omega sigma on the same lines
__global__ void k_cd_update(int n, const double* __restrict__ sigma, int j0, int nl, double omega,
                            double* __restrict__ u) {
  const int z = blockIdx.y;
  const int m = n - 2;
  const size_t total = (size_t)nl * m;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int l = (int)(t / m), i = (int)(t % m) + 1;
    u[(size_t)z * n * n + (size_t)(j0 + l) * n + i] += omega * sigma[(size_t)z * total + t];
  }
}

__global__ void k_cd_copy_max(const unsigned long long* __restrict__ bits, double* __restrict__ out, int n_inst) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z < n_inst) out[z] = __longlong_as_double((long long)bits[z]);
}

// per instance: the first nonzero EHL_INFO_* flag of its line systems (0 if none)
__global__ void k_cd_info(const int* __restrict__ pq_info, int nl, int n_inst, int* __restrict__ info) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= n_inst) return;
  int f = 0;
  for (int l = 0; l < nl && f == 0; ++l) f = pq_info[(size_t)z * nl + l];
  info[z] = f;
}

int cd_grid(size_t work) {
  size_t b = (work + kCdBlock - 1) / kCdBlock;
  const size_t cap = (size_t)kSmCount * 8;
  if (b > cap) b = cap;
  return b < 1 ? 1 : (int)b;
}

bool cd_ok(const ehl_cd_params* p, int n_inst) {
  return p && n_inst >= 1 && n_inst <= 65535 && p->n >= 5 && p->n <= 16385 && p->hi > p->lo && p->a > 0.0 &&
         p->b >= 0.0 && p->eps >= 0.0 && p->kappa >= -1.0 && p->kappa <= 1.0 && (p->splitting == 0 || p->splitting == 1) &&
         (p->order == 0 || p->order == 1) && p->omega > 0.0 && isfinite(p->a) && isfinite(p->b) && isfinite(p->eps);
}

CdCoef cd_coef(const ehl_cd_params* p) {
  CdCoef q;
  q.n = p->n;
  q.h = (p->hi - p->lo) / (p->n - 1);
  q.a = p->a;
  q.b = p->b;
  q.eps = p->eps;
  q.kappa = p->kappa;
  q.c = (2.0 - p->kappa) / 2.0 + (p->splitting == 0 ? (1.0 - p->kappa) / 4.0 : 0.0);
  return q;
}

// workspace layout of ehl_cd_relax
struct CdWs {
  size_t band, rhs, sigma, stack, fstore, info, bits, total;
};

bool cd_ws(const ehl_cd_params* p, int n_inst, CdWs& w) {
  const int m = p->n - 2;
  const int lines = (p->order == 1) ? m : 1;
  const size_t n_sys = (size_t)n_inst * lines;
  if (n_sys > (size_t)(1 << 24)) return false;
  const size_t st = paqif_stack_bytes((int)n_sys, m, 1);
  const size_t fs = paqif_factor_store_bytes((int)n_sys, m, 1);
  if (!st || !fs) return false;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, kWorkspaceAlign);
    return at;
  };
  w.band = take(n_sys * m * 3 * sizeof(double));
  w.rhs = take(n_sys * m * sizeof(double));
  w.sigma = take(n_sys * m * sizeof(double));
  w.stack = take(st);
  w.fstore = take(fs);
  w.info = take(n_sys * sizeof(int));
  w.bits = take((size_t)n_inst * sizeof(unsigned long long));
  w.total = o;
  return true;
}

}  // namespace

}  // namespace ehl

using namespace ehl;

extern "C" ehl_status ehl_cd_residual(const ehl_cd_params* p, int n_inst, const double* u, const double* f, double* r,
                                      double* rmax, void* stream) {
  if (!cd_ok(p, n_inst) || !u || !f) return EHL_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const CdCoef q = cd_coef(p);
  unsigned long long* bits = nullptr;
  cudaError_t e = cudaSuccess;
  if (rmax) {
    // the maximum is accumulated as integer bits in the caller's array, then converted in place
    bits = reinterpret_cast<unsigned long long*>(rmax);
    e = cudaMemsetAsync(bits, 0, (size_t)n_inst * sizeof(double), st);
  }
  if (e == cudaSuccess) {
    const size_t nn = (size_t)p->n * p->n;
    k_cd_residual<<<dim3(cd_grid(nn), n_inst), kCdBlock, 0, st>>>(q, u, f, r, bits);
    note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && rmax) {
    k_cd_copy_max<<<(n_inst + 127) / 128, 128, 0, st>>>(bits, rmax, n_inst);
    note_launch();
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return EHL_ECUDA;
  }
  return EHL_OK;
}

extern "C" ehl_status ehl_cd_workspace_size(const ehl_cd_params* p, int n_inst, size_t* bytes) {
  CdWs w;
  if (!bytes || !cd_ok(p, n_inst) || !cd_ws(p, n_inst, w)) return EHL_EINVAL;
  *bytes = w.total;
  return EHL_OK;
}

extern "C" ehl_status ehl_cd_relax(const ehl_cd_params* p, int n_inst, double* u, const double* f, int sweeps,
                                   double* rmax_hist, int* info, void* workspace, size_t workspace_bytes,
                                   void* stream) {
  CdWs w;
  if (!cd_ok(p, n_inst) || !u || !f || sweeps < 0 || !cd_ws(p, n_inst, w)) return EHL_EINVAL;
  if ((const void*)u == (const void*)f) return EHL_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  bool owned = false;
  if (workspace) {
    if (workspace_bytes < w.total || ((uintptr_t)workspace % kWorkspaceAlign) != 0) return EHL_EINVAL;
  } else {
    if (cudaMallocAsync(&workspace, w.total, st) != cudaSuccess) {
      cudaGetLastError();
      return EHL_ENOMEM;
    }
    owned = true;
  }
  unsigned char* ws = (unsigned char*)workspace;
  double* band = (double*)(ws + w.band);
  double* rhs = (double*)(ws + w.rhs);
  double* sigma = (double*)(ws + w.sigma);
  int* pq_info = (int*)(ws + w.info);
  unsigned long long* bits = (unsigned long long*)(ws + w.bits);
  const CdCoef q = cd_coef(p);
  const int n = p->n, m = n - 2;
  const bool all_lines = p->order == 1;
  const int nl = all_lines ? m : 1;  // lines per solve
  const int n_sys = n_inst * nl;
  PaqifLaunch L;
  L.n_sys = n_sys;
  L.n = m;
  L.beta = 1;
  L.mode = 0;
  L.band = band;
  L.rhs = rhs;
  L.act = nullptr;
  L.stack = ws + w.stack;
  L.x = sigma;
  L.iters = nullptr;
  L.info = pq_info;
  void* fstore = ws + w.fstore;
  cudaError_t e = cudaSuccess;
  if (info && sweeps == 0) e = cudaMemsetAsync(info, 0, (size_t)n_inst * sizeof(int), st);
  if (e == cudaSuccess) {
    k_cd_band<<<cd_grid((size_t)n_sys * m), kCdBlock, 0, st>>>(q, band, (size_t)n_sys * m);
    note_launch();
    e = cudaGetLastError();
  }
  bool factored = false;
  for (int s = 0; s < sweeps && e == cudaSuccess; ++s) {
    for (int j0 = 1; j0 <= m && e == cudaSuccess; j0 += nl) {
      k_cd_rhs<<<dim3(cd_grid((size_t)nl * m), n_inst), kCdBlock, 0, st>>>(q, u, f, j0, nl, rhs);
      note_launch();
      e = cudaGetLastError();
      if (e != cudaSuccess) break;
      e = factored ? launch_paqif_resolve(L, fstore, st) : launch_paqif_factor(L, fstore, st);
      factored = true;
      if (e != cudaSuccess) break;
      k_cd_update<<<dim3(cd_grid((size_t)nl * m), n_inst), kCdBlock, 0, st>>>(n, sigma, j0, nl, p->omega, u);
      note_launch();
      e = cudaGetLastError();
    }
    if (e == cudaSuccess && rmax_hist) {
      e = cudaMemsetAsync(bits, 0, (size_t)n_inst * sizeof(unsigned long long), st);
      if (e != cudaSuccess) break;
      k_cd_residual<<<dim3(cd_grid((size_t)n * n), n_inst), kCdBlock, 0, st>>>(q, u, f, nullptr, bits);
      note_launch();
      k_cd_copy_max<<<(n_inst + 127) / 128, 128, 0, st>>>(bits, rmax_hist + (size_t)s * n_inst, n_inst);
      note_launch();
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess && info && factored) {
    k_cd_info<<<(n_inst + 127) / 128, 128, 0, st>>>(pq_info, nl, n_inst, info);
    note_launch();
    e = cudaGetLastError();
  }
  if (owned) cudaFreeAsync(workspace, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return EHL_ECUDA;
  }
  return EHL_OK;
}
