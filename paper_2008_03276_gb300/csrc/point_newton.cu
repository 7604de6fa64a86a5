// point_newton.cu -- Newton-Krylov step of the point-contact solve.
//
// Phi_r = P_r (rows with P <= R/d) or R_r/d_r (the others), d = |dR_r/dP_r| floored
// at a tenth of the largest x-band entry of the row,
// Phi_n = h^2 sum P - 2 pi/3.  Each step: the exact x-line bands, scaled by
// 1/d; PAQIF factorization of every grid row's band (ny-2 systems per
// instance) solving for the border column dR/dH0; GMRES with classical
// Gram-Schmidt applied twice, right-preconditioned by the bordered x-line
// solve; the exact Jacobian product from one 2-D deformation of the Krylov
// vector; backtracking on ||Phi||_2 (projected trials first, unprojected
// after 2^-10, as in line contact).  Vector kernels use many blocks per
// instance, each thread kPtVPT elements; per-instance scalars are finished by
// one-block kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <vector>

#include "ehl_internal.h"
#include "point.h"
#include "graph_loop.h"

namespace ehl {

constexpr int kNB = 256;   // threads of the vector kernels
constexpr int kNV = 2;     // elements per thread (a 257^2 grid spreads over 128 blocks)

struct PtView {  // device pointers the vector kernels need
  const PointInst* inst;
  int nx, ny, NN, n, n1, m, nvb, beta;
  const int* done;
  const int* skip;
  double *V, *Z, *Hh, *cs, *sn, *g, *w, *dots, *hcol, *delta, *zH, *rhs, *sigma, *band, *jh, *dg, *R, *red;
  double *phinorm, *den, *rtol, *beta0, *tstep, *zh0, *H0t, *Pt, *znode;
  const uint8_t* act;
  int *gm_k, *gm_conv, *lsdone, *lsphase, *acc;
  // y-line stage (yline = 1): rhs and solution of the y-line systems (column-major interior
  // order r_y = (i-1)(ny-2) + (j-1)), their bordered correction zHy (row-major) and den_y, xi_y
  double *rhs_y, *sig_y, *zHy, *deny, *xiy;
  // device-driven solve: the Krylov index is read from here when not null
  const int* jd;
  // per node, fixed for a Newton step: drho H, 3 eps / H, eps (drho / rho - deta), 1 / d (interior)
  double* jc;
};

// the block's total of v, to every thread: warp shuffles, then one value per warp in shared
// memory (two barriers; the leading one lets a previous call's readers finish)
__device__ __forceinline__ double nk_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double nk_block_sum(double v, double* sh) {
  v = nk_warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < kNB / 32; ++w) t += sh[w];
  return t;
}

__device__ __forceinline__ int nk_node(int r, int nx) { return (r / (nx - 2) + 1) * nx + (r % (nx - 2)) + 1; }

// element k of this thread's share of [0, len)
#define NK_FOR(r, len)                                                         \
  for (int _k = 0, r = blockIdx.x * (kNB * kNV) + threadIdx.x; _k < kNV; ++_k, \
           r = blockIdx.x * (kNB * kNV) + threadIdx.x + _k * kNB)              \
    if (r < (len))

__global__ void k_pn_skip(const int* __restrict__ done, const int* __restrict__ other, int* __restrict__ skip, int ni) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z < ni) skip[z] = (done[z] != 0) || (other && other[z] != 0);
}

// scale equation rows by 1/d; rhs = (dR/dH0)/d; Phi into V_0 (unnormalised); partial |Phi|^2
__global__ void __launch_bounds__(kNB) k_pn_setup(PtView v, const double* __restrict__ P) {
  const int z = blockIdx.y;
  if (v.done[z]) return;
  __shared__ double sh[kNB];
  const int w = 2 * v.beta + 1;
  double ss = 0.0;
  double* V0 = v.V + (size_t)z * (v.m + 1) * v.n1;
  NK_FOR(r, v.n) {
    const size_t o = (size_t)z * v.n + r;
    const size_t node = (size_t)z * v.NN + nk_node(r, v.nx);
    double ph;
    if (v.act[o]) {
      ph = P[node];
      v.rhs[o] = 0.0;
    } else {
      const double d = v.dg[o];
      double* row = v.band + o * w;
      const double rd = 1.0 / d;  // one float64 division per row
      for (int t = 0; t < w; ++t) row[t] *= rd;
      v.rhs[o] = v.jh[o] / d;
      ph = v.R[node] / d;
    }
    V0[r] = ph;
    ss += ph * ph;
  }
  ss = nk_block_sum(ss, sh);
  if (threadIdx.x == 0) v.dots[((size_t)z * v.nvb + blockIdx.x) * (v.m + 2)] = ss;
}

// |Phi|, the GMRES start and the Newton-step tolerance
__global__ void __launch_bounds__(kNB) k_pn_setup2(PtView v) {
  const int z = blockIdx.x;
  if (v.done[z]) return;
  __shared__ double sh[kNB];
  double s = 0.0;
  for (int b = threadIdx.x; b < v.nvb; b += kNB) s += v.dots[((size_t)z * v.nvb + b) * (v.m + 2)];
  s = nk_block_sum(s, sh);
  if (threadIdx.x == 0) {
    const double f = v.red[z * 4 + 1];
    const double nrm = sqrt(s + f * f);
    double* V0 = v.V + (size_t)z * (v.m + 1) * v.n1;
    V0[v.n] = f;
    v.phinorm[z] = nrm;
    v.beta0[z] = nrm;
    v.g[(size_t)z * (v.m + 1)] = nrm;
    v.gm_k[z] = 0;
    v.gm_conv[z] = nrm > 0.0 ? 0 : 1;
    v.rtol[z] = fmin(1e-3, fmax(1e-6, 1e-2 * v.red[z * 4 + 0]));
    v.hcol[(size_t)z * (v.m + 2) + v.m + 1] = nrm > 0.0 ? -1.0 / nrm : 0.0;
  }
}

// x[0:len] *= hcol[m+1]; optionally rhs = x[0:n]
__global__ void __launch_bounds__(kNB) k_pn_scale(PtView v, double* __restrict__ x, size_t xstride, int copy_rhs,
                                                  const int* __restrict__ skip) {
  const int z = blockIdx.y;
  if (skip[z]) return;
  const double a = v.hcol[(size_t)z * (v.m + 2) + v.m + 1];
  double* xz = x + (size_t)z * xstride;
  NK_FOR(r, v.n1) {
    const double y = xz[r] * a;
    xz[r] = y;
    if (copy_rhs && r < v.n) v.rhs[(size_t)z * v.n + r] = y;
  }
}

// partial sums of a[0:n] (per instance stride astride) into dots slot q
__global__ void __launch_bounds__(kNB) k_pn_psum(PtView v, const double* __restrict__ a, size_t astride, int q,
                                                 const int* __restrict__ skip) {
  const int z = blockIdx.y;
  if (skip[z]) return;
  __shared__ double sh[kNB];
  double s = 0.0;
  NK_FOR(r, v.n) s += a[(size_t)z * astride + r];
  s = nk_block_sum(s, sh);
  if (threadIdx.x == 0) v.dots[((size_t)z * v.nvb + blockIdx.x) * (v.m + 2) + q] = s;
}

__device__ __forceinline__ double pn_total(const PtView& v, int z, int q, double* sh) {
  double s = 0.0;
  for (int b = threadIdx.x; b < v.nvb; b += kNB) s += v.dots[((size_t)z * v.nvb + b) * (v.m + 2) + q];
  return nk_block_sum(s, sh);
}

// partial sums of Z_j[0:n] into slot 0, j from v.jd (the device-driven solve)
__global__ void __launch_bounds__(kNB) k_pn_psum_zj(PtView v) {
  const int z = blockIdx.y;
  if (v.skip[z]) return;
  __shared__ double sh[kNB];
  const int j = *v.jd;
  const double* a = v.Z + ((size_t)z * v.m + j) * v.n1;
  double s = 0.0;
  NK_FOR(r, v.n) s += a[r];
  s = nk_block_sum(s, sh);
  if (threadIdx.x == 0) v.dots[((size_t)z * v.nvb + blockIdx.x) * (v.m + 2)] = s;
}

// zH = sigma; den = h^2 sum zH (after k_pn_psum of sigma into slot 0); first PAQIF input = V_0[0:n]
__global__ void __launch_bounds__(kNB) k_pn_border(PtView v) {
  const int z = blockIdx.x;
  if (v.done[z]) return;
  __shared__ double sh[kNB];
  const double s = pn_total(v, z, 0, sh);
  const double h = v.inst[z].h;
  if (threadIdx.x == 0) v.den[z] = fabs(h * h * s) > 1e-300 ? h * h * s : 1e-300;
  const double* V0 = v.V + (size_t)z * (v.m + 1) * v.n1;
  for (int r = threadIdx.x; r < v.n; r += kNB) {
    v.zH[(size_t)z * v.n + r] = v.sigma[(size_t)z * v.n + r];
    v.rhs[(size_t)z * v.n + r] = V0[r];
  }
}

// xi = (h^2 sum sigma - V_j[n]) / den  (after k_pn_psum of sigma into slot 0)
__global__ void __launch_bounds__(kNB) k_pn_prec2(PtView v, int j) {
  if (v.jd) j = *v.jd;
  const int z = blockIdx.x;
  if (v.skip[z]) return;
  __shared__ double sh[kNB];
  const double s = pn_total(v, z, 0, sh);
  if (threadIdx.x == 0) {
    const double h = v.inst[z].h;
    const double* Vj = v.V + ((size_t)z * (v.m + 1) + j) * v.n1;
    const double xi = (h * h * s - Vj[v.n]) / v.den[z];
    v.zh0[z] = xi;
    v.Z[((size_t)z * v.m + j) * v.n1 + v.n] = xi;
  }
}

// Z_j = sigma - xi zH on the interior; the nodal copy for the deformation (0 on the boundary)
__global__ void __launch_bounds__(kNB) k_pn_prec3(PtView v, int j) {
  if (v.jd) j = *v.jd;
  const int z = blockIdx.y;
  if (v.skip[z]) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= v.NN) return;
  const int jj = t / v.nx, ii = t % v.nx;
  double val = 0.0;
  if (ii >= 1 && ii <= v.nx - 2 && jj >= 1 && jj <= v.ny - 2) {
    const int r = (jj - 1) * (v.nx - 2) + (ii - 1);
    const size_t o = (size_t)z * v.n + r;
    val = v.sigma[o] - v.zh0[z] * v.zH[o];
    v.Z[((size_t)z * v.m + j) * v.n1 + r] = val;
  }
  v.znode[(size_t)z * v.NN + t] = val;
}

// ---- y-line stage of the preconditioner (Sec. 3.3.2-3.3.4: the y-line systems of the alternating
// splitting): z = z1 + M_y^-1 (v - J z1), M_y the bordered solve on the y-line bands
__device__ __forceinline__ int pn_ty(int r, int nx, int ny) {  // row-major interior -> column-major
  return (r % (nx - 2)) * (ny - 2) + r / (nx - 2);
}

// dst (column-major) = src (row-major) on the interior
__global__ void __launch_bounds__(kNB) k_pn_ytrans(PtView v, const double* __restrict__ src,
                                                   double* __restrict__ dst, const int* __restrict__ skip) {
  const int z = blockIdx.y;
  if (skip[z]) return;
  NK_FOR(r, v.n) dst[(size_t)z * v.n + pn_ty(r, v.nx, v.ny)] = src[(size_t)z * v.n + r];
}

// zHy (row-major) = sig_y (column-major): the y-line solve of the border column
__global__ void __launch_bounds__(kNB) k_pn_ytrans_back(PtView v, const int* __restrict__ skip) {
  const int z = blockIdx.y;
  if (skip[z]) return;
  NK_FOR(r, v.n) v.zHy[(size_t)z * v.n + r] = v.sig_y[(size_t)z * v.n + pn_ty(r, v.nx, v.ny)];
}

// den_y = h^2 sum zHy (after k_pn_psum of zHy into slot 0)
__global__ void __launch_bounds__(kNB) k_pn_yden(PtView v) {
  const int z = blockIdx.x;
  if (v.done[z]) return;
  __shared__ double sh[kNB];
  const double s = pn_total(v, z, 0, sh);
  if (threadIdx.x == 0) {
    const double h = v.inst[z].h;
    v.deny[z] = fabs(h * h * s) > 1e-300 ? h * h * s : 1e-300;
  }
}

// rhs_y = (V_j - J z1)[0:n] in column-major order (w holds J z1)
__global__ void __launch_bounds__(kNB) k_pn_yrhs(PtView v, int j) {
  if (v.jd) j = *v.jd;
  const int z = blockIdx.y;
  if (v.skip[z]) return;
  const double* Vj = v.V + ((size_t)z * (v.m + 1) + j) * v.n1;
  const double* wz = v.w + (size_t)z * v.n1;
  NK_FOR(r, v.n) v.rhs_y[(size_t)z * v.n + pn_ty(r, v.nx, v.ny)] = Vj[r] - wz[r];
}

// xi_y = (h^2 sum sig_y - (V_j[n] - w[n])) / den_y (after k_pn_psum of sig_y into slot 0); the
// border component of Z_j and of the deformation input grows by xi_y
__global__ void __launch_bounds__(kNB) k_pn_yprec2(PtView v, int j) {
  if (v.jd) j = *v.jd;
  const int z = blockIdx.x;
  if (v.skip[z]) return;
  __shared__ double sh[kNB];
  const double s = pn_total(v, z, 0, sh);
  if (threadIdx.x == 0) {
    const double h = v.inst[z].h;
    const double* Vj = v.V + ((size_t)z * (v.m + 1) + j) * v.n1;
    const double r1n = Vj[v.n] - v.w[(size_t)z * v.n1 + v.n];
    const double xi = (h * h * s - r1n) / v.deny[z];
    v.xiy[z] = xi;
    v.zh0[z] += xi;
    v.Z[((size_t)z * v.m + j) * v.n1 + v.n] += xi;
  }
}

// Z_j += sig_y - xi_y zHy on the interior; the nodal copy for the deformation (0 on the boundary)
__global__ void __launch_bounds__(kNB) k_pn_yprec3(PtView v, int j) {
  if (v.jd) j = *v.jd;
  const int z = blockIdx.y;
  if (v.skip[z]) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= v.NN) return;
  const int jj = t / v.nx, ii = t % v.nx;
  double val = 0.0;
  if (ii >= 1 && ii <= v.nx - 2 && jj >= 1 && jj <= v.ny - 2) {
    const int r = (jj - 1) * (v.nx - 2) + (ii - 1);
    const size_t o = (size_t)z * v.n + r;
    double* Zj = v.Z + ((size_t)z * v.m + j) * v.n1;
    val = Zj[r] + v.sig_y[(size_t)z * v.n + pn_ty(r, v.nx, v.ny)] - v.xiy[z] * v.zHy[o];
    Zj[r] = val;
  }
  v.znode[(size_t)z * v.NN + t] = val;
}

// w = J_Phi Z_j on the interior rows (the force row by k_pn_psum + k_pn_force)
struct PnRowArgs {
  const double *P, *H, *rho, *drho, *deta_rel, *eps, *psia, *psib, *dH;
};
// The direction-independent factors of the Jacobian product, once per Newton step, so that a
// Krylov product needs no float64 division (the FP64 pipe runs at 1/64 of the FP32 rate)
__global__ void __launch_bounds__(256) k_pn_jvcoef(PtView v, PnRowArgs q) {
  const int z = blockIdx.y;
  if (v.done[z]) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= v.NN) return;
  const size_t k = (size_t)z * v.NN + t;
  const double e = q.eps[k], Hk = q.H[k];
  double4_32a c;
  c.x = q.drho[k] * Hk;
  c.y = 3.0 * e / Hk;
  c.z = e * (q.drho[k] / q.rho[k] - q.deta_rel[k]);
  c.w = 0.0;
  const int jj = t / v.nx, ii = t % v.nx;
  if (ii >= 1 && ii <= v.nx - 2 && jj >= 1 && jj <= v.ny - 2) {
    const int r = (jj - 1) * (v.nx - 2) + (ii - 1);
    c.w = 1.0 / v.dg[(size_t)z * v.n + r];
  }
  reinterpret_cast<double4_32a*>(v.jc)[k] = c;
}

__global__ void __launch_bounds__(kNB) k_pn_jv(PtView v, PnRowArgs q, int j) {
  if (v.jd) j = *v.jd;
  const int z = blockIdx.y;
  if (v.skip[z]) return;
  const PointInst in = v.inst[z];
  const int nx = v.nx;
  const size_t base = (size_t)z * v.NN;
  const double* Zj = v.Z + ((size_t)z * v.m + j) * v.n1;
  const double ih = 1.0 / in.h, ih2 = ih * ih;
  NK_FOR(r, v.n) {
    const size_t o = (size_t)z * v.n + r;
    const int i = r % (nx - 2) + 1, jj = r / (nx - 2) + 1;
    double out;
    if (v.act[o]) {
      out = Zj[r];
    } else {
      auto idx = [&](int p, int qq) { return base + (size_t)qq * nx + p; };
      auto dH = [&](int p, int qq) { return q.dH[idx(p, qq)]; };
      auto zn = [&](int p, int qq) { return v.znode[idx(p, qq)]; };
      const double4_32a* jc = reinterpret_cast<const double4_32a*>(v.jc);
      auto dU = [&](int p, int qq) {
        const size_t k = idx(p, qq);
        return q.rho[k] * dH(p, qq) + jc[k].x * zn(p, qq);
      };
      auto dE = [&](int p, int qq) {
        const size_t k = idx(p, qq);
        const double4_32a cc = jc[k];
        return cc.y * dH(p, qq) + cc.z * zn(p, qq);
      };
      auto dF = [&](int f, int qq) {
        const double d0 = dU(f, qq);
        if (f == 0) return d0;
        const size_t k = idx(f, qq);
        return d0 + 0.5 * (q.psia[k] * (d0 - dU(f - 1, qq)) + q.psib[k] * (dU(f + 1, qq) - d0));
      };
      const size_t c = idx(i, jj);
      const double e = q.eps[c], p = q.P[c];
      const double ex1 = 0.5 * (e + q.eps[c + 1]), ex0 = 0.5 * (q.eps[c - 1] + e);
      const double ey1 = 0.5 * (e + q.eps[c + nx]), ey0 = 0.5 * (q.eps[c - nx] + e);
      const double dEc = dE(i, jj), z0 = zn(i, jj);
      const double dC = (dF(i, jj) - dF(i - 1, jj)) * ih;
      const double dq = 0.5 * (dEc + dE(i + 1, jj)) * (q.P[c + 1] - p) + ex1 * (zn(i + 1, jj) - z0) -
                        0.5 * (dE(i - 1, jj) + dEc) * (p - q.P[c - 1]) - ex0 * (z0 - zn(i - 1, jj)) +
                        0.5 * (dEc + dE(i, jj + 1)) * (q.P[c + nx] - p) + ey1 * (zn(i, jj + 1) - z0) -
                        0.5 * (dE(i, jj - 1) + dEc) * (p - q.P[c - nx]) - ey0 * (z0 - zn(i, jj - 1));
      out = (dC - dq * ih2) * jc[c].w;
    }
    v.w[(size_t)z * v.n1 + r] = out;
  }
}

// w[n] = h^2 sum Z_j[0:n] (after k_pn_psum of Z_j into slot 0)
__global__ void __launch_bounds__(kNB) k_pn_force(PtView v) {
  const int z = blockIdx.x;
  if (v.skip[z]) return;
  __shared__ double sh[kNB];
  const double s = pn_total(v, z, 0, sh);
  if (threadIdx.x == 0) {
    const double h = v.inst[z].h;
    v.w[(size_t)z * v.n1 + v.n] = h * h * s;
  }
}

// partial dot products w . V_i, i = 0..j, into dots slots 0..j
// the block's partials of V_i . w for i = 0..j: per i a warp-shuffle sum, one word per warp in
// shared memory, and every 32 dot products one combine of the warps (two barriers per 32)
__global__ void __launch_bounds__(kNB) k_pn_dots(PtView v, int j) {
  if (v.jd) j = *v.jd;
  const int z = blockIdx.y;
  if (v.skip[z]) return;
  __shared__ double sh[kNB / 32][32];
  const double* wz = v.w + (size_t)z * v.n1;
  double wv[kNV];
  int rr[kNV];
#pragma unroll
  for (int k = 0; k < kNV; ++k) {
    rr[k] = blockIdx.x * (kNB * kNV) + threadIdx.x + k * kNB;
    wv[k] = rr[k] < v.n1 ? wz[rr[k]] : 0.0;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* out = v.dots + ((size_t)z * v.nvb + blockIdx.x) * (v.m + 2);
  for (int i0 = 0; i0 <= j; i0 += 32) {
    const int i1 = min(j + 1, i0 + 32);
    for (int i = i0; i < i1; ++i) {
      const double* Vi = v.V + ((size_t)z * (v.m + 1) + i) * v.n1;
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < kNV; ++k)
        if (rr[k] < v.n1) s += wv[k] * Vi[rr[k]];
      s = nk_warp_sum(s);
      if (lane == 0) sh[warp][i - i0] = s;
    }
    __syncthreads();
    if (threadIdx.x < i1 - i0) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < kNB / 32; ++w) t += sh[w][threadIdx.x];
      out[i0 + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

// h_i = sum of the partials; H(:, j) = h (first pass) or += h (second pass)
// one warp per h_i: its lanes sum the blocks' partials with shuffles (no block barriers)
__global__ void __launch_bounds__(kNB) k_pn_hsum(PtView v, int j, int pass) {
  if (v.jd) j = *v.jd;
  const int z = blockIdx.x;
  if (v.skip[z]) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* H = v.Hh + (size_t)z * (v.m + 1) * v.m;
  for (int i = warp; i <= j; i += kNB / 32) {
    double s = 0.0;
    for (int b = lane; b < v.nvb; b += 32) s += v.dots[((size_t)z * v.nvb + b) * (v.m + 2) + i];
    s = nk_warp_sum(s);
    if (lane == 0) {
      v.hcol[(size_t)z * (v.m + 2) + i] = s;
      H[i + (size_t)j * (v.m + 1)] = pass == 0 ? s : H[i + (size_t)j * (v.m + 1)] + s;
    }
  }
}

// w -= sum_i h_i V_i
__global__ void __launch_bounds__(kNB) k_pn_orth(PtView v, int j) {
  if (v.jd) j = *v.jd;
  const int z = blockIdx.y;
  if (v.skip[z]) return;
  const double* hz = v.hcol + (size_t)z * (v.m + 2);
  double* wz = v.w + (size_t)z * v.n1;
  NK_FOR(r, v.n1) {
    double s = wz[r];
    for (int i = 0; i <= j; ++i) s -= hz[i] * v.V[((size_t)z * (v.m + 1) + i) * v.n1 + r];
    wz[r] = s;
  }
}

// partial |w|^2 into slot 0
__global__ void __launch_bounds__(kNB) k_pn_norm(PtView v) {
  const int z = blockIdx.y;
  if (v.skip[z]) return;
  __shared__ double sh[kNB];
  const double* wz = v.w + (size_t)z * v.n1;
  double s = 0.0;
  NK_FOR(r, v.n1) s += wz[r] * wz[r];
  s = nk_block_sum(s, sh);
  if (threadIdx.x == 0) v.dots[((size_t)z * v.nvb + blockIdx.x) * (v.m + 2)] = s;
}

// H(j+1, j) = |w|; Givens rotations; convergence; 1/|w| for the normalisation
__global__ void __launch_bounds__(kNB) k_pn_givens(PtView v, int j) {
  if (v.jd) j = *v.jd;
  const int z = blockIdx.x;
  if (v.skip[z]) return;
  __shared__ double sh[kNB];
  const double nn = sqrt(pn_total(v, z, 0, sh));
  if (threadIdx.x != 0) return;
  const int m = v.m;
  double* H = v.Hh + (size_t)z * (m + 1) * m;
  double* cs = v.cs + (size_t)z * m;
  double* sn = v.sn + (size_t)z * m;
  double* g = v.g + (size_t)z * (m + 1);
  H[j + 1 + (size_t)j * (m + 1)] = nn;
  for (int i = 0; i < j; ++i) {
    const double a = H[i + (size_t)j * (m + 1)], b = H[i + 1 + (size_t)j * (m + 1)];
    H[i + (size_t)j * (m + 1)] = cs[i] * a + sn[i] * b;
    H[i + 1 + (size_t)j * (m + 1)] = -sn[i] * a + cs[i] * b;
  }
  const double a = H[j + (size_t)j * (m + 1)], b = H[j + 1 + (size_t)j * (m + 1)];
  const double rr = hypot(a, b);
  const double c = rr > 0.0 ? a / rr : 1.0, s = rr > 0.0 ? b / rr : 0.0;
  cs[j] = c;
  sn[j] = s;
  H[j + (size_t)j * (m + 1)] = rr;
  H[j + 1 + (size_t)j * (m + 1)] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  v.gm_k[z] = j + 1;
  if (fabs(g[j + 1]) <= v.rtol[z] * v.beta0[z] || j + 1 == m || nn == 0.0) v.gm_conv[z] = 1;
  v.hcol[(size_t)z * (m + 2) + m + 1] = nn > 0.0 ? 1.0 / nn : 0.0;
}

// V_{j+1} = w / |w|, next PAQIF input
__global__ void __launch_bounds__(kNB) k_pn_next(PtView v, int j) {
  if (v.jd) j = *v.jd;
  const int z = blockIdx.y;
  if (v.skip[z]) return;
  const double a = v.hcol[(size_t)z * (v.m + 2) + v.m + 1];
  double* Vn = v.V + ((size_t)z * (v.m + 1) + j + 1) * v.n1;
  const double* wz = v.w + (size_t)z * v.n1;
  NK_FOR(r, v.n1) {
    const double y = wz[r] * a;
    Vn[r] = y;
    if (r < v.n) v.rhs[(size_t)z * v.n + r] = y;
  }
}

// y = R^-1 g (into hcol), then the step delta = sum y_q Z_q
__global__ void __launch_bounds__(kNB) k_pn_ysolve(PtView v) {
  const int z = blockIdx.x;
  if (v.done[z]) return;
  if (threadIdx.x != 0) return;
  const int m = v.m, k = v.gm_k[z];
  const double* H = v.Hh + (size_t)z * (m + 1) * m;
  const double* g = v.g + (size_t)z * (m + 1);
  double* y = v.hcol + (size_t)z * (m + 2);
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int q = i + 1; q < k; ++q) s -= H[i + (size_t)q * (m + 1)] * y[q];
    const double dgl = H[i + (size_t)i * (m + 1)];
    y[i] = dgl != 0.0 ? s / dgl : 0.0;
  }
  v.tstep[z] = 1.0;
  v.lsdone[z] = 0;
  v.lsphase[z] = 0;
}
__global__ void __launch_bounds__(kNB) k_pn_delta(PtView v) {
  const int z = blockIdx.y;
  if (v.done[z]) return;
  const int k = v.gm_k[z];
  const double* y = v.hcol + (size_t)z * (v.m + 2);
  NK_FOR(r, v.n1) {
    double s = 0.0;
    for (int q = 0; q < k; ++q) s += y[q] * v.Z[((size_t)z * v.m + q) * v.n1 + r];
    v.delta[(size_t)z * v.n1 + r] = s;
  }
}

// trial point (projected in phase 0)
__global__ void __launch_bounds__(kNB) k_pn_trial(PtView v, const double* __restrict__ P,
                                                  const double* __restrict__ H0) {
  const int z = blockIdx.y;
  if (v.skip[z]) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= v.NN) return;
  const int jj = t / v.nx, ii = t % v.nx;
  const double st = v.tstep[z];
  double val = 0.0;
  if (ii >= 1 && ii <= v.nx - 2 && jj >= 1 && jj <= v.ny - 2) {
    const int r = (jj - 1) * (v.nx - 2) + (ii - 1);
    val = P[(size_t)z * v.NN + t] + st * v.delta[(size_t)z * v.n1 + r];
    if (v.lsphase[z] == 0) val = val > 0.0 ? val : 0.0;
  }
  v.Pt[(size_t)z * v.NN + t] = val;
  if (t == 0) v.H0t[z] = H0[z] + st * v.delta[(size_t)z * v.n1 + v.n];
}

// partial |min(P_t, R_t/d)|^2 (slot 0) and a non-finite count (slot 1)
__global__ void __launch_bounds__(kNB) k_pn_merit1(PtView v) {
  const int z = blockIdx.y;
  if (v.skip[z]) return;
  __shared__ double sh[kNB];
  double s = 0.0, nf = 0.0;
  NK_FOR(r, v.n) {
    const size_t node = (size_t)z * v.NN + nk_node(r, v.nx);
    const double pt = v.Pt[node], rt = v.R[node] / v.dg[(size_t)z * v.n + r];
    const double ph = pt < rt ? pt : rt;
    if (!(ph == ph) || isinf(ph)) nf += 1.0;
    s += ph * ph;
  }
  s = nk_block_sum(s, sh);
  nf = nk_block_sum(nf, sh);
  if (threadIdx.x == 0) {
    double* d = v.dots + ((size_t)z * v.nvb + blockIdx.x) * (v.m + 2);
    d[0] = s;
    d[1] = nf;
  }
}

// accept (H0 here, P by k_pn_accept) or shorten the step
__global__ void __launch_bounds__(kNB) k_pn_merit2(PtView v, double* __restrict__ H0) {
  const int z = blockIdx.x;
  if (v.skip[z]) return;
  __shared__ double sh[kNB];
  const double s = pn_total(v, z, 0, sh);
  const double nf = pn_total(v, z, 1, sh);
  if (threadIdx.x != 0) return;
  const double f = v.red[z * 4 + 1];
  const double nrm = sqrt(s + f * f);
  const double t = v.tstep[z];
  const int phase = v.lsphase[z];
  const bool ok = nf == 0.0 && nrm == nrm && nrm <= (1.0 - 1e-4 * t) * v.phinorm[z];
  const bool accept = ok || (phase == 1 && t < 1e-10);
  v.acc[z] = accept ? 1 : 0;
  if (accept) {
    H0[z] = v.H0t[z];
    v.lsdone[z] = 1;
  } else if (phase == 0 && 0.5 * t < 0x1p-10) {
    v.lsphase[z] = 1;
    v.tstep[z] = 1.0;
  } else {
    v.tstep[z] = 0.5 * t;
  }
}

__global__ void k_pn_accept(PtView v, double* __restrict__ P) {
  const int z = blockIdx.y;
  if (v.skip[z] || !v.acc[z]) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < v.NN) P[(size_t)z * v.NN + t] = v.Pt[(size_t)z * v.NN + t];
}

// ----------------------------------------------------------------- host side
static PtView pt_view(PtCtx* c, const int* skip) {
  PtView v;
  v.inst = c->inst;
  v.nx = c->nx;
  v.ny = c->ny;
  v.NN = c->NN;
  v.n = c->n;
  v.n1 = c->n + 1;
  v.m = c->m;
  v.nvb = c->nvb;
  v.beta = c->beta;
  v.done = c->done;
  v.skip = skip;
  v.V = c->V;
  v.Z = c->Z;
  v.Hh = c->Hh;
  v.cs = c->cs;
  v.sn = c->sn;
  v.g = c->g;
  v.w = c->w;
  v.dots = c->dots;
  v.hcol = c->hcol;
  v.delta = c->delta;
  v.zH = c->zH;
  v.rhs = c->rhs;
  v.sigma = c->sigma;
  v.band = c->band;
  v.jh = c->jh;
  v.dg = c->dg;
  v.R = c->R;
  v.red = c->red;
  v.phinorm = c->phinorm;
  v.den = c->den;
  v.rtol = c->rtol;
  v.beta0 = c->beta0;
  v.tstep = c->tstep;
  v.zh0 = c->zh0;
  v.H0t = c->H0t;
  v.Pt = c->Pt;
  v.znode = c->znode;
  v.act = c->act;
  v.gm_k = c->gm_k;
  v.gm_conv = c->gm_conv;
  v.lsdone = c->lsdone;
  v.lsphase = c->lsphase;
  v.acc = c->acc;
  v.rhs_y = c->rhs_y;
  v.sig_y = c->sig_y;
  v.zHy = c->zHy;
  v.deny = c->deny;
  v.xiy = c->xiy;
  v.jd = nullptr;
  v.jc = c->jc;
  return v;
}

static cudaError_t pn_paqif(PtCtx* c, const double* rhs, double* x, bool factor) {
  PaqifLaunch L;
  L.n_sys = c->lines;
  L.n = c->nx - 2;
  L.beta = c->beta;
  L.mode = 0;
  L.band = c->band;
  L.rhs = rhs;
  L.act = nullptr;
  L.stack = c->pq_ws;
  L.x = x;
  L.iters = nullptr;
  L.info = c->pq_info;
  L.parts = c->pq_r;
  // double-float sweeps at every precision: with float32 x-line solves the 2-D Newton
  // iteration stalls (C4: 60 steps without convergence, against 14 in double-float)
  return factor ? launch_paqif_factor(L, c->fstore, c->st) : launch_paqif_resolve(L, c->fstore, c->st);
}

static cudaError_t pn_paqif_y(PtCtx* c, bool factor) {
  PaqifLaunch L;
  L.n_sys = c->ylines;
  L.n = c->ny - 2;
  L.beta = c->beta;
  L.mode = 0;
  L.band = c->band_y;
  L.rhs = c->rhs_y;
  L.act = nullptr;
  L.stack = c->pq_ws_y;
  L.x = c->sig_y;
  L.iters = nullptr;
  L.info = c->pq_info_y;
  return factor ? launch_paqif_factor(L, c->fstore_y, c->st) : launch_paqif_resolve(L, c->fstore_y, c->st);
}

static bool pn_all(PtCtx* c, const int* a, const int* b, cudaError_t& e) {
  std::vector<int> ha(c->n_inst), hb(c->n_inst);
  e = cudaMemcpyAsync(ha.data(), a, sizeof(int) * c->n_inst, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess && b) e = cudaMemcpyAsync(hb.data(), b, sizeof(int) * c->n_inst, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  for (int k = 0; k < c->n_inst; ++k)
    if (!ha[k] && !(b && hb[k])) return false;
  return true;
}

cudaError_t pt_nk_step(PtCtx* c, double* P, double* H0, const double* rough) {
  const int ni = c->n_inst;
  cudaError_t e = pt_state(c, P, H0, rough, c->done);
  if (e == cudaSuccess) e = pt_finalize(c, c->done, c->iters);
  if (e == cudaSuccess) e = pt_jac_band(c, P, c->band, c->act, c->jh, c->dg, c->done);
  if (e != cudaSuccess) return e;
  const dim3 gv(c->nvb, ni), gn((c->NN + 255) / 256, ni);
  PtView vd = pt_view(c, c->done);
  k_pn_setup<<<gv, kNB, 0, c->st>>>(vd, P);
  note_launch();
  k_pn_setup2<<<ni, kNB, 0, c->st>>>(vd);
  note_launch();
  {
    const PnRowArgs qc{P, c->H, c->rho, c->drho, c->deta_rel, c->eps, c->psia, c->psib, c->dH};
    k_pn_jvcoef<<<gn, 256, 0, c->st>>>(vd, qc);
    note_launch();
  }
  k_pn_scale<<<gv, kNB, 0, c->st>>>(vd, c->V, (size_t)(c->m + 1) * (c->n + 1), 0, c->done);
  note_launch();
  if (c->yline) {
    // y-line bands of the scaled system, their factorization solving for the border column
    e = pt_jac_yband(c, P, c->act, c->dg, c->band_y, 1, c->done);
    if (e != cudaSuccess) return e;
    k_pn_ytrans<<<gv, kNB, 0, c->st>>>(vd, c->rhs, c->rhs_y, c->done);
    note_launch();
    e = pn_paqif_y(c, true);  // sig_y = B_y^-1 (dR/dH0)/d
    if (e != cudaSuccess) return e;
    k_pn_ytrans_back<<<gv, kNB, 0, c->st>>>(vd, c->done);
    note_launch();
    k_pn_psum<<<gv, kNB, 0, c->st>>>(vd, c->zHy, (size_t)c->n, 0, c->done);
    note_launch();
    k_pn_yden<<<ni, kNB, 0, c->st>>>(vd);
    note_launch();
  }
  e = pn_paqif(c, c->rhs, c->sigma, true);  // factor; sigma = B^-1 (dR/dH0)/d
  if (e != cudaSuccess) return e;
  k_pn_psum<<<gv, kNB, 0, c->st>>>(vd, c->sigma, (size_t)c->n, 0, c->done);
  note_launch();
  k_pn_border<<<ni, kNB, 0, c->st>>>(vd);
  note_launch();
  PtView vs = pt_view(c, c->skip);
  const PnRowArgs q{P, c->H, c->rho, c->drho, c->deta_rel, c->eps, c->psia, c->psib, c->dH};
  for (int j = 0; j < c->m; ++j) {
    k_pn_skip<<<(ni + 127) / 128, 128, 0, c->st>>>(c->done, c->gm_conv, c->skip, ni);
    note_launch();
    e = pn_paqif(c, c->rhs, c->sigma, false);
    if (e != cudaSuccess) return e;
    k_pn_psum<<<gv, kNB, 0, c->st>>>(vs, c->sigma, (size_t)c->n, 0, c->skip);
    note_launch();
    k_pn_prec2<<<ni, kNB, 0, c->st>>>(vs, j);
    note_launch();
    k_pn_prec3<<<gn, 256, 0, c->st>>>(vs, j);
    note_launch();
    if (c->yline) {
      // w = J z1, then Z_j = z1 + M_y^-1 (V_j - w)
      e = pt_deform_dir(c, c->znode, c->zh0, c->skip);
      if (e != cudaSuccess) return e;
      k_pn_jv<<<gv, kNB, 0, c->st>>>(vs, q, j);
      note_launch();
      k_pn_psum<<<gv, kNB, 0, c->st>>>(vs, c->Z + (size_t)j * (c->n + 1), (size_t)c->m * (c->n + 1), 0, c->skip);
      note_launch();
      k_pn_force<<<ni, kNB, 0, c->st>>>(vs);
      note_launch();
      k_pn_yrhs<<<gv, kNB, 0, c->st>>>(vs, j);
      note_launch();
      e = pn_paqif_y(c, false);
      if (e != cudaSuccess) return e;
      k_pn_psum<<<gv, kNB, 0, c->st>>>(vs, c->sig_y, (size_t)c->n, 0, c->skip);
      note_launch();
      k_pn_yprec2<<<ni, kNB, 0, c->st>>>(vs, j);
      note_launch();
      k_pn_yprec3<<<gn, 256, 0, c->st>>>(vs, j);
      note_launch();
    }
    // dH = K z + xi: the deformation of the Krylov vector
    e = pt_deform_dir(c, c->znode, c->zh0, c->skip);
    if (e != cudaSuccess) return e;
    k_pn_jv<<<gv, kNB, 0, c->st>>>(vs, q, j);
    note_launch();
    k_pn_psum<<<gv, kNB, 0, c->st>>>(vs, c->Z + (size_t)j * (c->n + 1), (size_t)c->m * (c->n + 1), 0, c->skip);
    note_launch();
    k_pn_force<<<ni, kNB, 0, c->st>>>(vs);
    note_launch();
    for (int pass = 0; pass < 2; ++pass) {
      k_pn_dots<<<gv, kNB, 0, c->st>>>(vs, j);
      note_launch();
      k_pn_hsum<<<ni, kNB, 0, c->st>>>(vs, j, pass);
      note_launch();
      k_pn_orth<<<gv, kNB, 0, c->st>>>(vs, j);
      note_launch();
    }
    k_pn_norm<<<gv, kNB, 0, c->st>>>(vs);
    note_launch();
    k_pn_givens<<<ni, kNB, 0, c->st>>>(vs, j);
    note_launch();
    k_pn_next<<<gv, kNB, 0, c->st>>>(vs, j);
    note_launch();
    if ((j + 1) % 8 == 0 && j + 1 < c->m) {
      if (pn_all(c, c->done, c->gm_conv, e)) break;
      if (e != cudaSuccess) return e;
    }
  }
  std::vector<int> tk, tc;
  std::vector<double> tphin;
  if (c->trace) {
    const int nt = c->trace < ni ? c->trace : ni;
    tk.resize(nt);
    tc.resize(nt);
    tphin.resize(nt);
    e = cudaMemcpyAsync(tk.data(), c->gm_k, sizeof(int) * nt, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tc.data(), c->gm_conv, sizeof(int) * nt, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(tphin.data(), c->phinorm, sizeof(double) * nt, cudaMemcpyDeviceToHost, c->st);
    if (e != cudaSuccess) return e;
  }
  k_pn_ysolve<<<ni, kNB, 0, c->st>>>(vd);
  note_launch();
  k_pn_delta<<<gv, kNB, 0, c->st>>>(vd);
  note_launch();
  for (int trial = 0; trial < 64; ++trial) {
    k_pn_skip<<<(ni + 127) / 128, 128, 0, c->st>>>(c->done, c->lsdone, c->skip, ni);
    note_launch();
    k_pn_trial<<<gn, 256, 0, c->st>>>(vs, P, H0);
    note_launch();
    e = pt_state(c, c->Pt, c->H0t, rough, c->skip);
    if (e == cudaSuccess) e = pt_finalize(c, nullptr, nullptr);
    if (e != cudaSuccess) return e;
    k_pn_merit1<<<gv, kNB, 0, c->st>>>(vs);
    note_launch();
    k_pn_merit2<<<ni, kNB, 0, c->st>>>(vs, H0);
    note_launch();
    k_pn_accept<<<gn, 256, 0, c->st>>>(vs, P);
    note_launch();
    if (pn_all(c, c->done, c->lsdone, e)) break;
    if (e != cudaSuccess) return e;
  }
  if (c->trace) {
    const int nt = (int)tk.size();
    std::vector<double> tt(nt), tred(4 * nt);
    std::vector<int> tph(nt), tdone(nt), tit(nt);
    e = cudaMemcpyAsync(tt.data(), c->tstep, sizeof(double) * nt, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tph.data(), c->lsphase, sizeof(int) * nt, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tdone.data(), c->done, sizeof(int) * nt, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tit.data(), c->iters, sizeof(int) * nt, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return e;
    for (int z = 0; z < nt; ++z)
      if (!tdone[z])
        fprintf(stderr, "ehl pt %dx%d inst %d it %d |Phi| %.3e gmres %d conv %d t %.3e phase %d\n", c->nx, c->ny, z,
                tit[z], tphin[z], tk[z], tc[z], tt[z], tph[z]);
  }
  return cudaGetLastError();
}


// ============================================= device-driven solve (graph mode 2)
// The Newton steps of one grid, their GMRES iterations and line-search trials as three nested
// while-nodes of one CUDA graph (as for line contact): the kernels of pt_nk_step, the Krylov index
// read from a device counter, each loop's condition set by k_nk_loop.
namespace {
cudaError_t pn_loop(PtCtx* c, cudaGraphConditionalHandle h, int slot, int total_slot, int cap, int next,
                    const int* other) {
  k_nk_loop<<<1, 256, 0, c->st>>>(h, c->loop + slot, total_slot >= 0 ? c->loop + total_slot : nullptr, cap, next,
                                  c->done, other, c->n_inst);
  note_launch();
  return cudaGetLastError();
}
}  // namespace

cudaError_t pt_nk_capture_solve(PtCtx* c, double* P, double* H0, const double* rough, cudaStream_t s1, cudaStream_t s2,
                                PtGraphCounts& n) {
  const int ni = c->n_inst;
  const cudaStream_t s0 = c->st;
  const dim3 gv(c->nvb, ni), gn((c->NN + 255) / 256, ni);
  PtView vd = pt_view(c, c->done);
  PtView vs = pt_view(c, c->skip);
  vs.jd = c->loop + 1;
  const PnRowArgs q{P, c->H, c->rho, c->drho, c->deta_rel, c->eps, c->psia, c->psib, c->dH};
  const unsigned long long l0 = thread_launches();
  cudaError_t e = cudaMemsetAsync(c->done, 0, sizeof(int) * ni, s0);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->iters, 0, sizeof(int) * ni, s0);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->best, 0x7f, sizeof(double) * ni, s0);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->stall, 0, sizeof(int) * ni, s0);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->loop, 0, sizeof(int) * 8, s0);
  auto krylov_body = [&](cudaGraphConditionalHandle hk) -> cudaError_t {
    k_pn_skip<<<(ni + 127) / 128, 128, 0, c->st>>>(c->done, c->gm_conv, c->skip, ni);
    note_launch();
    cudaError_t ee = pn_paqif(c, c->rhs, c->sigma, false);
    if (ee != cudaSuccess) return ee;
    k_pn_psum<<<gv, kNB, 0, c->st>>>(vs, c->sigma, (size_t)c->n, 0, c->skip);
    note_launch();
    k_pn_prec2<<<ni, kNB, 0, c->st>>>(vs, 0);
    note_launch();
    k_pn_prec3<<<gn, 256, 0, c->st>>>(vs, 0);
    note_launch();
    if (c->yline) {
      ee = pt_deform_dir(c, c->znode, c->zh0, c->skip);
      if (ee != cudaSuccess) return ee;
      k_pn_jv<<<gv, kNB, 0, c->st>>>(vs, q, 0);
      note_launch();
      k_pn_psum_zj<<<gv, kNB, 0, c->st>>>(vs);
      note_launch();
      k_pn_force<<<ni, kNB, 0, c->st>>>(vs);
      note_launch();
      k_pn_yrhs<<<gv, kNB, 0, c->st>>>(vs, 0);
      note_launch();
      ee = pn_paqif_y(c, false);
      if (ee != cudaSuccess) return ee;
      k_pn_psum<<<gv, kNB, 0, c->st>>>(vs, c->sig_y, (size_t)c->n, 0, c->skip);
      note_launch();
      k_pn_yprec2<<<ni, kNB, 0, c->st>>>(vs, 0);
      note_launch();
      k_pn_yprec3<<<gn, 256, 0, c->st>>>(vs, 0);
      note_launch();
    }
    ee = pt_deform_dir(c, c->znode, c->zh0, c->skip);
    if (ee != cudaSuccess) return ee;
    k_pn_jv<<<gv, kNB, 0, c->st>>>(vs, q, 0);
    note_launch();
    k_pn_psum_zj<<<gv, kNB, 0, c->st>>>(vs);
    note_launch();
    k_pn_force<<<ni, kNB, 0, c->st>>>(vs);
    note_launch();
    for (int pass = 0; pass < 2; ++pass) {
      k_pn_dots<<<gv, kNB, 0, c->st>>>(vs, 0);
      note_launch();
      k_pn_hsum<<<ni, kNB, 0, c->st>>>(vs, 0, pass);
      note_launch();
      k_pn_orth<<<gv, kNB, 0, c->st>>>(vs, 0);
      note_launch();
    }
    k_pn_norm<<<gv, kNB, 0, c->st>>>(vs);
    note_launch();
    k_pn_givens<<<ni, kNB, 0, c->st>>>(vs, 0);
    note_launch();
    k_pn_next<<<gv, kNB, 0, c->st>>>(vs, 0);
    note_launch();
    return pn_loop(c, hk, 1, 3, c->m, 1, c->gm_conv);
  };
  auto trial_body = [&](cudaGraphConditionalHandle ht) -> cudaError_t {
    k_pn_skip<<<(ni + 127) / 128, 128, 0, c->st>>>(c->done, c->lsdone, c->skip, ni);
    note_launch();
    k_pn_trial<<<gn, 256, 0, c->st>>>(vs, P, H0);
    note_launch();
    cudaError_t ee = pt_state(c, c->Pt, c->H0t, rough, c->skip);
    if (ee == cudaSuccess) ee = pt_finalize(c, nullptr, nullptr);
    if (ee != cudaSuccess) return ee;
    k_pn_merit1<<<gv, kNB, 0, c->st>>>(vs);
    note_launch();
    k_pn_merit2<<<ni, kNB, 0, c->st>>>(vs, H0);
    note_launch();
    k_pn_accept<<<gn, 256, 0, c->st>>>(vs, P);
    note_launch();
    return pn_loop(c, ht, 2, 4, 64, 1, c->lsdone);
  };
  auto newton_body = [&](cudaGraphConditionalHandle hn) -> cudaError_t {
    const unsigned long long m0 = thread_launches();
    cudaError_t ee = pt_state(c, P, H0, rough, c->done);
    if (ee == cudaSuccess) ee = pt_finalize(c, c->done, c->iters);
    if (ee == cudaSuccess) ee = pt_jac_band(c, P, c->band, c->act, c->jh, c->dg, c->done);
    if (ee != cudaSuccess) return ee;
    k_pn_setup<<<gv, kNB, 0, c->st>>>(vd, P);
    note_launch();
    k_pn_setup2<<<ni, kNB, 0, c->st>>>(vd);
    note_launch();
    k_pn_jvcoef<<<gn, 256, 0, c->st>>>(vd, q);
    note_launch();
    k_pn_scale<<<gv, kNB, 0, c->st>>>(vd, c->V, (size_t)(c->m + 1) * (c->n + 1), 0, c->done);
    note_launch();
    if (c->yline) {
      ee = pt_jac_yband(c, P, c->act, c->dg, c->band_y, 1, c->done);
      if (ee != cudaSuccess) return ee;
      k_pn_ytrans<<<gv, kNB, 0, c->st>>>(vd, c->rhs, c->rhs_y, c->done);
      note_launch();
      ee = pn_paqif_y(c, true);
      if (ee != cudaSuccess) return ee;
      k_pn_ytrans_back<<<gv, kNB, 0, c->st>>>(vd, c->done);
      note_launch();
      k_pn_psum<<<gv, kNB, 0, c->st>>>(vd, c->zHy, (size_t)c->n, 0, c->done);
      note_launch();
      k_pn_yden<<<ni, kNB, 0, c->st>>>(vd);
      note_launch();
    }
    ee = pn_paqif(c, c->rhs, c->sigma, true);
    if (ee != cudaSuccess) return ee;
    k_pn_psum<<<gv, kNB, 0, c->st>>>(vd, c->sigma, (size_t)c->n, 0, c->done);
    note_launch();
    k_pn_border<<<ni, kNB, 0, c->st>>>(vd);
    note_launch();
    const cudaStream_t here = c->st;
    ee = capture_while(
        c, here, s2, [&](cudaGraphConditionalHandle hk) { return pn_loop(c, hk, 1, -1, c->m, 0, c->gm_conv); },
        krylov_body, &n.krylov);
    if (ee != cudaSuccess) return ee;
    k_pn_ysolve<<<ni, kNB, 0, c->st>>>(vd);
    note_launch();
    k_pn_delta<<<gv, kNB, 0, c->st>>>(vd);
    note_launch();
    ee = capture_while(
        c, here, s2, [&](cudaGraphConditionalHandle ht) { return pn_loop(c, ht, 2, -1, 64, 0, c->lsdone); },
        trial_body, &n.trial);
    if (ee != cudaSuccess) return ee;
    ee = pn_loop(c, hn, 0, -1, c->max_iter, 1, nullptr);
    n.newton = (long long)(thread_launches() - m0) - n.krylov - n.trial;
    return ee;
  };
  if (e == cudaSuccess)
    e = capture_while(
        c, s0, s1, [&](cudaGraphConditionalHandle hn) { return pn_loop(c, hn, 0, -1, c->max_iter, 0, nullptr); },
        newton_body, nullptr);
  c->st = s0;
  n.fixed = (long long)(thread_launches() - l0) - n.newton - n.krylov - n.trial;
  return e;
}

// ===================================================================== adjoint
// Sensitivities of a converged point-contact state, as for line contact: the
// transposed bordered system of the equation rows solved by restarted GMRES on
// the exact transposed operator (the transposed 2-D stencil of the residual
// plus one float64 deformation per product; K is symmetric and H = ... + K P),
// preconditioned by PAQIF on the transposed x-line bands, with the force
// column h^2 and the dR/dH0 row as border.
namespace {

struct PtAdj {
  double *bandT = nullptr, *cb = nullptr, *hvec = nullptr, *zr = nullptr, *gx = nullptr, *mu = nullptr;
  double *res = nullptr, *wn = nullptr, *gHn = nullptr, *gPn = nullptr, *relres = nullptr, *gxn = nullptr;
  int* adone = nullptr;
  void* fstore = nullptr;
};

struct PaNodes {
  const double *P, *H, *rho, *drho, *deta_rel, *eps, *psia, *psib;
};

// adjoint of the node perturbations (dU, dE, zn) at node (p, q) for row weights wn
__device__ __forceinline__ void pa_local(const PaNodes& q, const double* __restrict__ wn, size_t base, int p, int qq,
                                         int nx, int ny, double h, double& aU, double& aE, double& aZ) {
  auto W = [&](int i, int j) { return (i >= 0 && i < nx && j >= 0 && j < ny) ? wn[base + (size_t)j * nx + i] : 0.0; };
  auto idx = [&](int i, int j) { return base + (size_t)j * nx + i; };
  auto phx = [&](int f) { return (f >= 0 && f <= nx - 2) ? (W(f, qq) - W(f + 1, qq)) / h : 0.0; };
  auto phy = [&](int g) { return (g >= 0 && g <= ny - 2) ? (W(p, g) - W(p, g + 1)) / h : 0.0; };
  auto pa = [&](int f) { return (f >= 0 && f <= nx - 2) ? q.psia[idx(f, qq)] : 0.0; };
  auto pb = [&](int f) { return (f >= 0 && f <= nx - 2) ? q.psib[idx(f, qq)] : 0.0; };
  const double fm = phx(p), fm1 = phx(p - 1), fp1 = phx(p + 1);
  aU = fm * (1.0 + 0.5 * pa(p) - 0.5 * pb(p)) - 0.5 * pa(p + 1) * fp1 + 0.5 * pb(p - 1) * fm1;
  const double cx = -fm / h, cx1 = -fm1 / h;
  const double dPx = (p <= nx - 2) ? q.P[idx(p + 1, qq)] - q.P[idx(p, qq)] : 0.0;
  const double dPx1 = (p >= 1) ? q.P[idx(p, qq)] - q.P[idx(p - 1, qq)] : 0.0;
  const double ex = (p <= nx - 2) ? 0.5 * (q.eps[idx(p, qq)] + q.eps[idx(p + 1, qq)]) : 0.0;
  const double ex1 = (p >= 1) ? 0.5 * (q.eps[idx(p - 1, qq)] + q.eps[idx(p, qq)]) : 0.0;
  const double cy = -phy(qq) / h, cy1 = -phy(qq - 1) / h;
  const double dPy = (qq <= ny - 2) ? q.P[idx(p, qq + 1)] - q.P[idx(p, qq)] : 0.0;
  const double dPy1 = (qq >= 1) ? q.P[idx(p, qq)] - q.P[idx(p, qq - 1)] : 0.0;
  const double ey = (qq <= ny - 2) ? 0.5 * (q.eps[idx(p, qq)] + q.eps[idx(p, qq + 1)]) : 0.0;
  const double ey1 = (qq >= 1) ? 0.5 * (q.eps[idx(p, qq - 1)] + q.eps[idx(p, qq)]) : 0.0;
  aE = 0.5 * (cx * dPx + cx1 * dPx1) + 0.5 * (cy * dPy + cy1 * dPy1);
  aZ = (cx1 * ex1 - cx * ex) + (cy1 * ey1 - cy * ey);
}

__global__ void k_pa_local(const PointInst* __restrict__ inst, PaNodes q, const double* __restrict__ wn,
                           const int* __restrict__ skip, double* __restrict__ gHn, double* __restrict__ gPn) {
  const int z = blockIdx.y;
  if (skip && skip[z]) return;
  const PointInst in = inst[z];
  const int nx = in.nx, ny = in.ny, NN = nx * ny;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NN) return;
  const size_t base = (size_t)z * NN, o = base + t;
  double aU, aE, aZ;
  pa_local(q, wn, base, t % nx, t / nx, nx, ny, in.h, aU, aE, aZ);
  const double e = q.eps[o], H = q.H[o], r = q.rho[o];
  gHn[o] = aU * r + aE * 3.0 * e / H;
  gPn[o] = aU * q.drho[o] * H + aE * e * (q.drho[o] / r - q.deta_rel[o]) + aZ;
}

__global__ void k_pa_prepare(PtView v, PtAdj a) {
  const int z = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= v.n) return;
  const int w = 2 * v.beta + 1;
  const size_t o = (size_t)z * v.n + r;
  if (!v.act[o]) {
    const double d = v.dg[o];
    double* row = v.band + o * w;
    const double rd = 1.0 / d;
    for (int t = 0; t < w; ++t) row[t] *= rd;
    a.cb[o] = v.jh[o] / d;
  } else {
    a.cb[o] = 0.0;
  }
  const double h = v.inst[z].h;
  a.hvec[o] = h * h;
}

// transposed x-line bands: bandT[line][r][j] = band[line][r - beta + j][2 beta - j]
__global__ void k_pa_transpose(PtView v, PtAdj a) {
  const int z = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= v.n) return;
  const int ni = v.nx - 2, beta = v.beta, w = 2 * beta + 1;
  const int line = r / ni, rl = r % ni;
  const double* B = v.band + ((size_t)z * v.n + (size_t)line * ni) * w;
  double* T = a.bandT + ((size_t)z * v.n + r) * w;
  for (int j = 0; j < w; ++j) {
    const int sr = rl - beta + j;
    T[j] = (sr >= 0 && sr < ni) ? B[(size_t)sr * w + (2 * beta - j)] : 0.0;
  }
}

// gx[0:n] = gP + K gH (dH holds K gH), partial |gx|^2 in slot 0; partial sum gH over nodes in slot 1
__global__ void __launch_bounds__(kNB) k_pa_rhs(PtView v, PtAdj a, const double* __restrict__ gP,
                                                const double* __restrict__ gH, const double* __restrict__ dH) {
  const int z = blockIdx.y;
  __shared__ double sh[kNB];
  double ss = 0.0, sH = 0.0;
  NK_FOR(r, v.n) {
    const size_t node = (size_t)z * v.NN + nk_node(r, v.nx);
    const double g = (gP ? gP[node] : 0.0) + (gH ? dH[node] : 0.0);
    a.gx[(size_t)z * v.n1 + r] = g;
    ss += g * g;
  }
  // nodes by a grid-stride loop (NN exceeds the interior count the vector blocks cover)
  if (gH)
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < v.NN; t += gridDim.x * blockDim.x)
      sH += gH[(size_t)z * v.NN + t];
  ss = nk_block_sum(ss, sh);
  sH = nk_block_sum(sH, sh);
  if (threadIdx.x == 0) {
    double* d = v.dots + ((size_t)z * v.nvb + blockIdx.x) * (v.m + 2);
    d[0] = ss;
    d[1] = sH;
  }
}

__global__ void __launch_bounds__(kNB) k_pa_rhs2(PtView v, PtAdj a, const double* __restrict__ gH0) {
  const int z = blockIdx.x;
  __shared__ double sh[kNB];
  const double ss = pn_total(v, z, 0, sh), sH = pn_total(v, z, 1, sh);
  if (threadIdx.x == 0) {
    const double gn = (gH0 ? gH0[z] : 0.0) + sH;
    a.gx[(size_t)z * v.n1 + v.n] = gn;
    a.gxn[z] = sqrt(ss + gn * gn);
    a.adone[z] = 0;
  }
}

__global__ void __launch_bounds__(kNB) k_pa_init(PtView v, PtAdj a) {
  const int z = blockIdx.y;
  NK_FOR(r, v.n1) {
    a.mu[(size_t)z * v.n1 + r] = 0.0;
    a.res[(size_t)z * v.n1 + r] = a.gx[(size_t)z * v.n1 + r];
  }
}

// partial sum of cb . x[0:n] into slot 0 (x of instance z at x + z xstride)
__global__ void __launch_bounds__(kNB) k_pa_cdot(PtView v, PtAdj a, const double* __restrict__ x, size_t xstride,
                                                 const int* __restrict__ skip) {
  const int z = blockIdx.y;
  if (skip && skip[z]) return;
  __shared__ double sh[kNB];
  double s = 0.0;
  NK_FOR(r, v.n) s += a.cb[(size_t)z * v.n + r] * x[(size_t)z * xstride + r];
  s = nk_block_sum(s, sh);
  if (threadIdx.x == 0) v.dots[((size_t)z * v.nvb + blockIdx.x) * (v.m + 2)] = s;
}

__global__ void __launch_bounds__(kNB) k_pa_den(PtView v, PtAdj a) {
  const int z = blockIdx.x;
  __shared__ double sh[kNB];
  const double s = pn_total(v, z, 0, sh);
  if (threadIdx.x == 0) v.den[z] = fabs(s) > 1e-300 ? s : 1e-300;
}

// restart: |res| (after partial sums of res^2 in slot 0), V_0 = res/|res|, GMRES state
__global__ void __launch_bounds__(kNB) k_pa_norm_res(PtView v, PtAdj a) {
  const int z = blockIdx.y;
  if (a.adone[z]) return;
  __shared__ double sh[kNB];
  double s = 0.0;
  NK_FOR(r, v.n1) {
    const double x = a.res[(size_t)z * v.n1 + r];
    s += x * x;
  }
  s = nk_block_sum(s, sh);
  if (threadIdx.x == 0) v.dots[((size_t)z * v.nvb + blockIdx.x) * (v.m + 2)] = s;
}

__global__ void __launch_bounds__(kNB) k_pa_start2(PtView v, PtAdj a, double tol, int* __restrict__ skip) {
  const int z = blockIdx.x;
  __shared__ double sh[kNB];
  const double nrm = a.adone[z] ? 0.0 : sqrt(pn_total(v, z, 0, sh));
  if (threadIdx.x == 0) {
    v.g[(size_t)z * (v.m + 1)] = nrm;
    v.gm_k[z] = 0;
    v.beta0[z] = a.gxn[z];
    v.rtol[z] = 0.1 * tol;
    v.gm_conv[z] = (a.adone[z] || nrm <= 0.1 * tol * a.gxn[z]) ? 1 : 0;
    skip[z] = v.gm_conv[z];
    v.hcol[(size_t)z * (v.m + 2) + v.m + 1] = nrm > 0.0 ? 1.0 / nrm : 0.0;
  }
}

__global__ void __launch_bounds__(kNB) k_pa_v0(PtView v, PtAdj a) {
  const int z = blockIdx.y;
  if (v.skip[z]) return;
  const double s = v.hcol[(size_t)z * (v.m + 2) + v.m + 1];
  double* V0 = v.V + (size_t)z * (v.m + 1) * v.n1;
  NK_FOR(r, v.n1) {
    const double y = a.res[(size_t)z * v.n1 + r] * s;
    V0[r] = y;
    if (r < v.n) v.rhs[(size_t)z * v.n + r] = y;
  }
}

// xi = (cb . sigma - V_j[n]) / den (after k_pa_cdot of sigma)
__global__ void __launch_bounds__(kNB) k_pa_prec2(PtView v, int j) {
  const int z = blockIdx.x;
  if (v.skip[z]) return;
  __shared__ double sh[kNB];
  const double s = pn_total(v, z, 0, sh);
  if (threadIdx.x == 0) {
    const double* Vj = v.V + ((size_t)z * (v.m + 1) + j) * v.n1;
    const double xi = (s - Vj[v.n]) / v.den[z];
    v.zh0[z] = xi;
    v.Z[((size_t)z * v.m + j) * v.n1 + v.n] = xi;
  }
}

// Z_j = sigma - xi zr; row weights wn = Z_j / d on the equation rows
__global__ void __launch_bounds__(kNB) k_pa_prec3(PtView v, PtAdj a, int j) {
  const int z = blockIdx.y;
  if (v.skip[z]) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= v.NN) return;
  const int jj = t / v.nx, ii = t % v.nx;
  double wv = 0.0;
  if (ii >= 1 && ii <= v.nx - 2 && jj >= 1 && jj <= v.ny - 2) {
    const int r = (jj - 1) * (v.nx - 2) + (ii - 1);
    const size_t o = (size_t)z * v.n + r;
    const double val = v.sigma[o] - v.zh0[z] * a.zr[o];
    v.Z[((size_t)z * v.m + j) * v.n1 + r] = val;
    wv = v.act[o] ? 0.0 : val / v.dg[o];
  }
  a.wn[(size_t)z * v.NN + t] = wv;
}

// wn = x / d on the equation rows (x of instance z at x + z n1)
__global__ void k_pa_weights(PtView v, PtAdj a, const double* __restrict__ x, const int* __restrict__ skip) {
  const int z = blockIdx.y;
  if (skip && skip[z]) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= v.NN) return;
  const int jj = t / v.nx, ii = t % v.nx;
  double wv = 0.0;
  if (ii >= 1 && ii <= v.nx - 2 && jj >= 1 && jj <= v.ny - 2) {
    const int r = (jj - 1) * (v.nx - 2) + (ii - 1);
    const size_t o = (size_t)z * v.n + r;
    wv = v.act[o] ? 0.0 : x[(size_t)z * v.n1 + r] / v.dg[o];
  }
  a.wn[(size_t)z * v.NN + t] = wv;
}

// out[0:n] = gP(w) + K gH(w) + x on identity rows + h^2 xi; partial cb . x into slot 0
__global__ void __launch_bounds__(kNB) k_pa_combine(PtView v, PtAdj a, const double* __restrict__ x, size_t xstride,
                                                    const double* __restrict__ dH, double* __restrict__ out,
                                                    const int* __restrict__ skip) {
  const int z = blockIdx.y;
  if (skip && skip[z]) return;
  __shared__ double sh[kNB];
  const double* xz = x + (size_t)z * xstride;
  const double h = v.inst[z].h, xi = xz[v.n];
  double s = 0.0;
  NK_FOR(r, v.n) {
    const size_t o = (size_t)z * v.n + r;
    const size_t node = (size_t)z * v.NN + nk_node(r, v.nx);
    out[(size_t)z * v.n1 + r] = a.gPn[node] + dH[node] + (v.act[o] ? xz[r] : 0.0) + h * h * xi;
    s += a.cb[o] * xz[r];
  }
  s = nk_block_sum(s, sh);
  if (threadIdx.x == 0) v.dots[((size_t)z * v.nvb + blockIdx.x) * (v.m + 2)] = s;
}

__global__ void __launch_bounds__(kNB) k_pa_combine2(PtView v, double* __restrict__ out, const int* __restrict__ skip) {
  const int z = blockIdx.x;
  if (skip && skip[z]) return;
  __shared__ double sh[kNB];
  const double s = pn_total(v, z, 0, sh);
  if (threadIdx.x == 0) out[(size_t)z * v.n1 + v.n] = s;
}

__global__ void __launch_bounds__(kNB) k_pa_mu(PtView v, PtAdj a) {
  const int z = blockIdx.y;
  if (a.adone[z]) return;
  NK_FOR(r, v.n1) a.mu[(size_t)z * v.n1 + r] += v.delta[(size_t)z * v.n1 + r];
}

// res = gx - w, partial |res|^2 in slot 0
__global__ void __launch_bounds__(kNB) k_pa_resid(PtView v, PtAdj a) {
  const int z = blockIdx.y;
  if (a.adone[z]) return;
  __shared__ double sh[kNB];
  double s = 0.0;
  NK_FOR(r, v.n1) {
    const size_t o = (size_t)z * v.n1 + r;
    const double x = a.gx[o] - v.w[o];
    a.res[o] = x;
    s += x * x;
  }
  s = nk_block_sum(s, sh);
  if (threadIdx.x == 0) v.dots[((size_t)z * v.nvb + blockIdx.x) * (v.m + 2)] = s;
}

__global__ void __launch_bounds__(kNB) k_pa_resid2(PtView v, PtAdj a, double tol) {
  const int z = blockIdx.x;
  if (a.adone[z]) return;
  __shared__ double sh[kNB];
  const double s = pn_total(v, z, 0, sh);
  if (threadIdx.x == 0) {
    const double gn = a.gxn[z];
    const double rel = gn > 0.0 ? sqrt(s) / gn : 0.0;
    a.relres[z] = rel;
    if (!(rel > tol)) a.adone[z] = 1;
  }
}

// grad_rough = gH - g_H(lambda) per node; partial parameter sums (M slot 0, L slot 1)
__global__ void __launch_bounds__(kNB) k_pa_grad(PtView v, PtAdj a, PaNodes q, const double* __restrict__ gH,
                                                 double* __restrict__ grad_rough) {
  const int z = blockIdx.y;
  __shared__ double sh[kNB];
  const PointInst in = v.inst[z];
  const size_t base = (size_t)z * v.NN;
  // point Moes: d ln(lambda)/dM = -4/(3M), d ln(pH)/dM = 1/(3M), d ln(pH)/dL = 1/L
  const double lpM = 1.0 / (3.0 * in.m.M), lpL = 1.0 / in.m.L, llM = -4.0 / (3.0 * in.m.M);
  double sM = 0.0, sL = 0.0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < v.NN; t += gridDim.x * blockDim.x) {
    const size_t o = base + t;
    double aU, aE, aZ;
    pa_local(q, a.wn, base, t % v.nx, t / v.nx, v.nx, v.ny, in.h, aU, aE, aZ);
    const double P = q.P[o], H = q.H[o], r = q.rho[o], e = q.eps[o];
    const double drl = q.drho[o] * P, del = q.deta_rel[o] * P;
    sM += aU * H * drl * lpM + aE * e * ((drl / r - del) * lpM - llM);
    sL += aU * H * drl * lpL + aE * e * ((drl / r - del) * lpL);
    if (grad_rough) grad_rough[o] = (gH ? gH[o] : 0.0) - a.gHn[o];
  }
  sM = nk_block_sum(sM, sh);
  sL = nk_block_sum(sL, sh);
  if (threadIdx.x == 0) {
    double* d = v.dots + ((size_t)z * v.nvb + blockIdx.x) * (v.m + 2);
    d[0] = sM;
    d[1] = sL;
  }
}

__global__ void __launch_bounds__(kNB) k_pa_grad2(PtView v, double* __restrict__ grad_ML) {
  const int z = blockIdx.x;
  __shared__ double sh[kNB];
  const double sM = pn_total(v, z, 0, sh), sL = pn_total(v, z, 1, sh);
  if (threadIdx.x == 0 && grad_ML) {
    grad_ML[2 * z] = -sM;
    grad_ML[2 * z + 1] = -sL;
  }
}

}  // namespace

static cudaError_t pa_paqif(PtCtx* c, PtAdj& a, const double* rhs, double* x, bool factor) {
  PaqifLaunch L;
  L.n_sys = c->lines;
  L.n = c->nx - 2;
  L.beta = c->beta;
  L.mode = 0;
  L.band = a.bandT;
  L.rhs = rhs;
  L.act = nullptr;
  L.stack = c->pq_ws;
  L.x = x;
  L.iters = nullptr;
  L.info = c->pq_info;
  return factor ? launch_paqif_factor(L, a.fstore, c->st) : launch_paqif_resolve(L, a.fstore, c->st);
}

// out = Phi_x^T x with the row weights of x in a.wn
static cudaError_t pa_apply(PtCtx* c, PtAdj& a, const PtView& v, const PaNodes& q, const double* x, size_t xstride,
                            double* out, const int* skip) {
  const int ni = c->n_inst;
  const dim3 gn((c->NN + 255) / 256, ni), gv(c->nvb, ni);
  k_pa_local<<<gn, 256, 0, c->st>>>(c->inst, q, a.wn, skip, a.gHn, a.gPn);
  note_launch();
  cudaError_t e = pt_deform_dir64(c, a.gHn, skip);  // dH = K gH
  if (e != cudaSuccess) return e;
  k_pa_combine<<<gv, kNB, 0, c->st>>>(v, a, x, xstride, c->dH, out, skip);
  note_launch();
  k_pa_combine2<<<ni, kNB, 0, c->st>>>(v, out, skip);
  note_launch();
  return cudaGetLastError();
}

void pt_adj_free(PtCtx* c) {
  delete (PtAdj*)c->adj;
  c->adj = nullptr;
}

cudaError_t pt_adjoint(PtCtx* c, const double* P, const double* H0, const double* rough, const double* gP,
                       const double* gH, const double* gH0, double* grad_rough, double* grad_ML, double* relres,
                       double tol, int max_cycles) {
  const int ni = c->n_inst;
  if (!c->adj) {
    PtAdj* a = new PtAdj();
    c->adj = a;
    const size_t nt = (size_t)ni * c->n, n1t = (size_t)ni * (c->n + 1), NNt = (size_t)ni * c->NN;
    struct A {
      void** p;
      size_t bytes;
    } al[] = {{(void**)&a->bandT, sizeof(double) * nt * (2 * c->beta + 1)},
              {(void**)&a->cb, sizeof(double) * nt},
              {(void**)&a->hvec, sizeof(double) * nt},
              {(void**)&a->zr, sizeof(double) * nt},
              {(void**)&a->gx, sizeof(double) * n1t},
              {(void**)&a->mu, sizeof(double) * n1t},
              {(void**)&a->res, sizeof(double) * n1t},
              {(void**)&a->wn, sizeof(double) * NNt},
              {(void**)&a->gHn, sizeof(double) * NNt},
              {(void**)&a->gPn, sizeof(double) * NNt},
              {(void**)&a->relres, sizeof(double) * ni},
              {(void**)&a->gxn, sizeof(double) * ni},
              {(void**)&a->adone, sizeof(int) * ni},
              {(void**)&a->fstore, paqif_factor_store_bytes(c->lines, c->nx - 2, c->beta)}};
    for (auto& x : al) {
      cudaError_t e = pt_alloc(c, x.p, x.bytes);
      if (e != cudaSuccess) return e;
    }
  }
  PtAdj& a = *(PtAdj*)c->adj;
  cudaError_t e = pt_state(c, P, H0, rough, nullptr);
  if (e == cudaSuccess) e = pt_jac_band(c, P, c->band, c->act, c->jh, c->dg, nullptr);
  if (e != cudaSuccess) return e;
  PtView v = pt_view(c, c->skip);
  v.done = a.adone;
  const PaNodes q{P, c->H, c->rho, c->drho, c->deta_rel, c->eps, c->psia, c->psib};
  const dim3 gr((c->n + 127) / 128, ni), gv(c->nvb, ni), gn((c->NN + 255) / 256, ni);
  k_pa_prepare<<<gr, 128, 0, c->st>>>(v, a);
  note_launch();
  k_pa_transpose<<<gr, 128, 0, c->st>>>(v, a);
  note_launch();
  if (gH) {
    e = pt_deform_dir64(c, gH, nullptr);  // dH = K gH
    if (e != cudaSuccess) return e;
  }
  k_pa_rhs<<<gv, kNB, 0, c->st>>>(v, a, gP, gH, c->dH);
  note_launch();
  k_pa_rhs2<<<ni, kNB, 0, c->st>>>(v, a, gH0);
  note_launch();
  k_pa_init<<<gv, kNB, 0, c->st>>>(v, a);
  note_launch();
  e = pa_paqif(c, a, a.hvec, a.zr, true);  // factor B^T; zr = B^-T h^2
  if (e != cudaSuccess) return e;
  k_pa_cdot<<<gv, kNB, 0, c->st>>>(v, a, a.zr, (size_t)c->n, nullptr);
  note_launch();
  k_pa_den<<<ni, kNB, 0, c->st>>>(v, a);
  note_launch();
  for (int cyc = 0; cyc < max_cycles; ++cyc) {
    k_pa_norm_res<<<gv, kNB, 0, c->st>>>(v, a);
    note_launch();
    k_pa_start2<<<ni, kNB, 0, c->st>>>(v, a, tol, c->skip);
    note_launch();
    k_pa_v0<<<gv, kNB, 0, c->st>>>(v, a);
    note_launch();
    for (int j = 0; j < c->m; ++j) {
      e = pa_paqif(c, a, c->rhs, c->sigma, false);
      if (e != cudaSuccess) return e;
      k_pa_cdot<<<gv, kNB, 0, c->st>>>(v, a, c->sigma, (size_t)c->n, c->skip);
      note_launch();
      k_pa_prec2<<<ni, kNB, 0, c->st>>>(v, j);
      note_launch();
      k_pa_prec3<<<gn, 256, 0, c->st>>>(v, a, j);
      note_launch();
      e = pa_apply(c, a, v, q, c->Z + (size_t)j * (c->n + 1), (size_t)c->m * (c->n + 1), c->w, c->skip);
      if (e != cudaSuccess) return e;
      for (int pass = 0; pass < 2; ++pass) {
        k_pn_dots<<<gv, kNB, 0, c->st>>>(v, j);
        note_launch();
        k_pn_hsum<<<ni, kNB, 0, c->st>>>(v, j, pass);
        note_launch();
        k_pn_orth<<<gv, kNB, 0, c->st>>>(v, j);
        note_launch();
      }
      k_pn_norm<<<gv, kNB, 0, c->st>>>(v);
      note_launch();
      k_pn_givens<<<ni, kNB, 0, c->st>>>(v, j);
      note_launch();
      k_pn_next<<<gv, kNB, 0, c->st>>>(v, j);
      note_launch();
      k_pn_skip<<<(ni + 127) / 128, 128, 0, c->st>>>(a.adone, c->gm_conv, c->skip, ni);
      note_launch();
      if ((j + 1) % 8 == 0 && j + 1 < c->m) {
        if (pn_all(c, a.adone, c->gm_conv, e)) break;
        if (e != cudaSuccess) return e;
      }
    }
    k_pn_ysolve<<<ni, kNB, 0, c->st>>>(v);
    note_launch();
    k_pn_delta<<<gv, kNB, 0, c->st>>>(v);
    note_launch();
    k_pa_mu<<<gv, kNB, 0, c->st>>>(v, a);
    note_launch();
    k_pa_weights<<<gn, 256, 0, c->st>>>(v, a, a.mu, a.adone);
    note_launch();
    e = pa_apply(c, a, v, q, a.mu, (size_t)(c->n + 1), c->w, a.adone);
    if (e != cudaSuccess) return e;
    k_pa_resid<<<gv, kNB, 0, c->st>>>(v, a);
    note_launch();
    k_pa_resid2<<<ni, kNB, 0, c->st>>>(v, a, tol);
    note_launch();
    if (pn_all(c, a.adone, nullptr, e)) break;
    if (e != cudaSuccess) return e;
  }
  // lambda = mu / d on the equation rows; g_H(lambda); gradients
  k_pa_weights<<<gn, 256, 0, c->st>>>(v, a, a.mu, nullptr);
  note_launch();
  k_pa_local<<<gn, 256, 0, c->st>>>(c->inst, q, a.wn, nullptr, a.gHn, a.gPn);
  note_launch();
  k_pa_grad<<<gv, kNB, 0, c->st>>>(v, a, q, gH, grad_rough);
  note_launch();
  k_pa_grad2<<<ni, kNB, 0, c->st>>>(v, grad_ML);
  note_launch();
  if (relres) e = cudaMemcpyAsync(relres, a.relres, sizeof(double) * ni, cudaMemcpyDeviceToDevice, c->st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace ehl
