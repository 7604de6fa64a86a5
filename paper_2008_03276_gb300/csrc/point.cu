// point.cu -- point-contact hot path: 2-D deformation, TVD residual, x-line band
// Jacobian and the Newton-Krylov solve.
//
// Discrete problem (Sec. 3.3 Example 6 in two dimensions, Sec. 3.3.1 Case 2,
// Sec. 3.3.3): nodes X_i = xa + i h, Y_j = ya + j h, P = 0 on the boundary;
//   H_ij = H0 + X_i^2/2 + Y_j^2/2 + (2/pi^2) sum_kl G(i-k, j-l) P_kl + rough_ij,
//   G = cell integral of 1/r (closed form with asinh),
//   R_ij = (F_{i+1/2,j} - F_{i-1/2,j})/h - [x- and y-Poiseuille 5-point terms]/h^2,
//   F the limited x-face value of rho H (first order at the inflow face),
//   P >= 0, R >= 0, P R = 0,  h^2 sum P = 2 pi / 3.
// Arrays are [instance][j][i] (x fastest).  The solve is the semismooth
// Newton-Krylov method of the line contact: Phi = (min(P, R/d), h^2 sum P -
// 2 pi/3), GMRES on the exact Jacobian (one 2-D deformation per product),
// right-preconditioned by PAQIF on the x-line bands of the scaled exact
// Jacobian -- the paper's x-line systems, one per grid row -- bordered with
// the dR/dH0 column and the force row.  Vector reductions run over many
// blocks per instance (an instance has up to ~65k unknowns); the Arnoldi
// step is classical Gram-Schmidt applied twice.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <string.h>

#include <type_traits>
#include <vector>

#include "df64.cuh"
#include "ehl_internal.h"
#include "point.h"

namespace ehl {

constexpr int kPtNode = 256;    // threads of the node kernels
constexpr int kPtTI = 64;       // deformation tile: outputs along x
constexpr int kPtTJ = 4;        //                   output rows
constexpr int kPtSK = 128;      // source chunk along x (one partial sum per chunk)
constexpr int kPtSL = 8;        // source rows per shared-memory stage
constexpr int kPtVB = 256;      // threads of the vector kernels
constexpr int kPtVPT = 2;       // vector elements per thread (the Krylov kernels' kNV)

__device__ __forceinline__ double pt_block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ double pt_nan_max(double a, double b) { return (a != a || b != b) ? NAN : fmax(a, b); }

// interior index r -> node offset within the instance
__device__ __forceinline__ int pt_node(int r, int nx) {
  const int ni = nx - 2;
  return (r / ni + 1) * nx + (r % ni) + 1;
}

// F(x, y) = x asinh(y/|x|) + y asinh(x/|y|): antiderivative of 1/r over a cell
__device__ __forceinline__ double pt_F(double x, double y) {
  return x * asinh(y / fabs(x)) + y * asinh(x / fabs(y));
}

// -------------------------------------------------------------------- table
__global__ void k_pt_gtab(const PointInst* __restrict__ inst, float2* __restrict__ gtab, double* __restrict__ gtab64) {
  const int z = blockIdx.y;
  const PointInst q = inst[z];
  const int NN = q.nx * q.ny;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NN) return;
  const int b = t / q.nx, a = t % q.nx;  // y offset b, x offset a
  const double h = q.h;
  const double xp = (a + 0.5) * h, xm = (a - 0.5) * h, yp = (b + 0.5) * h, ym = (b - 0.5) * h;
  const double G = pt_F(xp, yp) - pt_F(xm, yp) - pt_F(xp, ym) + pt_F(xm, ym);
  const double v = (2.0 / (M_PI * M_PI)) * G;
  const df d = df_from_double(v);
  gtab[(size_t)z * NN + t] = make_float2(d.hi, d.lo);
  gtab64[(size_t)z * NN + t] = v;
}

// -------------------------------------------------------------- deformation
// partial[kc][z][j][i] = sum_{l} sum_{k in chunk kc} T[|j-l|][|i-k|] V[z][l][k]
template <bool F64>
__global__ void __launch_bounds__(kPtTI* kPtTJ) k_pt_deform(const PointInst* __restrict__ inst,
                                                           const float2* __restrict__ gtab,
                                                           const double* __restrict__ gtab64,
                                                           const double* __restrict__ V, const int* __restrict__ skip,
                                                           void* __restrict__ partial, int n_inst, int ksplit) {
  const int z = blockIdx.z / ksplit, kc = blockIdx.z % ksplit;
  if (skip && skip[z]) return;
  const PointInst q = inst[z];
  const int nx = q.nx, ny = q.ny, NN = nx * ny;
  const int i0 = blockIdx.x * kPtTI, j0 = blockIdx.y * kPtTJ, k0 = kc * kPtSK;
  const int ti = threadIdx.x % kPtTI, tj = threadIdx.x / kPtTI;
  const int i = i0 + ti, j = j0 + tj;
  using T = typename std::conditional<F64, double, float2>::type;
  __shared__ T Ps[kPtSL][kPtSK];
  __shared__ T Ts[kPtTJ + kPtSL - 1][kPtTI + kPtSK - 1];
  const double* Vz = V + (size_t)z * NN;
  double acc64 = 0.0;
  float s = 0.f, c = 0.f;
  if (q.m.elastic) {
    for (int l0 = 0; l0 < ny; l0 += kPtSL) {
      for (int t = threadIdx.x; t < kPtSL * kPtSK; t += blockDim.x) {
        const int ll = t / kPtSK, kk = t % kPtSK;
        const int l = l0 + ll, k = k0 + kk;
        const double v = (l < ny && k < nx) ? Vz[(size_t)l * nx + k] : 0.0;
        if constexpr (F64) {
          Ps[ll][kk] = v;
        } else {
          const df d = df_from_double(v);
          Ps[ll][kk] = make_float2(d.hi, d.lo);
        }
      }
      const int dy0 = j0 - l0 - kPtSL + 1, dx0 = i0 - k0 - kPtSK + 1;
      for (int t = threadIdx.x; t < (kPtTJ + kPtSL - 1) * (kPtTI + kPtSK - 1); t += blockDim.x) {
        const int qq = t / (kPtTI + kPtSK - 1), mm = t % (kPtTI + kPtSK - 1);
        int b = dy0 + qq, a = dx0 + mm;
        b = b < 0 ? -b : b;
        a = a < 0 ? -a : a;
        if constexpr (F64) {
          Ts[qq][mm] = (a < nx && b < ny) ? gtab64[(size_t)z * NN + (size_t)b * nx + a] : 0.0;
        } else {
          Ts[qq][mm] = (a < nx && b < ny) ? gtab[(size_t)z * NN + (size_t)b * nx + a] : make_float2(0.f, 0.f);
        }
      }
      __syncthreads();
      const int lmax = min(kPtSL, ny - l0), kmax = min(kPtSK, nx - k0);
      for (int ll = 0; ll < lmax; ++ll) {
        const T* trow = Ts[tj - ll + kPtSL - 1];
        const T* prow = Ps[ll];
#pragma unroll 4
        for (int kk = 0; kk < kmax; ++kk) {
          const T g = trow[ti - kk + kPtSK - 1];
          const T v = prow[kk];
          if constexpr (F64) {
            acc64 = fma(g, v, acc64);
          } else {
            const float p = __fmul_rn(g.x, v.x);
            float e = __fmaf_rn(g.x, v.x, -p);
            e = __fmaf_rn(g.x, v.y, e);
            e = __fmaf_rn(g.y, v.x, e);
            float t1, t2;
            two_sum(s, p, t1, t2);
            s = t1;
            c = __fadd_rn(c, __fadd_rn(t2, e));
          }
        }
      }
      __syncthreads();
    }
  }
  if (i >= nx || j >= ny) return;
  const size_t o = ((size_t)kc * n_inst + z) * NN + (size_t)j * nx + i;
  if constexpr (F64) {
    reinterpret_cast<double*>(partial)[o] = acc64;
  } else {
    float hi, lo;
    fast_two_sum(s, c, hi, lo);
    reinterpret_cast<float2*>(partial)[o] = make_float2(hi, lo);
  }
}

// mode 0: H = H0 + X^2/2 + Y^2/2 + D + rough;  mode 1: out = D + dh0
__global__ void k_pt_film(const PointInst* __restrict__ inst, const void* __restrict__ partial, int ksplit, int p64,
                          const double* __restrict__ H0, const double* __restrict__ rough, const int* __restrict__ skip,
                          double* __restrict__ out, int n_inst, int mode) {
  const int z = blockIdx.y;
  if (skip && skip[z]) return;
  const PointInst q = inst[z];
  const int NN = q.nx * q.ny;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NN) return;
  double D;
  if (p64 == 2) {  // one float32 product [n_inst][ny][ldc] (the GEMM path; ksplit carries ldc)
    const int ldc = ksplit, jj = t / q.nx, ii = t - jj * q.nx;
    D = (double)reinterpret_cast<const float*>(partial)[((size_t)z * q.ny + jj) * ldc + ii];
  } else if (p64) {
    const double* pd = reinterpret_cast<const double*>(partial);
    D = 0.0;
    for (int y = 0; y < ksplit; ++y) D += pd[((size_t)y * n_inst + z) * NN + t];
  } else {
    const float2* pf = reinterpret_cast<const float2*>(partial);
    df acc = df_zero();
    for (int y = 0; y < ksplit; ++y) {
      const float2 p = pf[((size_t)y * n_inst + z) * NN + t];
      acc = df_add(acc, make_df(p.x, p.y));
    }
    D = df_to_double(acc);
  }
  const size_t o = (size_t)z * NN + t;
  if (mode == 0) {
    const int j = t / q.nx, i = t % q.nx;
    const double X = q.xa + i * q.h, Y = q.ya + j * q.h;
    double H = H0[z] + 0.5 * X * X + 0.5 * Y * Y + D;
    if (rough) H += rough[o];
    out[o] = H;
  } else {
    out[o] = D + (H0 ? H0[z] : 0.0);
  }
}

// ------------------------------------------------------------------- state
__global__ void k_pt_nodes(const PointInst* __restrict__ inst, const double* __restrict__ P,
                           const double* __restrict__ H, const int* __restrict__ skip, double* __restrict__ rho,
                           double* __restrict__ drho, double* __restrict__ deta_rel, double* __restrict__ eps,
                           double* __restrict__ u) {
  const int z = blockIdx.y;
  if (skip && skip[z]) return;
  const PointInst q = inst[z];
  const int NN = q.nx * q.ny;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NN) return;
  const size_t o = (size_t)z * NN + t;
  double r, dr, ln_eta, de;
  line_material(q.m, P[o], r, dr, ln_eta, de);
  const double Hh = H[o];
  rho[o] = r;
  drho[o] = dr;
  deta_rel[o] = de;
  eps[o] = r * Hh * Hh * Hh / q.m.lam * exp(-ln_eta);
  u[o] = r * Hh;
}

// x-faces (j, f) between nodes f and f+1, f = 0..nx-2 (stored at j*nx + f)
__global__ void k_pt_faces(const PointInst* __restrict__ inst, const double* __restrict__ u,
                           const int* __restrict__ skip, double* __restrict__ F, double* __restrict__ psia,
                           double* __restrict__ psib) {
  const int z = blockIdx.y;
  if (skip && skip[z]) return;
  const PointInst q = inst[z];
  const int nx = q.nx, NN = nx * q.ny;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NN) return;
  const int f = t % nx;
  const size_t o = (size_t)z * NN + t;
  if (f > nx - 2) {
    F[o] = psia[o] = psib[o] = 0.0;
    return;
  }
  double ps = 0.0, pa = 0.0, pb = 0.0;
  if (f >= 1) line_limiter(q.m.limiter, q.m.kappa, u[o] - u[o - 1], u[o + 1] - u[o], ps, pa, pb);
  F[o] = u[o] + 0.5 * ps;
  psia[o] = pa;
  psib[o] = pb;
}

// residual at interior nodes; block partials (max |min(P,R)|, sum P, min H, max term)
__global__ void __launch_bounds__(kPtNode) k_pt_residual(const PointInst* __restrict__ inst,
                                                         const double* __restrict__ P, const double* __restrict__ H,
                                                         const double* __restrict__ eps, const double* __restrict__ F,
                                                         const int* __restrict__ skip, double* __restrict__ R,
                                                         double* __restrict__ blk, int nblk) {
  const int z = blockIdx.y;
  if (skip && skip[z]) return;
  const PointInst q = inst[z];
  const int nx = q.nx, ny = q.ny, NN = nx * ny;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const double h = q.h;
  double cres = 0.0, sp = 0.0, hmin = INFINITY, term = 0.0;
  if (t < NN) {
    const size_t o = (size_t)z * NN + t;
    const int j = t / nx, i = t % nx;
    hmin = H[o];
    if (i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2) {
      const double C = (F[o] - F[o - 1]) / h;
      const double ex1 = 0.5 * (eps[o] + eps[o + 1]), ex0 = 0.5 * (eps[o - 1] + eps[o]);
      const double ey1 = 0.5 * (eps[o] + eps[o + nx]), ey0 = 0.5 * (eps[o - nx] + eps[o]);
      const double p = P[o];
      const double qx1 = ex1 * (P[o + 1] - p), qx0 = ex0 * (p - P[o - 1]);
      const double qy1 = ey1 * (P[o + nx] - p), qy0 = ey0 * (p - P[o - nx]);
      const double r = C - (qx1 - qx0 + qy1 - qy0) / (h * h);
      R[o] = r;
      cres = fabs(p < r ? p : r);
      sp = p;
      term = (fabs(F[o]) + fabs(F[o - 1])) / h + (fabs(qx1) + fabs(qx0) + fabs(qy1) + fabs(qy0)) / (h * h);
    } else {
      R[o] = 0.0;
    }
  }
  __shared__ double s_c[kPtNode], s_s[kPtNode], s_h[kPtNode], s_t[kPtNode];
  s_c[threadIdx.x] = cres;
  s_s[threadIdx.x] = sp;
  s_h[threadIdx.x] = hmin;
  s_t[threadIdx.x] = term;
  __syncthreads();
  for (int w = kPtNode / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s_c[threadIdx.x] = pt_nan_max(s_c[threadIdx.x], s_c[threadIdx.x + w]);
      s_s[threadIdx.x] += s_s[threadIdx.x + w];
      s_h[threadIdx.x] = fmin(s_h[threadIdx.x], s_h[threadIdx.x + w]);
      s_t[threadIdx.x] = fmax(s_t[threadIdx.x], s_t[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double* b = blk + ((size_t)z * nblk + blockIdx.x) * 4;
    b[0] = s_c[0];
    b[1] = s_s[0];
    b[2] = s_h[0];
    b[3] = s_t[0];
  }
}

// red[z] = (max|min(P,R)|, h^2 sum P - 2 pi/3, sum P, min H); convergence as in line contact
__global__ void k_pt_finalize(const PointInst* __restrict__ inst, const double* __restrict__ blk, int nblk,
                              double* __restrict__ red, int* __restrict__ done, int* __restrict__ iters,
                              double* __restrict__ best, int* __restrict__ stall, int n_inst) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= n_inst) return;
  if (done && done[z]) return;
  double c = 0.0, s = 0.0, hm = INFINITY, tm = 0.0;
  for (int b = 0; b < nblk; ++b) {
    const double* p = blk + ((size_t)z * nblk + b) * 4;
    c = pt_nan_max(c, p[0]);
    s += p[1];
    hm = fmin(hm, p[2]);
    tm = fmax(tm, p[3]);
  }
  const double h = inst[z].h;
  const double force = h * h * s - 2.0 * M_PI / 3.0;
  red[z * 4 + 0] = c;
  red[z * 4 + 1] = force;
  red[z * 4 + 2] = s;
  red[z * 4 + 3] = hm;
  if (done) {
    const double tol = inst[z].m.tol;
    if (c <= tol && fabs(force) <= tol) {
      done[z] = 1;
      return;
    }
    if (!(c == c) || !(force == force)) {
      done[z] = 2;
      return;
    }
    if (best && stall) {
      if (c < 0.5 * best[z]) {
        best[z] = c;
        stall[z] = 0;
      } else {
        stall[z] += 1;
      }
      if (stall[z] >= 5 && c <= fmax(tol, 1e3 * DBL_EPSILON * tm) && fabs(force) <= tol) {
        done[z] = 1;
        return;
      }
    }
    if (iters) iters[z] += 1;
  }
}

__global__ void k_pt_hertz(const PointInst* __restrict__ inst, double* __restrict__ P) {
  const int z = blockIdx.y;
  const PointInst q = inst[z];
  const int NN = q.nx * q.ny;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NN) return;
  const int j = t / q.nx, i = t % q.nx;
  double v = 0.0;
  if (i >= 1 && i <= q.nx - 2 && j >= 1 && j <= q.ny - 2) {
    const double X = q.xa + i * q.h, Y = q.ya + j * q.h;
    const double r2 = 1.0 - X * X - Y * Y;
    v = r2 > 0.0 ? sqrt(r2) : 0.0;
  }
  P[(size_t)z * NN + t] = v;
}

__global__ void k_pt_set_h0(const PointInst* __restrict__ inst, const double* __restrict__ blk, int nblk,
                            double* __restrict__ H0, int n_inst) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= n_inst) return;
  double hm = INFINITY;
  for (int b = 0; b < nblk; ++b) hm = fmin(hm, blk[((size_t)z * nblk + b) * 4 + 2]);
  H0[z] = inst[z].m.h_init - hm;
}

// ------------------------------------------------------- exact linearisation
// Directional derivative of R at interior node (i, j) for the film change dH(p, q)
// and the pressure change zn(p, q) (functors of the node coordinates).
struct PtRow {
  const double *P, *H, *rho, *drho, *deta_rel, *eps, *psia, *psib;
  size_t base;
  int nx;
  double h;
  template <class DH, class ZN>
  __device__ __forceinline__ double jv(int i, int j, const DH& dH, const ZN& zn) const {
    auto idx = [&](int p, int q) { return base + (size_t)q * nx + p; };
    auto dU = [&](int p, int q) {
      const size_t o = idx(p, q);
      return rho[o] * dH(p, q) + drho[o] * H[o] * zn(p, q);
    };
    auto dE = [&](int p, int q) {
      const size_t o = idx(p, q);
      return (3.0 * eps[o] / H[o]) * dH(p, q) + eps[o] * (drho[o] / rho[o] - deta_rel[o]) * zn(p, q);
    };
    auto dF = [&](int f, int q) {
      const double d0 = dU(f, q);
      if (f == 0) return d0;
      const size_t o = idx(f, q);
      return d0 + 0.5 * (psia[o] * (d0 - dU(f - 1, q)) + psib[o] * (dU(f + 1, q) - d0));
    };
    const double dC = (dF(i, j) - dF(i - 1, j)) / h;
    const size_t o = idx(i, j);
    const double e = eps[o], p = P[o];
    const double ex1 = 0.5 * (e + eps[o + 1]), ex0 = 0.5 * (eps[o - 1] + e);
    const double ey1 = 0.5 * (e + eps[o + nx]), ey0 = 0.5 * (eps[o - nx] + e);
    const double dEc = dE(i, j);
    const double z0 = zn(i, j);
    const double dq = 0.5 * (dEc + dE(i + 1, j)) * (P[o + 1] - p) + ex1 * (zn(i + 1, j) - z0) -
                      0.5 * (dE(i - 1, j) + dEc) * (p - P[o - 1]) - ex0 * (z0 - zn(i - 1, j)) +
                      0.5 * (dEc + dE(i, j + 1)) * (P[o + nx] - p) + ey1 * (zn(i, j + 1) - z0) -
                      0.5 * (dE(i, j - 1) + dEc) * (p - P[o - nx]) - ey0 * (z0 - zn(i, j - 1));
    return dC - dq / (h * h);
  }
};

// exact x-line band: row (i, j), columns (i', j) with |i' - i| <= beta
__global__ void k_pt_jac_band(const PointInst* __restrict__ inst, PtRow c, const double* __restrict__ gtab64,
                              const double* __restrict__ R, const int* __restrict__ skip, int beta,
                              double* __restrict__ band, uint8_t* __restrict__ act, double* __restrict__ jh,
                              double* __restrict__ dg) {
  const int z = blockIdx.y;
  if (skip && skip[z]) return;
  const PointInst q = inst[z];
  const int nx = q.nx, ny = q.ny, NN = nx * ny, ni = nx - 2, n = ni * (ny - 2);
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  PtRow row = c;
  row.base = (size_t)z * NN;
  row.h = q.h;
  row.nx = nx;
  const int i = r % ni + 1, j = r / ni + 1;
  const double* T = gtab64 + (size_t)z * NN;
  const bool el = q.m.elastic != 0;
  auto column = [&](int ic) {  // dR_ij / dP_{ic, j}
    auto dH = [&](int p, int qq) {
      if (!el) return 0.0;
      const int a = p > ic ? p - ic : ic - p, b = qq > j ? qq - j : j - qq;
      return T[(size_t)b * nx + a];
    };
    auto zn = [&](int p, int qq) { return (p == ic && qq == j) ? 1.0 : 0.0; };
    return row.jv(i, j, dH, zn);
  };
  const int bw = 2 * beta + 1;
  double* out = band + ((size_t)z * n + r) * bw;
  // row scale d = max(|J_ii|, |J_i|_max / 10) over the band (as in line contact)
  double rmax = 0.0, jii = 0.0;
  for (int t = 0; t < bw; ++t) {
    const int ic = i - beta + t;
    double v = 0.0;
    if (ic >= 1 && ic <= nx - 2) v = column(ic);
    out[t] = v;
    rmax = fmax(rmax, fabs(v));
    if (t == beta) jii = v;
  }
  double d = fmax(fabs(jii), 0.1 * rmax);
  d = d > 0.0 ? d : 1.0;
  const size_t o = (size_t)z * NN + (size_t)j * nx + i;
  const bool a = c.P[o] <= R[o] / d;
  if (a)
    for (int t = 0; t < bw; ++t) out[t] = (t == beta ? 1.0 : 0.0);
  if (jh) {
    auto one = [&](int, int) { return 1.0; };
    auto zero = [&](int, int) { return 0.0; };
    jh[(size_t)z * n + r] = a ? 0.0 : row.jv(i, j, one, zero);
  }
  if (dg) dg[(size_t)z * n + r] = d;
  act[(size_t)z * n + r] = a ? 1 : 0;
}

// exact y-line band: system (z, i) (grid column i), row j - 1, columns (i, jc) with |jc - j| <= beta;
// rows the x-band kernel marked active become identity rows; scale != 0 divides the others by
// the row scale d of the x-band (the scaled Newton system of the Krylov solve)
__global__ void k_pt_jac_yband(const PointInst* __restrict__ inst, PtRow c, const double* __restrict__ gtab64,
                               const double* __restrict__ dg, const uint8_t* __restrict__ act,
                               const int* __restrict__ skip, int beta, int scale, double* __restrict__ band) {
  const int z = blockIdx.y;
  if (skip && skip[z]) return;
  const PointInst q = inst[z];
  const int nx = q.nx, ny = q.ny, NN = nx * ny, ni = nx - 2, nj = ny - 2, n = ni * nj;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  PtRow row = c;
  row.base = (size_t)z * NN;
  row.h = q.h;
  row.nx = nx;
  const int i = r % ni + 1, j = r / ni + 1;
  const double* T = gtab64 + (size_t)z * NN;
  const bool el = q.m.elastic != 0;
  const int bw = 2 * beta + 1;
  double* out = band + (((size_t)z * ni + (i - 1)) * nj + (j - 1)) * bw;
  const size_t o = (size_t)z * n + r;
  if (act[o]) {
    for (int t = 0; t < bw; ++t) out[t] = (t == beta ? 1.0 : 0.0);
    return;
  }
  const double rd = scale ? 1.0 / dg[o] : 1.0;
  for (int t = 0; t < bw; ++t) {
    const int jc = j - beta + t;
    double v = 0.0;
    if (jc >= 1 && jc <= ny - 2) {
      auto dH = [&](int p, int qq) {
        if (!el) return 0.0;
        const int a = p > i ? p - i : i - p, b = qq > jc ? qq - jc : jc - qq;
        return T[(size_t)b * nx + a];
      };
      auto zn = [&](int p, int qq) { return (p == i && qq == jc) ? 1.0 : 0.0; };
      v = row.jv(i, j, dH, zn) * rd;
    }
    out[t] = v;
  }
}

// (dR/dP) v + (dR/dH0) v_h0 at interior nodes (dH = K v + v_h0 precomputed), 0 on the boundary
__global__ void k_pt_jv_raw(const PointInst* __restrict__ inst, PtRow c, const double* __restrict__ dH,
                            const double* __restrict__ v, double* __restrict__ out) {
  const int z = blockIdx.y;
  const PointInst q = inst[z];
  const int nx = q.nx, ny = q.ny, NN = nx * ny;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NN) return;
  const int j = t / nx, i = t % nx;
  const size_t base = (size_t)z * NN;
  double r = 0.0;
  if (i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2) {
    PtRow row = c;
    row.base = base;
    row.h = q.h;
    row.nx = nx;
    auto fH = [&](int p, int qq) { return dH[base + (size_t)qq * nx + p]; };
    auto fz = [&](int p, int qq) { return v[base + (size_t)qq * nx + p]; };
    r = row.jv(i, j, fH, fz);
  }
  out[base + t] = r;
}

// ------------------------------------------------------------ grid sequence
// coarse values of a fine nodal array: dst[z][jc][ic] = src[z][jc*sy][ic*sx]
__global__ void k_pt_inject(const double* __restrict__ src, int nxf, int nyf, double* __restrict__ dst, int nxc,
                            int nyc) {
  const int z = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nxc * nyc) return;
  const int jc = t / nxc, ic = t % nxc;
  const int sx = (nxf - 1) / (nxc - 1), sy = (nyf - 1) / (nyc - 1);
  dst[(size_t)z * nxc * nyc + t] = src[(size_t)z * nxf * nyf + (size_t)(jc * sy) * nxf + ic * sx];
}

// bilinear prolongation of (P, H0) to the grid with halved spacing; instances whose
// coarse solve did not converge (cdone != 1) keep their fine start
__global__ void k_pt_prolong(const double* __restrict__ Pc, const double* __restrict__ H0c,
                             const int* __restrict__ cdone, int nxc, int nyc, double* __restrict__ Pf,
                             double* __restrict__ H0f) {
  const int z = blockIdx.y;
  if (cdone && cdone[z] != 1) return;
  const int nxf = 2 * nxc - 1, nyf = 2 * nyc - 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nxf * nyf) return;
  const int j = t / nxf, i = t % nxf;
  const double* pc = Pc + (size_t)z * nxc * nyc;
  const int ci = i >> 1, cj = j >> 1;
  const int ci1 = (i & 1) ? ci + 1 : ci, cj1 = (j & 1) ? cj + 1 : cj;
  const double v = 0.25 * (pc[(size_t)cj * nxc + ci] + pc[(size_t)cj * nxc + ci1] + pc[(size_t)cj1 * nxc + ci] +
                           pc[(size_t)cj1 * nxc + ci1]);
  Pf[(size_t)z * nxf * nyf + t] = v;
  if (t == 0) H0f[z] = H0c[z];
}

cudaError_t pt_inject(const PtCtx* fine, const double* src, PtCtx* coarse, double* dst) {
  const dim3 g((coarse->NN + 255) / 256, coarse->n_inst);
  k_pt_inject<<<g, 256, 0, coarse->st>>>(src, fine->nx, fine->ny, dst, coarse->nx, coarse->ny);
  note_launch();
  return cudaGetLastError();
}

cudaError_t pt_prolong(const PtCtx* coarse, PtCtx* fine) {
  const dim3 g((fine->NN + 255) / 256, fine->n_inst);
  k_pt_prolong<<<g, 256, 0, fine->st>>>(coarse->Pw, coarse->H0w, coarse->done, coarse->nx, coarse->ny, fine->Pw,
                                         fine->H0w);
  note_launch();
  return cudaGetLastError();
}

// --------------------------------------------------------------- host: setup
cudaError_t pt_alloc(PtCtx* c, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 16);
  if (e == cudaSuccess) c->allocs.push_back(*p);
  return e;
}

void pt_free(PtCtx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  if (c->gs0) cudaStreamDestroy(c->gs0);
  if (c->gs1) cudaStreamDestroy(c->gs1);
  if (c->gs2) cudaStreamDestroy(c->gs2);
  if (c->gev) cudaEventDestroy(c->gev);
  c->gs0 = c->gs1 = c->gs2 = nullptr;
  c->gev = nullptr;
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  pt_adj_free(c);
  if (c->blas) cublasDestroy(c->blas);
  c->blas = nullptr;
}

// leading dimension of a GEMM operand: a multiple of 8 floats
static size_t pt_ld8(size_t x) { return (x + 7) / 8 * 8; }

// T_all[i + (d nx + k) ldt] = T[d][|i - k|]  (column-major nx x (nx ny), float32, leading
// dimension ldt = nx rounded up to 8 floats: 32-byte aligned columns)
__global__ void k_pt_tall(const double* __restrict__ gtab64, float* __restrict__ Tall, int nx, int ny, int ldt) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)ldt * nx * ny;
  if (t >= total) return;
  const int i = (int)(t % ldt);
  const size_t col = t / ldt;
  const int d = (int)(col / nx), k = (int)(col % nx);
  Tall[t] = (i < nx) ? (float)gtab64[(size_t)d * nx + (i > k ? i - k : k - i)] : 0.f;
}

// Q[(d nx + k) + j ldq] = V[j][k] (d = 0) or V[j-d][k] + V[j+d][k] (rows outside the grid are 0);
// ldq = nx ny rounded up to 8 floats
__global__ void k_pt_qmat(const double* __restrict__ V, float* __restrict__ Q, int nx, int ny, int ldq) {
  const int z = blockIdx.y;
  const size_t NN = (size_t)nx * ny;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)ldq * ny) return;
  const int j = (int)(t / ldq);
  const size_t rem = t % ldq;
  float* Qz = Q + (size_t)z * ldq * ny;
  if (rem >= NN) {
    Qz[t] = 0.f;
    return;
  }
  const int d = (int)(rem / nx), k = (int)(rem % nx);
  const double* Vz = V + (size_t)z * NN;
  double s;
  if (d == 0) {
    s = Vz[(size_t)j * nx + k];
  } else {
    s = (j - d >= 0 ? Vz[(size_t)(j - d) * nx + k] : 0.0) + (j + d < ny ? Vz[(size_t)(j + d) * nx + k] : 0.0);
  }
  Qz[t] = (float)s;
}

static PtRow pt_row(PtCtx* c, const double* P) {
  PtRow r;
  r.P = P;
  r.H = c->H;
  r.rho = c->rho;
  r.drho = c->drho;
  r.deta_rel = c->deta_rel;
  r.eps = c->eps;
  r.psia = c->psia;
  r.psib = c->psib;
  r.base = 0;
  r.nx = c->nx;
  r.h = 0.0;
  return r;
}

__global__ void k_pt_unit_diagonal(double* __restrict__ band, size_t rows, int bw, int beta) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < rows) band[t * bw + beta] = 1.0;
}

ehl_status pt_init(PtCtx* c, const std::vector<PointInst>& insts, int beta, int max_iter, int krylov_dim,
                   int precision, int deform, int yline, int autotune) {
  const int ni = (int)insts.size();
  c->n_inst = ni;
  c->nx = insts[0].nx;
  c->ny = insts[0].ny;
  c->NN = c->nx * c->ny;
  c->n = (c->nx - 2) * (c->ny - 2);
  c->lines = ni * (c->ny - 2);
  c->beta = beta;
  c->max_iter = max_iter;
  c->m = krylov_dim;
  c->h_inst = insts;
  c->ksplit = (c->nx + kPtSK - 1) / kPtSK;
  c->nblk = (c->NN + kPtNode - 1) / kPtNode;
  const int n1 = c->n + 1;
  c->nvb = (n1 + kPtVB * kPtVPT - 1) / (kPtVB * kPtVPT);
  const size_t NNt = (size_t)ni * c->NN, nt = (size_t)ni * c->n, n1t = (size_t)ni * n1;
  const int bw = 2 * beta + 1, m = c->m;
  bool ok = true;
  auto A = [&](void** p, size_t bytes) {
    if (ok && pt_alloc(c, p, bytes) != cudaSuccess) ok = false;
  };
  A((void**)&c->inst, sizeof(PointInst) * ni);
  A((void**)&c->gtab, sizeof(float2) * NNt);
  A((void**)&c->gtab64, sizeof(double) * NNt);
  A(&c->partial, sizeof(double) * NNt * c->ksplit);
  double** nodal[] = {&c->H, &c->rho, &c->drho, &c->deta_rel, &c->eps, &c->u, &c->F, &c->psia, &c->psib,
                      &c->R, &c->Pw, &c->dH, &c->Pt, &c->znode};
  for (double** q : nodal) A((void**)q, sizeof(double) * NNt);
  A((void**)&c->blk, sizeof(double) * ni * c->nblk * 4);
  A((void**)&c->red, sizeof(double) * ni * 4);
  double** per[] = {&c->H0w, &c->best, &c->phinorm, &c->den, &c->H0t, &c->tstep, &c->rtol, &c->beta0, &c->zh0};
  for (double** q : per) A((void**)q, sizeof(double) * ni);
  int** iper[] = {&c->done, &c->iters, &c->stall, &c->gm_k, &c->gm_conv, &c->lsdone, &c->lsphase, &c->skip,
                  &c->acc};
  for (int** q : iper) A((void**)q, sizeof(int) * ni);
  A((void**)&c->band, sizeof(double) * nt * bw);
  A((void**)&c->act, nt);
  double** vec[] = {&c->jh, &c->dg, &c->rhs, &c->sigma, &c->zH};
  for (double** q : vec) A((void**)q, sizeof(double) * nt);
  A((void**)&c->V, sizeof(double) * n1t * (m + 1));
  A((void**)&c->Z, sizeof(double) * n1t * m);
  A((void**)&c->Hh, sizeof(double) * ni * (size_t)(m + 1) * m);
  A((void**)&c->cs, sizeof(double) * ni * (size_t)m);
  A((void**)&c->sn, sizeof(double) * ni * (size_t)m);
  A((void**)&c->g, sizeof(double) * ni * (size_t)(m + 1));
  A((void**)&c->w, sizeof(double) * n1t);
  A((void**)&c->delta, sizeof(double) * n1t);
  A((void**)&c->dots, sizeof(double) * ni * (size_t)c->nvb * (m + 2));
  A((void**)&c->hcol, sizeof(double) * ni * (size_t)(m + 2));
  A((void**)&c->pq_info, sizeof(int) * c->lines);
  A((void**)&c->loop, sizeof(int) * 8);
  A((void**)&c->jc, sizeof(double) * 4 * NNt);
  c->pq_r = 0;
  if (ok && autotune) {
    // the fastest partition count of the x-line systems (ny - 2 per instance, order nx - 2), timed
    // on identity bands in the context's band / rhs / sigma arrays (rewritten by every Newton step)
    const size_t rows = nt, bwz = (size_t)bw;
    cudaError_t e = cudaMemsetAsync(c->band, 0, sizeof(double) * rows * bwz, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->rhs, 0, sizeof(double) * rows, c->st);
    if (e == cudaSuccess) {
      k_pt_unit_diagonal<<<(unsigned)((rows + 255) / 256), 256, 0, c->st>>>(c->band, rows, bw, beta);
      note_launch();
      e = cudaGetLastError();
    }
    int r = 0;
    if (e == cudaSuccess &&
        ehl_paqif_autotune(c->lines, c->nx - 2, beta, 0, c->band, c->rhs, c->sigma, 3, c->st, &r, nullptr) == EHL_OK &&
        r > 0)
      c->pq_r = r;
    cudaGetLastError();
  }
  if (ok) {
    size_t wb = 0, wb2 = 0;
    ehl_paqif_workspace_size(c->lines, c->nx - 2, beta, 0, &wb);
    ehl_paqif_workspace_size_partitioned(c->lines, c->nx - 2, beta, c->pq_r, 0, &wb2);
    A(&c->pq_ws, wb > wb2 ? wb : wb2);
    A(&c->fstore, paqif_factor_store_bytes(c->lines, c->nx - 2, beta, c->pq_r));
  }
  if (ok && yline) {
    c->yline = 1;
    c->ylines = ni * (c->nx - 2);
    size_t wb = 0;
    ehl_paqif_workspace_size(c->ylines, c->ny - 2, beta, 0, &wb);
    A(&c->pq_ws_y, wb);
    A(&c->fstore_y, paqif_factor_store_bytes(c->ylines, c->ny - 2, beta));
    A((void**)&c->band_y, sizeof(double) * nt * bw);
    double** yv[] = {&c->rhs_y, &c->sig_y, &c->zHy};
    for (double** q : yv) A((void**)q, sizeof(double) * nt);
    double** yp[] = {&c->deny, &c->xiy};
    for (double** q : yp) A((void**)q, sizeof(double) * ni);
    A((void**)&c->pq_info_y, sizeof(int) * c->ylines);
  }
  if (!ok) {
    cudaGetLastError();
    return EHL_ENOMEM;
  }
  cudaError_t e = cudaMemcpyAsync(c->inst, insts.data(), sizeof(PointInst) * ni, cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess) {
    dim3 g((c->NN + 255) / 256, ni);
    k_pt_gtab<<<g, 256, 0, c->st>>>(c->inst, c->gtab, c->gtab64);
    note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && deform == 1 && insts[0].m.elastic) {
    void* mem = nullptr;
    if (pt_alloc(c, &mem, fft2_bytes(c->nx, c->ny, ni)) != cudaSuccess) {
      cudaGetLastError();
      return EHL_ENOMEM;
    }
    e = fft2_init(c->fft, c->nx, c->ny, ni, mem, c->gtab64, c->st);
    c->use_fft = e == cudaSuccess;
  }
  if (e == cudaSuccess && precision > 0 && insts[0].m.elastic && !c->use_fft) {
    const size_t ldt = pt_ld8(c->nx), ldq = pt_ld8((size_t)c->NN);
    const size_t tall = ldt * c->nx * c->ny, q = ldq * c->ny * ni, dn = ldt * c->ny * ni;
    if (pt_alloc(c, (void**)&c->Tall, sizeof(float) * tall) != cudaSuccess ||
        pt_alloc(c, (void**)&c->Qf, sizeof(float) * q) != cudaSuccess ||
        pt_alloc(c, (void**)&c->Df, sizeof(float) * dn) != cudaSuccess) {
      cudaGetLastError();
      return EHL_ENOMEM;
    }
    if (cublasCreate(&c->blas) != CUBLAS_STATUS_SUCCESS) return EHL_ECUDA;
    cublasSetStream(c->blas, c->st);
    if (precision == 2) cublasSetEmulationStrategy(c->blas, CUBLAS_EMULATION_STRATEGY_EAGER);
    k_pt_tall<<<(unsigned)((tall + 255) / 256), 256, 0, c->st>>>(c->gtab64, c->Tall, c->nx, c->ny, (int)ldt);
    note_launch();
    c->precision = precision;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return EHL_ECUDA;
  }
  return EHL_OK;
}

// D = K V into c->partial: `parts` partial sums, float64 (p64 = 1) or double-float (0)
static cudaError_t pt_deform(PtCtx* c, const double* V, const int* skip, bool f64, int& parts, int& p64,
                             bool direct = false) {
  if (c->use_fft && !direct) {
    parts = 1;
    p64 = 1;
    return fft2_conv(c->fft, V, skip, reinterpret_cast<double*>(c->partial), c->st);
  }
  parts = c->ksplit;
  p64 = f64 ? 1 : 0;
  dim3 g((c->nx + kPtTI - 1) / kPtTI, (c->ny + kPtTJ - 1) / kPtTJ, c->n_inst * c->ksplit);
  if (f64)
    k_pt_deform<true><<<g, kPtTI * kPtTJ, 0, c->st>>>(c->inst, c->gtab, c->gtab64, V, skip, c->partial, c->n_inst,
                                                      c->ksplit);
  else
    k_pt_deform<false><<<g, kPtTI * kPtTJ, 0, c->st>>>(c->inst, c->gtab, c->gtab64, V, skip, c->partial, c->n_inst,
                                                       c->ksplit);
  note_launch();
  return cudaGetLastError();
}

cudaError_t pt_state(PtCtx* c, const double* P, const double* H0, const double* rough, const int* skip) {
  int parts = 1, p64 = 1;
  cudaError_t e = pt_deform(c, P, skip, true, parts, p64);
  if (e != cudaSuccess) return e;
  const dim3 gn((c->NN + kPtNode - 1) / kPtNode, c->n_inst);
  k_pt_film<<<gn, kPtNode, 0, c->st>>>(c->inst, c->partial, parts, p64, H0, rough, skip, c->H, c->n_inst, 0);
  note_launch();
  k_pt_nodes<<<gn, kPtNode, 0, c->st>>>(c->inst, P, c->H, skip, c->rho, c->drho, c->deta_rel, c->eps, c->u);
  note_launch();
  k_pt_faces<<<gn, kPtNode, 0, c->st>>>(c->inst, c->u, skip, c->F, c->psia, c->psib);
  note_launch();
  k_pt_residual<<<gn, kPtNode, 0, c->st>>>(c->inst, P, c->H, c->eps, c->F, skip, c->R, c->blk, c->nblk);
  note_launch();
  return cudaGetLastError();
}

cudaError_t pt_finalize(PtCtx* c, int* done, int* iters) {
  k_pt_finalize<<<(c->n_inst + 127) / 128, 128, 0, c->st>>>(c->inst, c->blk, c->nblk, c->red, done, iters,
                                                             done ? c->best : nullptr, done ? c->stall : nullptr,
                                                             c->n_inst);
  note_launch();
  return cudaGetLastError();
}

cudaError_t pt_jac_band(PtCtx* c, const double* P, double* band, uint8_t* act, double* jh, double* dg,
                        const int* skip) {
  const dim3 g((c->n + 127) / 128, c->n_inst);
  k_pt_jac_band<<<g, 128, 0, c->st>>>(c->inst, pt_row(c, P), c->gtab64, c->R, skip, c->beta, band, act, jh, dg);
  note_launch();
  return cudaGetLastError();
}

cudaError_t pt_jac_yband(PtCtx* c, const double* P, const uint8_t* act, const double* dg, double* band, int scale,
                         const int* skip) {
  const dim3 g((c->n + 127) / 128, c->n_inst);
  k_pt_jac_yband<<<g, 128, 0, c->st>>>(c->inst, pt_row(c, P), c->gtab64, dg, act, skip, c->beta, scale, band);
  note_launch();
  return cudaGetLastError();
}

cudaError_t pt_start(PtCtx* c, double* P, double* H0, const double* rough) {
  const dim3 gn((c->NN + 255) / 256, c->n_inst);
  k_pt_hertz<<<gn, 256, 0, c->st>>>(c->inst, P);
  note_launch();
  cudaError_t e = cudaMemsetAsync(H0, 0, sizeof(double) * c->n_inst, c->st);
  if (e == cudaSuccess) e = pt_state(c, P, H0, rough, nullptr);
  if (e != cudaSuccess) return e;
  k_pt_set_h0<<<(c->n_inst + 127) / 128, 128, 0, c->st>>>(c->inst, c->blk, c->nblk, H0, c->n_inst);
  note_launch();
  return cudaGetLastError();
}

// The Krylov products with precision > 0: per instance one GEMM T_all [nx x nx ny] . Q [nx ny x ny]
// (precision 1 float32, 2 float32 with the BF16x9 emulation requested, 3 TF32, 4 BF16), float32
// output.  cuBLAS runs SIMT SGEMM kernels for precision 2 at these shapes (measured kernel names).
static cudaError_t pt_deform_gemm(PtCtx* c, const double* zn, const int* skip, const double* zh0) {
  const int ldt = (int)pt_ld8(c->nx), ldq = (int)pt_ld8((size_t)c->NN);
  const size_t qn = (size_t)ldq * c->ny;
  dim3 g((unsigned)((qn + 255) / 256), c->n_inst);
  k_pt_qmat<<<g, 256, 0, c->st>>>(zn, c->Qf, c->nx, c->ny, ldq);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cublasComputeType_t ct = CUBLAS_COMPUTE_32F;
  if (c->precision == 2) ct = CUBLAS_COMPUTE_32F_EMULATED_16BFX9;
  if (c->precision == 3) ct = CUBLAS_COMPUTE_32F_FAST_TF32;
  if (c->precision == 4) ct = CUBLAS_COMPUTE_32F_FAST_16BF;
  const float one = 1.0f, zero = 0.0f;
  const int m = c->nx, n = c->ny, k = c->nx * c->ny;
  if (cublasGemmStridedBatchedEx(c->blas, CUBLAS_OP_N, CUBLAS_OP_N, m, n, k, &one, c->Tall, CUDA_R_32F, ldt, 0,
                                 c->Qf, CUDA_R_32F, ldq, (long long)qn, &zero, c->Df, CUDA_R_32F, ldt,
                                 (long long)ldt * c->ny, c->n_inst, ct, CUBLAS_GEMM_DEFAULT) != CUBLAS_STATUS_SUCCESS)
    return cudaErrorUnknown;
  const dim3 gn((c->NN + kPtNode - 1) / kPtNode, c->n_inst);
  k_pt_film<<<gn, kPtNode, 0, c->st>>>(c->inst, c->Df, ldt, 2, zh0, nullptr, skip, c->dH, c->n_inst, 1);
  note_launch();
  return cudaGetLastError();
}

cudaError_t pt_deform_dir(PtCtx* c, const double* zn, const double* zh0, const int* skip) {
  if (c->precision > 0 && !c->use_fft) return pt_deform_gemm(c, zn, skip, zh0);
  int parts = 1, p64 = 0;
  cudaError_t e = pt_deform(c, zn, skip, false, parts, p64);
  if (e != cudaSuccess) return e;
  const dim3 gn((c->NN + kPtNode - 1) / kPtNode, c->n_inst);
  k_pt_film<<<gn, kPtNode, 0, c->st>>>(c->inst, c->partial, parts, p64, zh0, nullptr, skip, c->dH, c->n_inst, 1);
  note_launch();
  return cudaGetLastError();
}

cudaError_t pt_deform_dir64(PtCtx* c, const double* v, const int* skip) {
  int parts = 1, p64 = 1;
  cudaError_t e = pt_deform(c, v, skip, true, parts, p64, /*direct=*/true);
  if (e != cudaSuccess) return e;
  const dim3 gn((c->NN + kPtNode - 1) / kPtNode, c->n_inst);
  k_pt_film<<<gn, kPtNode, 0, c->st>>>(c->inst, c->partial, parts, p64, nullptr, nullptr, skip, c->dH, c->n_inst,
                                       1);
  note_launch();
  return cudaGetLastError();
}

cudaError_t pt_jacobian_apply(PtCtx* c, const double* P, const double* H0, const double* rough, const double* v,
                              const double* v_h0, double* out) {
  cudaError_t e = pt_state(c, P, H0, rough, nullptr);
  if (e == cudaSuccess) e = pt_deform_dir(c, v, v_h0, nullptr);
  if (e != cudaSuccess) return e;
  const dim3 gn((c->NN + kPtNode - 1) / kPtNode, c->n_inst);
  k_pt_jv_raw<<<gn, kPtNode, 0, c->st>>>(c->inst, pt_row(c, P), c->dH, v, out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace ehl
