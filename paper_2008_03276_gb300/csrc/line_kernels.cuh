// line_kernels.cuh -- device code of the line-contact hot path (Sec. 3.3).
//
// Discrete problem: nodes X_i = xa + i h, i = 0..N-1, P_0 = P_{N-1} = 0.
//  * film (Sec. 3.3.1 Case 1, Eq. eqn19):  H_i = H0 + X_i^2/2 - sum_k K_{|i-k|} P_k + rough_i,
//    K_d = G_d / pi with the closed-form cell integral G_d of log|x - x'|;
//  * lubricant (Sec. 3.3, Example 6): Roelands eta, Dowson-Higginson rho, eps = rho H^3/(eta lambda);
//  * TVD residual (Sec. 3.3.3, Eqs. eqn62-eqn65 in the standard upwind form):
//    F_{j+1/2} = u_j + psi(u_j - u_{j-1}, u_{j+1} - u_j)/2 (F_{1/2} = u_0), u = rho H, psi a
//    limiter (minmod, van Leer) or the linear kappa-scheme (Sec. 3.1, Eq. eqn41),
//    R_i = (F_{i+1/2} - F_{i-1/2})/h - [eps_{i+1/2}(P_{i+1}-P_i) - eps_{i-1/2}(P_i-P_{i-1})]/h^2.
#pragma once
#include <cuda_runtime.h>

#include "df64.cuh"

namespace ehl {

struct LineInst {
  int N;             // nodes including the two boundary nodes
  int beta;          // half-band of the Jacobian
  int limiter;       // 0 minmod, 1 van Leer, 2 the unlimited kappa-scheme
  int compressible;  // 0: rho = eta = 1
  int elastic;       // 0: rigid surfaces
  int splitting;     // kind-0 Couette part: 0 frozen limiter, 1 L_hs1, 2 L_hs2
  double xa, h;
  double lam, abar, alpha, p0, z, pH;
  double switch_eps_h, dist_w, c_h0, omega, tol, h_init;
  double M, L;       // Moes parameters (lam = 3 pi^2/(8 M^2), pH = L sqrt(M/(2 pi))/alpha)
  double kappa;      // kappa of limiter 2
};

// Coefficient c of the upwind Couette difference in the kind-0 Newton matrix of the hybrid
// splittings (Sec. 3.3.2, Eqs. eqn57, eqn59): L_hs1 keeps (2 - kappa)/2 of the kappa-scheme's
// first-order part, L_hs2 adds the (1 - kappa)/4 it moves over from the upwind node; 0 selects
// the frozen limiter factor of Sec. 3.3.3.
__host__ __device__ __forceinline__ double line_split_coef(const LineInst& q) {
  if (q.splitting == 1) return (2.0 - q.kappa) / 2.0;
  if (q.splitting == 2) return (2.0 - q.kappa) / 2.0 + (1.0 - q.kappa) / 4.0;
  return 0.0;
}

// rho, d rho/dP, ln eta and (d eta/dP)/eta at pressure P (float64).
__device__ __forceinline__ void line_material(const LineInst& q, double P, double& rho, double& drho,
                                              double& lneta, double& deta_rel) {
  if (!q.compressible) {
    rho = 1.0;
    drho = 0.0;
    lneta = 0.0;
    deta_rel = 0.0;
    return;
  }
  const double base = 1.0 + P * q.pH / q.p0;
  const double bz = pow(base, q.z);
  lneta = (q.alpha * q.p0 / q.z) * (bz - 1.0);
  deta_rel = q.alpha * q.pH * bz / base;
  const double a = 0.59e9;
  const double den = a + P * q.pH;
  rho = (a + 1.34 * P * q.pH) / den;
  drho = a * (1.34 * q.pH - q.pH) / (den * den);
}

// Limiter function psi(a, b) and its partial derivatives on the current branch; kind 2 is the
// unlimited kappa-scheme (Eq. eqn41: F = u_i + (1-kappa)/4 a + (1+kappa)/4 b), linear in a, b.
__device__ __forceinline__ void line_limiter(int kind, double kappa, double a, double b, double& psi, double& pa,
                                             double& pb) {
  if (kind == 2) {
    pa = 0.5 * (1.0 - kappa);
    pb = 0.5 * (1.0 + kappa);
    psi = pa * a + pb * b;
    return;
  }
  if (!(a * b > 0.0)) {
    psi = pa = pb = 0.0;
    return;
  }
  if (kind == 0) {
    if (fabs(a) <= fabs(b)) {
      psi = a;
      pa = 1.0;
      pb = 0.0;
    } else {
      psi = b;
      pa = 0.0;
      pb = 1.0;
    }
  } else {
    const double s = a + b;
    psi = 2.0 * a * b / s;
    pa = 2.0 * b * b / (s * s);
    pb = 2.0 * a * a / (s * s);
  }
}

// Film H_i = H0 + X_i^2/2 - D_i at node i (the roughness is added by the caller).
__device__ __forceinline__ double line_film_h(const LineInst& q, int i, double H0, double D) {
  const double X = q.xa + i * q.h;
  return H0 + 0.5 * X * X - D;
}

// rho, eps, u and the material derivatives of node o from P[o] and H[o] (float64).
// (No restrict qualifiers: a fused kernel reads back what its other threads wrote.)
__device__ __forceinline__ void line_node(const LineInst& q, size_t o, const double* P, const double* H, double* rho,
                                          double* drho, double* deta_rel, double* eps, double* u) {
  double r, dr, ln_eta, de;
  line_material(q, P[o], r, dr, ln_eta, de);
  const double Hh = H[o];
  rho[o] = r;
  drho[o] = dr;
  deta_rel[o] = de;
  eps[o] = r * Hh * Hh * Hh / q.lam * exp(-ln_eta);
  u[o] = r * Hh;
}

// One chunk k0 .. k0 + kmax - 1 of the deformation sum of node i in double-float,
// sum_k K_{|i-k|} V_k, accumulated in order by the Ogita-Rump-Oishi Dot2 scheme (error-free
// products and sums, the errors summed in float32) and normalised to (hi, lo).
__device__ __forceinline__ float2 line_deform_chunk(const float2* __restrict__ gtab, const double* __restrict__ V,
                                                    int i, int k0, int kmax) {
  float s = 0.f, c = 0.f;
  for (int k = 0; k < kmax; ++k) {
    int d = i - (k0 + k);
    d = d < 0 ? -d : d;
    const float2 g = gtab[d];
    const df vd = df_from_double(V[k0 + k]);
    const float p = __fmul_rn(g.x, vd.hi);
    float e = __fmaf_rn(g.x, vd.hi, -p);
    e = __fmaf_rn(g.x, vd.lo, e);
    e = __fmaf_rn(g.y, vd.hi, e);
    float t1, t2;
    two_sum(s, p, t1, t2);
    s = t1;
    c = __fadd_rn(c, __fadd_rn(t2, e));
  }
  float hi, lo;
  fast_two_sum(s, c, hi, lo);
  return make_float2(hi, lo);
}

// Cell integral of log|x_i - x'| over a cell at distance d (in cells), float64.
__device__ __forceinline__ double line_cell_integral(int d, double h) {
  const double tp = (d + 0.5) * h, tm = (d - 0.5) * h;
  return tp * (log(fabs(tp)) - 1.0) - tm * (log(fabs(tm)) - 1.0);
}

}  // namespace ehl
