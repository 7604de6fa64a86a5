// line_adjoint.cu -- sensitivities of a converged line-contact state.
//
// At a solution of the discrete problem (Sec. 3.3, Example 6: P >= 0,
// R >= 0, P R = 0 and h sum P = pi/2) the Newton-Krylov equations
//   Phi_i = P_i (rows with P_i <= R_i/d_i)  or  R_i/d_i (the others),
//   Phi_n = h sum P - pi/2,     d_i = max(|dR_i/dP_i|, max_{|j-i|<=beta} |dR_i/dP_j| / 10),
// define (P, H0) implicitly as functions of the roughness profile and the
// Moes parameters M, L.  For an objective J(P, H, H0):
//   Phi_x^T mu = dJ/dx,   dJ/dtheta = dJ/dtheta|_explicit - mu^T dPhi/dtheta.
// The transposed system is solved by restarted GMRES on the exact transposed
// operator, right-preconditioned by PAQIF on the transpose of the scaled
// exact band bordered with the force column h and the dR/dH0 row:
//   Phi_x^T (z, xi) = ( J^T w + z_I + h xi ,  c^T z ),  w = z / d on
// equation rows (0 elsewhere), c = (dR/dH0) / d on equation rows,
//   J^T w = g_P(w) - K g_H(w)
// where g_H, g_P are the transposed local stencil of the residual (the face
// fluxes and the Poiseuille term, through rho, eta, eps and the limiter on
// its current branch) and K the deformation matrix, symmetric, so that one
// deformation of g_H per product suffices.  The products are summed in
// float64: the residual the restarted GMRES can reach is the rounding of
// the transposed product times the conditioning of the system.
#include <cuda_runtime.h>
#include <math.h>

#include <vector>

#include "ehl_internal.h"
#include "line.h"

namespace ehl {

constexpr int kAdjBlock = 256;
constexpr int kAdjKrylov = 120;  // GMRES basis of the transposed solve (at most 200, see k_adj_update)

struct AdjBuf {
  int m = 0;
  double *V = nullptr, *Z = nullptr, *Hh = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr;
  double *w = nullptr, *mu = nullptr, *gx = nullptr, *res = nullptr, *zr = nullptr, *cb = nullptr;
  double *den = nullptr, *gxn = nullptr, *relres = nullptr, *bandT = nullptr, *hvec = nullptr;
  double *wn = nullptr, *gHn = nullptr, *gPn = nullptr;
  int *gm_k = nullptr, *gm_conv = nullptr, *done = nullptr, *skip = nullptr;
  void* fstore = nullptr;
};

// the block's total of v, to every thread: warp shuffles, then one value per warp in shared
// memory (two barriers; the leading one lets a previous call's readers finish)
__device__ __forceinline__ double adj_block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < kAdjBlock / 32; ++w) t += sh[w];
  return t;
}

// Node state the transposed stencil reads (from line_state).
struct AdjNodes {
  const double *P, *H, *rho, *drho, *deta_rel, *eps, *psia, *psib;
};

// Adjoints of the nodal perturbations dU = d(rho H), dE = d eps and of the
// pressure perturbation zn directly in the Poiseuille term, at node m, for
// row weights w (nodal, zero at the two boundary nodes):
//   sum_i w_i (dR_i) = sum_m aU_m dU_m + aE_m dE_m + aZ_m zn_m.
// Face f lies between nodes f and f+1 (f = 0..N-2); phi_f = (w_f - w_{f+1})/h
// weighs the flux F_{f+1/2}, chi_f = -phi_f/h the Poiseuille flux of face f.
__device__ __forceinline__ void adj_local(const AdjNodes& q, const double* __restrict__ wn, size_t base, int m, int N,
                                          double h, double& aU, double& aE, double& aZ) {
  auto W = [&](int j) { return (j >= 0 && j < N) ? wn[base + j] : 0.0; };
  auto phi = [&](int f) { return (f >= 0 && f <= N - 2) ? (W(f) - W(f + 1)) / h : 0.0; };
  auto pa = [&](int f) { return (f >= 0 && f <= N - 2) ? q.psia[base + f] : 0.0; };
  auto pb = [&](int f) { return (f >= 0 && f <= N - 2) ? q.psib[base + f] : 0.0; };
  const double fm = phi(m), fm1 = phi(m - 1), fp1 = phi(m + 1);
  // dF(f) = (1 + psia_f/2 - psib_f/2) dU_f - psia_f/2 dU_{f-1} + psib_f/2 dU_{f+1}
  aU = fm * (1.0 + 0.5 * pa(m) - 0.5 * pb(m)) - 0.5 * pa(m + 1) * fp1 + 0.5 * pb(m - 1) * fm1;
  // Q_f = (dE_f + dE_{f+1})/2 (P_{f+1} - P_f) + eps_{f+1/2} (zn_{f+1} - zn_f)
  const double cm = -fm / h, cm1 = -fm1 / h;
  const double dPm = (m <= N - 2) ? q.P[base + m + 1] - q.P[base + m] : 0.0;
  const double dPm1 = (m >= 1) ? q.P[base + m] - q.P[base + m - 1] : 0.0;
  aE = 0.5 * (cm * dPm + cm1 * dPm1);
  const double efm = (m <= N - 2) ? 0.5 * (q.eps[base + m] + q.eps[base + m + 1]) : 0.0;
  const double efm1 = (m >= 1) ? 0.5 * (q.eps[base + m - 1] + q.eps[base + m]) : 0.0;
  aZ = cm1 * efm1 - cm * efm;
}

// g_H (adjoint of the film) and g_P (direct adjoint of P) at every node for the weights wn
__global__ void k_adj_local(const LineInst* __restrict__ inst, AdjNodes q, const double* __restrict__ wn,
                            const int* __restrict__ skip, double* __restrict__ gHn, double* __restrict__ gPn, int N) {
  const int z = blockIdx.y;
  if (skip && skip[z]) return;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= N) return;
  const size_t base = (size_t)z * N, o = base + m;
  double aU, aE, aZ;
  adj_local(q, wn, base, m, N, inst[z].h, aU, aE, aZ);
  const double e = q.eps[o], H = q.H[o], r = q.rho[o];
  // dU = rho dH + rho' H zn,  dE = 3 eps/H dH + eps (rho'/rho - (ln eta)') zn
  gHn[o] = aU * r + aE * 3.0 * e / H;
  gPn[o] = aU * q.drho[o] * H + aE * e * (q.drho[o] / r - q.deta_rel[o]) + aZ;
}

// Scale the band rows of the equation rows by 1/d, border row c = (dR/dH0)/d, force column h.
__global__ void k_adj_prepare(const LineInst* __restrict__ inst, double* __restrict__ band,
                              const uint8_t* __restrict__ act, const double* __restrict__ jh,
                              const double* __restrict__ dg, double* __restrict__ cb, double* __restrict__ hvec,
                              int n, int bw) {
  const int z = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const size_t o = (size_t)z * n + r;
  if (!act[o]) {
    const double d = dg[o];
    double* row = band + o * bw;
    const double rd = 1.0 / d;  // one float64 division per row
    for (int j = 0; j < bw; ++j) row[j] *= rd;
    cb[o] = jh[o] / d;
  } else {
    cb[o] = 0.0;
  }
  hvec[o] = inst[z].h;
}

// bandT[r][j] = A^T(r, r - beta + j) = A(r - beta + j, r) = band[r - beta + j][2 beta - j]
__global__ void k_adj_transpose(const double* __restrict__ band, double* __restrict__ bandT, int n, int beta) {
  const int z = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int bw = 2 * beta + 1;
  const double* B = band + (size_t)z * n * bw;
  double* T = bandT + ((size_t)z * n + r) * bw;
  for (int j = 0; j < bw; ++j) {
    const int s = r - beta + j;
    T[j] = (s >= 0 && s < n) ? B[(size_t)s * bw + (2 * beta - j)] : 0.0;
  }
}

// Right-hand side dJ/dx: dJ/dP_int = gP - K gH (D = -K gH in dH), dJ/dH0 = gH0 + sum gH
__global__ void __launch_bounds__(kAdjBlock) k_adj_rhs(AdjBuf b, const double* __restrict__ gP,
                                                       const double* __restrict__ gH, const double* __restrict__ gH0,
                                                       const double* __restrict__ dH, int N) {
  const int z = blockIdx.x;
  __shared__ double sh[kAdjBlock];
  const int n = N - 2, n1 = n + 1;
  const size_t base = (size_t)z * N;
  double* gx = b.gx + (size_t)z * n1;
  double sH = 0.0, ss = 0.0;
  for (int j = threadIdx.x; j < N; j += kAdjBlock) {
    if (gH) sH += gH[base + j];
    if (j >= 1 && j <= N - 2) {
      const double v = (gP ? gP[base + j] : 0.0) + (gH ? dH[base + j] : 0.0);
      gx[j - 1] = v;
      ss += v * v;
    }
  }
  sH = adj_block_sum(sH, sh);
  ss = adj_block_sum(ss, sh);
  const double gn = (gH0 ? gH0[z] : 0.0) + sH;
  if (threadIdx.x == 0) {
    gx[n] = gn;
    b.gxn[z] = sqrt(ss + gn * gn);
  }
  __syncthreads();
  for (int r = threadIdx.x; r < n1; r += kAdjBlock) {
    b.mu[(size_t)z * n1 + r] = 0.0;
    b.res[(size_t)z * n1 + r] = gx[r];
  }
}

// den = c^T zr (zr = B^-T h)
__global__ void __launch_bounds__(kAdjBlock) k_adj_border(AdjBuf b, int n) {
  const int z = blockIdx.x;
  __shared__ double sh[kAdjBlock];
  double s = 0.0;
  for (int r = threadIdx.x; r < n; r += kAdjBlock) s += b.cb[(size_t)z * n + r] * b.zr[(size_t)z * n + r];
  s = adj_block_sum(s, sh);
  if (threadIdx.x == 0) b.den[z] = fabs(s) > 1e-300 ? s : 1e-300;
}

// start of a GMRES cycle from the residual: V_0 = res/|res|, PAQIF input V_0[0:n]
__global__ void __launch_bounds__(kAdjBlock) k_adj_start(AdjBuf b, double tol, double* __restrict__ rhs, int n) {
  const int z = blockIdx.x;
  if (b.done[z]) {
    if (threadIdx.x == 0) b.skip[z] = 1;
    return;
  }
  __shared__ double sh[kAdjBlock];
  const int n1 = n + 1;
  const double* res = b.res + (size_t)z * n1;
  double ss = 0.0;
  for (int r = threadIdx.x; r < n1; r += kAdjBlock) ss += res[r] * res[r];
  const double nrm = sqrt(adj_block_sum(ss, sh));
  double* v0 = b.V + (size_t)z * (b.m + 1) * n1;
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (int r = threadIdx.x; r < n1; r += kAdjBlock) {
    v0[r] = res[r] * inv;
    if (r < n) rhs[(size_t)z * n + r] = res[r] * inv;
  }
  if (threadIdx.x == 0) {
    b.g[(size_t)z * (b.m + 1)] = nrm;
    b.gm_k[z] = 0;
    b.gm_conv[z] = (nrm <= tol * b.gxn[z]) ? 1 : 0;
    b.skip[z] = b.gm_conv[z];
  }
}

// z = M^-T v:  z1 = B^-T v[0:n] (sigma),  xi = (c^T z1 - v[n]) / den,  z = (z1 - xi zr, xi);
// also the row weights wn = z/d on equation rows for the operator
__global__ void __launch_bounds__(kAdjBlock) k_adj_prec(AdjBuf b, int j, const double* __restrict__ sigma,
                                                        const uint8_t* __restrict__ act,
                                                        const double* __restrict__ dg, int N) {
  const int z = blockIdx.x;
  if (b.skip[z]) return;
  __shared__ double sh[kAdjBlock];
  const int n = N - 2, n1 = n + 1;
  double s = 0.0;
  for (int r = threadIdx.x; r < n; r += kAdjBlock) s += b.cb[(size_t)z * n + r] * sigma[(size_t)z * n + r];
  s = adj_block_sum(s, sh);
  const double* vj = b.V + ((size_t)z * (b.m + 1) + j) * n1;
  const double xi = (s - vj[n]) / b.den[z];
  double* Zj = b.Z + ((size_t)z * b.m + j) * n1;
  for (int r = threadIdx.x; r < n; r += kAdjBlock) {
    const size_t o = (size_t)z * n + r;
    const double v = sigma[o] - xi * b.zr[o];
    Zj[r] = v;
    b.wn[(size_t)z * N + r + 1] = act[o] ? 0.0 : v / dg[o];
  }
  if (threadIdx.x == 0) {
    Zj[n] = xi;
    b.wn[(size_t)z * N] = 0.0;
    b.wn[(size_t)z * N + N - 1] = 0.0;
  }
}

// wn = x/d on equation rows for a given vector x (n1 per instance)
__global__ void k_adj_weights(const double* __restrict__ x, const uint8_t* __restrict__ act,
                              const double* __restrict__ dg, const int* __restrict__ skip, double* __restrict__ wn,
                              int N) {
  const int z = blockIdx.y;
  if (skip && skip[z]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int n = N - 2;
  double v = 0.0;
  if (i >= 1 && i <= N - 2) {
    const size_t o = (size_t)z * n + (i - 1);
    v = act[o] ? 0.0 : x[(size_t)z * (n + 1) + (i - 1)] / dg[o];
  }
  wn[(size_t)z * N + i] = v;
}

// out = Phi_x^T x from g_P, D = -K g_H (in dH) and x itself
// (x of instance z at x + z * xstride)
__global__ void __launch_bounds__(kAdjBlock) k_adj_combine(const LineInst* __restrict__ inst, AdjBuf b,
                                                           const double* __restrict__ x, size_t xstride,
                                                           const double* __restrict__ dH,
                                                           const uint8_t* __restrict__ act,
                                                           const int* __restrict__ skip, double* __restrict__ out,
                                                           int N) {
  const int z = blockIdx.x;
  if (skip && skip[z]) return;
  __shared__ double sh[kAdjBlock];
  const int n = N - 2, n1 = n + 1;
  const double* xz = x + (size_t)z * xstride;
  double* oz = out + (size_t)z * n1;
  const double h = inst[z].h, xi = xz[n];
  double s = 0.0;
  for (int r = threadIdx.x; r < n; r += kAdjBlock) {
    const size_t o = (size_t)z * n + r;
    const size_t node = (size_t)z * N + r + 1;
    oz[r] = b.gPn[node] + dH[node] + (act[o] ? xz[r] : 0.0) + h * xi;
    s += b.cb[o] * xz[r];
  }
  s = adj_block_sum(s, sh);
  if (threadIdx.x == 0) oz[n] = s;
}

// Arnoldi step j (modified Gram-Schmidt), Givens rotations, convergence test;
// the next PAQIF input V_{j+1}[0:n]
__global__ void __launch_bounds__(kAdjBlock) k_adj_arnoldi(AdjBuf b, int j, double tol, double* __restrict__ rhs,
                                                           int n) {
  const int z = blockIdx.x;
  if (b.skip[z]) return;
  __shared__ double sh[kAdjBlock];
  const int n1 = n + 1, m = b.m;
  double* w = b.w + (size_t)z * n1;
  double* H = b.Hh + (size_t)z * (m + 1) * m;
  for (int i = 0; i <= j; ++i) {
    const double* Vi = b.V + ((size_t)z * (m + 1) + i) * n1;
    double d = 0.0;
    for (int r = threadIdx.x; r < n1; r += kAdjBlock) d += w[r] * Vi[r];
    d = adj_block_sum(d, sh);
    for (int r = threadIdx.x; r < n1; r += kAdjBlock) w[r] -= d * Vi[r];
    if (threadIdx.x == 0) H[i + (size_t)j * (m + 1)] = d;
    __syncthreads();
  }
  double nn = 0.0;
  for (int r = threadIdx.x; r < n1; r += kAdjBlock) nn += w[r] * w[r];
  nn = sqrt(adj_block_sum(nn, sh));
  double* Vn = b.V + ((size_t)z * (m + 1) + j + 1) * n1;
  const double inv = nn > 0.0 ? 1.0 / nn : 0.0;
  for (int r = threadIdx.x; r < n1; r += kAdjBlock) {
    const double v = w[r] * inv;
    Vn[r] = v;
    if (r < n) rhs[(size_t)z * n + r] = v;
  }
  if (threadIdx.x == 0) {
    H[j + 1 + (size_t)j * (m + 1)] = nn;
    double* cs = b.cs + (size_t)z * m;
    double* sn = b.sn + (size_t)z * m;
    double* g = b.g + (size_t)z * (m + 1);
    for (int i = 0; i < j; ++i) {
      const double a = H[i + (size_t)j * (m + 1)], c2 = H[i + 1 + (size_t)j * (m + 1)];
      H[i + (size_t)j * (m + 1)] = cs[i] * a + sn[i] * c2;
      H[i + 1 + (size_t)j * (m + 1)] = -sn[i] * a + cs[i] * c2;
    }
    const double a = H[j + (size_t)j * (m + 1)], c2 = H[j + 1 + (size_t)j * (m + 1)];
    const double rr = hypot(a, c2);
    const double c = rr > 0.0 ? a / rr : 1.0, s = rr > 0.0 ? c2 / rr : 0.0;
    cs[j] = c;
    sn[j] = s;
    H[j + (size_t)j * (m + 1)] = rr;
    H[j + 1 + (size_t)j * (m + 1)] = 0.0;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    b.gm_k[z] = j + 1;
    if (fabs(g[j + 1]) <= tol * b.gxn[z] || j + 1 == m || nn == 0.0) {
      b.gm_conv[z] = 1;
      b.skip[z] = 1;
    }
  }
}

// mu += sum_q y_q Z_q with y = R^-1 g over the cycle's k steps
__global__ void __launch_bounds__(kAdjBlock) k_adj_update(AdjBuf b, int n) {
  const int z = blockIdx.x;
  if (b.done[z]) return;
  const int n1 = n + 1, m = b.m, k = b.gm_k[z];
  __shared__ double y[256];
  if (threadIdx.x == 0) {
    const double* H = b.Hh + (size_t)z * (m + 1) * m;
    const double* g = b.g + (size_t)z * (m + 1);
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int q = i + 1; q < k; ++q) s -= H[i + (size_t)q * (m + 1)] * y[q];
      const double dgl = H[i + (size_t)i * (m + 1)];
      y[i] = dgl != 0.0 ? s / dgl : 0.0;
    }
  }
  __syncthreads();
  double* mu = b.mu + (size_t)z * n1;
  for (int r = threadIdx.x; r < n1; r += kAdjBlock) {
    double s = 0.0;
    for (int q = 0; q < k; ++q) s += y[q] * b.Z[((size_t)z * m + q) * n1 + r];
    mu[r] += s;
  }
}

// res = gx - Phi_x^T mu (in w); relative residual and the done flag
__global__ void __launch_bounds__(kAdjBlock) k_adj_residual(AdjBuf b, double tol, int n) {
  const int z = blockIdx.x;
  if (b.done[z]) return;
  __shared__ double sh[kAdjBlock];
  const int n1 = n + 1;
  double ss = 0.0;
  for (int r = threadIdx.x; r < n1; r += kAdjBlock) {
    const size_t o = (size_t)z * n1 + r;
    const double v = b.gx[o] - b.w[o];
    b.res[o] = v;
    ss += v * v;
  }
  ss = adj_block_sum(ss, sh);
  if (threadIdx.x == 0) {
    const double gn = b.gxn[z];
    const double rel = gn > 0.0 ? sqrt(ss) / gn : 0.0;
    b.relres[z] = rel;
    if (!(rel > tol)) b.done[z] = 1;  // also stops a NaN
  }
}

// gradients from lambda = mu/d (in wn, with g_H(lambda) in gHn):
//   rough_m = gH_m - g_H(lambda)_m;  (M, L) = -sum_m aU_m dU_theta(m) + aE_m dE_theta(m)
__global__ void __launch_bounds__(kAdjBlock) k_adj_grad(const LineInst* __restrict__ inst, AdjNodes q, AdjBuf b,
                                                        const double* __restrict__ gH, double* __restrict__ grad_rough,
                                                        double* __restrict__ grad_ML, int N) {
  const int z = blockIdx.x;
  __shared__ double sh[kAdjBlock];
  const LineInst qi = inst[z];
  const size_t base = (size_t)z * N;
  // d ln(lambda)/dM = -2/M;  d ln(pH)/dM = 1/(2M), d ln(pH)/dL = 1/L;  rho, eta depend on P pH
  const double lpM = 0.5 / qi.M, lpL = 1.0 / qi.L, llM = -2.0 / qi.M;
  double sM = 0.0, sL = 0.0;
  for (int m = threadIdx.x; m < N; m += kAdjBlock) {
    const size_t o = base + m;
    double aU, aE, aZ;
    adj_local(q, b.wn, base, m, N, qi.h, aU, aE, aZ);
    const double P = q.P[o], H = q.H[o], r = q.rho[o], dr = q.drho[o], e = q.eps[o], de = q.deta_rel[o];
    const double drl = dr * P;   // d rho / d ln pH
    const double del = de * P;   // d ln eta / d ln pH
    // dU = H d rho;  dE = eps (d rho/rho - d ln eta - d ln lambda)
    sM += aU * H * drl * lpM + aE * e * ((drl / r - del) * lpM - llM);
    sL += aU * H * drl * lpL + aE * e * ((drl / r - del) * lpL);
    if (grad_rough) grad_rough[o] = (gH ? gH[o] : 0.0) - b.gHn[o];
  }
  sM = adj_block_sum(sM, sh);
  sL = adj_block_sum(sL, sh);
  if (grad_ML && threadIdx.x == 0) {
    grad_ML[2 * z] = -sM;
    grad_ML[2 * z + 1] = -sL;
  }
}

// ----------------------------------------------------------------- host side
void line_adj_free(LineCtx* c) {
  delete (AdjBuf*)c->adj;
  c->adj = nullptr;
}

static cudaError_t adj_alloc(LineCtx* c) {
  AdjBuf* b = new AdjBuf();
  c->adj = b;
  // a wider basis than the Newton steps use: the transposed solve runs to a
  // tight tolerance, and restarts with a short basis stagnate near contact
  const int m = c->krylov_dim > kAdjKrylov ? c->krylov_dim : kAdjKrylov;
  const int n = c->n, n1 = n + 1, ni = c->n_inst, N = c->N;
  b->m = m;
  const size_t bw = 2 * c->beta + 1;
  struct A {
    void** p;
    size_t bytes;
  } al[] = {{(void**)&b->V, sizeof(double) * ni * (m + 1) * (size_t)n1},
            {(void**)&b->Z, sizeof(double) * ni * (size_t)m * n1},
            {(void**)&b->Hh, sizeof(double) * ni * (m + 1) * (size_t)m},
            {(void**)&b->cs, sizeof(double) * ni * (size_t)m},
            {(void**)&b->sn, sizeof(double) * ni * (size_t)m},
            {(void**)&b->g, sizeof(double) * ni * (size_t)(m + 1)},
            {(void**)&b->w, sizeof(double) * ni * (size_t)n1},
            {(void**)&b->mu, sizeof(double) * ni * (size_t)n1},
            {(void**)&b->gx, sizeof(double) * ni * (size_t)n1},
            {(void**)&b->res, sizeof(double) * ni * (size_t)n1},
            {(void**)&b->zr, sizeof(double) * ni * (size_t)n},
            {(void**)&b->cb, sizeof(double) * ni * (size_t)n},
            {(void**)&b->hvec, sizeof(double) * ni * (size_t)n},
            {(void**)&b->den, sizeof(double) * ni},
            {(void**)&b->gxn, sizeof(double) * ni},
            {(void**)&b->relres, sizeof(double) * ni},
            {(void**)&b->bandT, sizeof(double) * ni * (size_t)n * bw},
            {(void**)&b->wn, sizeof(double) * ni * (size_t)N},
            {(void**)&b->gHn, sizeof(double) * ni * (size_t)N},
            {(void**)&b->gPn, sizeof(double) * ni * (size_t)N},
            {(void**)&b->gm_k, sizeof(int) * ni},
            {(void**)&b->gm_conv, sizeof(int) * ni},
            {(void**)&b->done, sizeof(int) * ni},
            {(void**)&b->skip, sizeof(int) * ni},
            {(void**)&b->fstore, paqif_factor_store_bytes(ni, n, c->beta)}};
  for (auto& x : al) {
    cudaError_t e = ctx_alloc(c, x.p, x.bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static cudaError_t adj_paqif(LineCtx* c, AdjBuf& b, const double* rhs, double* x, bool factor) {
  PaqifLaunch L;
  L.n_sys = c->n_inst;
  L.n = c->n;
  L.beta = c->beta;
  L.mode = 0;
  L.band = b.bandT;
  L.rhs = rhs;
  L.act = nullptr;
  L.stack = c->pq_ws;
  L.x = x;
  L.iters = nullptr;
  L.info = c->pq_info;
  return factor ? launch_paqif_factor(L, b.fstore, c->st) : launch_paqif_resolve(L, b.fstore, c->st);
}

// out = Phi_x^T x (x of instance z at x + z * xstride), with the row weights of x already in b.wn
static cudaError_t adj_apply(LineCtx* c, AdjBuf& b, const AdjNodes& q, const double* x, size_t xstride, double* out,
                             const int* skip) {
  const dim3 gn((c->N + 255) / 256, c->n_inst);
  k_adj_local<<<gn, 256, 0, c->st>>>(c->inst, q, b.wn, skip, b.gHn, b.gPn, c->N);
  note_launch();
  cudaError_t e = line_deform64(c, b.gHn, c->N, skip);
  if (e == cudaSuccess) e = line_film_dir(c, nullptr, skip, true);  // dH = -K gH
  if (e != cudaSuccess) return e;
  k_adj_combine<<<c->n_inst, kAdjBlock, 0, c->st>>>(c->inst, b, x, xstride, c->dH, c->act, skip, out, c->N);
  note_launch();
  return cudaGetLastError();
}

static bool adj_all(LineCtx* c, const int* flags, cudaError_t& e) {
  std::vector<int> h(c->n_inst);
  e = cudaMemcpyAsync(h.data(), flags, sizeof(int) * c->n_inst, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  for (int v : h)
    if (!v) return false;
  return true;
}

cudaError_t line_adjoint(LineCtx* c, const double* P, const double* H0, const double* rough, const double* gP,
                         const double* gH, const double* gH0, double* grad_rough, double* grad_ML, double* relres,
                         double tol, int max_cycles, int* cycles) {
  if (!c->adj) {
    cudaError_t e = adj_alloc(c);
    if (e != cudaSuccess) return e;
  }
  AdjBuf& b = *(AdjBuf*)c->adj;
  const int ni = c->n_inst, N = c->N, n = c->n, bw = 2 * c->beta + 1;
  cudaError_t e = line_state(c, P, H0, rough, nullptr, nullptr);
  if (e == cudaSuccess) e = line_jac_band(c, P, 1, c->band, c->act, c->jh, c->dg, nullptr);
  if (e != cudaSuccess) return e;
  const AdjNodes q{P, c->H, c->rho, c->drho, c->deta_rel, c->eps, c->psia, c->psib};
  const dim3 gr((n + 127) / 128, ni);
  k_adj_prepare<<<gr, 128, 0, c->st>>>(c->inst, c->band, c->act, c->jh, c->dg, b.cb, b.hvec, n, bw);
  note_launch();
  k_adj_transpose<<<gr, 128, 0, c->st>>>(c->band, b.bandT, n, c->beta);
  note_launch();
  if (gH) {
    e = line_deform64(c, gH, N, nullptr);
    if (e == cudaSuccess) e = line_film_dir(c, nullptr, nullptr, true);
    if (e != cudaSuccess) return e;
  }
  k_adj_rhs<<<ni, kAdjBlock, 0, c->st>>>(b, gP, gH, gH0, c->dH, N);
  note_launch();
  e = adj_paqif(c, b, b.hvec, b.zr, true);  // factor B^T, zr = B^-T h
  if (e != cudaSuccess) return e;
  k_adj_border<<<ni, kAdjBlock, 0, c->st>>>(b, n);
  note_launch();
  e = cudaMemsetAsync(b.done, 0, sizeof(int) * ni, c->st);
  if (e != cudaSuccess) return e;
  int cyc = 0;
  for (; cyc < max_cycles; ++cyc) {
    k_adj_start<<<ni, kAdjBlock, 0, c->st>>>(b, 0.1 * tol, c->rhs, n);
    note_launch();
    for (int j = 0; j < b.m; ++j) {
      e = adj_paqif(c, b, c->rhs, c->sigma, false);
      if (e != cudaSuccess) return e;
      k_adj_prec<<<ni, kAdjBlock, 0, c->st>>>(b, j, c->sigma, c->act, c->dg, N);
      note_launch();
      // w = Phi_x^T Z_j (Z is [inst][m][n1])
      e = adj_apply(c, b, q, b.Z + (size_t)j * (n + 1), (size_t)b.m * (n + 1), b.w, b.skip);
      if (e != cudaSuccess) return e;
      k_adj_arnoldi<<<ni, kAdjBlock, 0, c->st>>>(b, j, 0.1 * tol, c->rhs, n);
      note_launch();
      if ((j + 1) % 8 == 0 && j + 1 < b.m) {
        if (adj_all(c, b.skip, e)) break;
        if (e != cudaSuccess) return e;
      }
    }
    k_adj_update<<<ni, kAdjBlock, 0, c->st>>>(b, n);
    note_launch();
    // true residual of the transposed system at mu
    const dim3 gn((N + 255) / 256, ni);
    k_adj_weights<<<gn, 256, 0, c->st>>>(b.mu, c->act, c->dg, b.done, b.wn, N);
    note_launch();
    e = adj_apply(c, b, q, b.mu, (size_t)(n + 1), b.w, b.done);
    if (e != cudaSuccess) return e;
    k_adj_residual<<<ni, kAdjBlock, 0, c->st>>>(b, tol, n);
    note_launch();
    if (adj_all(c, b.done, e)) {
      ++cyc;
      break;
    }
    if (e != cudaSuccess) return e;
  }
  // lambda = mu/d on the equation rows; g_H(lambda); gradients
  const dim3 gn((N + 255) / 256, ni);
  k_adj_weights<<<gn, 256, 0, c->st>>>(b.mu, c->act, c->dg, nullptr, b.wn, N);
  note_launch();
  k_adj_local<<<gn, 256, 0, c->st>>>(c->inst, q, b.wn, nullptr, b.gHn, b.gPn, N);
  note_launch();
  k_adj_grad<<<ni, kAdjBlock, 0, c->st>>>(c->inst, q, b, gH, grad_rough, grad_ML, N);
  note_launch();
  if (relres) {
    e = cudaMemcpyAsync(relres, b.relres, sizeof(double) * ni, cudaMemcpyDeviceToDevice, c->st);
    if (e != cudaSuccess) return e;
  }
  if (cycles) *cycles = cyc;
  return cudaGetLastError();
}

}  // namespace ehl
