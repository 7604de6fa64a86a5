// line_newton.cu -- Newton-Krylov method for line contact (ehl_params.method = 1).
//
// The fixed point is the paper's discrete problem (Sec. 3.3, Example 6): the
// TVD residual R with P >= 0, R >= 0, P R = 0 and the force balance.  The
// paper's banded Newton relaxation (method 0) diverges at high loads; this
// method keeps its three hot-path parts -- the TVD residual, the deformation
// integral and PAQIF on a band Jacobian -- and uses them in an inexact
// semismooth Newton iteration:
//   Phi_i = min(P_i, R_i / d_i)   (a row scaling: d_i = |dR_i/dP_i|, floored at a
//                                   tenth of the largest band entry of the row),
//   Phi_n = h sum P - pi/2,
// each step solving J_Phi dz = -Phi by GMRES on the exact Jacobian (J v from
// one deformation of v and a local directional derivative), right-
// preconditioned by PAQIF on the band of the scaled exact Jacobian bordered
// with the dR/dH0 column and the force row (one extra PAQIF solve per step
// for the border), followed by a backtracking line search on ||Phi||_2.
#include <cuda_runtime.h>
#include <stdio.h>
#include <math.h>

#include <vector>

#include "ehl_internal.h"
#include "line.h"
#include "graph_loop.h"

namespace ehl {

constexpr int kNkBlock = 256;
constexpr int kLoopSlots = 8;  // NkBuf::loop: newton, krylov, trial, krylov total, trial total

struct NkBuf {
  int m = 0, n1 = 0;
  double *V = nullptr, *Z = nullptr, *Hh = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr;
  double *phi = nullptr, *phinorm = nullptr, *zH = nullptr, *den = nullptr, *delta = nullptr;
  double *Pt = nullptr, *H0t = nullptr, *tstep = nullptr, *rtol = nullptr, *beta0 = nullptr;
  double *znode = nullptr, *zh0 = nullptr, *w = nullptr;
  double* jc = nullptr;  // per node, fixed for a Newton step: drho H, 3 eps/H, eps (drho/rho - deta), 1/d
  int *gm_k = nullptr, *gm_conv = nullptr, *lsdone = nullptr, *skip = nullptr;
  int* lsphase = nullptr;  // line search: 0 projected trials (P_t >= 0), 1 unprojected
  void* fstore = nullptr;  // PAQIF factor store of the current preconditioner
  // device-driven solve: loop counters (Newton step, Krylov index, line-search trial) and the
  // totals of Krylov iterations and trials over the solve
  int* loop = nullptr;
};

// the block's total of v, to every thread: warp shuffles, then one value per warp in shared
// memory (two barriers; the leading one lets a previous call's readers finish)
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < kNkBlock / 32; ++w) t += sh[w];
  return t;
}

// skip[z] = done[z] | other[z]
__global__ void k_nk_skip(const int* __restrict__ done, const int* __restrict__ other, int* __restrict__ skip,
                          int n_inst) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z < n_inst) skip[z] = (done[z] != 0) || (other && other[z] != 0);
}

// Scale the exact band rows by 1/d, form Phi, v_0 = -Phi/||Phi||, the border rhs.
__global__ void __launch_bounds__(kNkBlock) k_nk_setup(const LineInst* __restrict__ inst, NkBuf b,
                                                       const double* __restrict__ P, const double* __restrict__ R,
                                                       const double* __restrict__ red, const uint8_t* __restrict__ act,
                                                       const double* __restrict__ dg, const double* __restrict__ jh,
                                                       const int* __restrict__ done, double* __restrict__ band,
                                                       double* __restrict__ rhs, int N, int beta) {
  const int z = blockIdx.x;
  if (done[z]) return;
  __shared__ double sh[kNkBlock];
  const int n = N - 2, n1 = n + 1, bw = 2 * beta + 1;
  double* phi = b.phi + (size_t)z * n1;
  double ss = 0.0;
  for (int r = threadIdx.x; r < n; r += kNkBlock) {
    const size_t o = (size_t)z * n + r;
    const double d = dg[o];
    const double Pi = P[(size_t)z * N + r + 1], Ri = R[(size_t)z * N + r + 1];
    double ph;
    if (act[o]) {
      ph = Pi;
      rhs[o] = 0.0;
    } else {
      ph = Ri / d;  // as in k_nk_merit, so the line search compares like with like
      // the preconditioner's band: one division per row, not per entry (FP64 runs at 1/64 rate)
      const double rd = 1.0 / d;
      double* row = band + o * bw;
      for (int j = 0; j < bw; ++j) row[j] *= rd;
      rhs[o] = jh[o] / d;
    }
    phi[r] = ph;
    ss += ph * ph;
  }
  const double f = red[z * 4 + 1];
  if (threadIdx.x == 0) phi[n] = f;
  ss = block_sum(ss, sh) + f * f;
  const double nrm = sqrt(ss);
  double* v0 = b.V + (size_t)z * (b.m + 1) * n1;
  const double rn = nrm > 0.0 ? -1.0 / nrm : 0.0;
  for (int r = threadIdx.x; r < n1; r += kNkBlock) v0[r] = phi[r] * rn;
  if (threadIdx.x == 0) {
    b.phinorm[z] = nrm;
    b.beta0[z] = nrm;
    b.g[(size_t)z * (b.m + 1)] = nrm;
    b.gm_k[z] = 0;
    b.gm_conv[z] = nrm > 0.0 ? 0 : 1;
    const double rc = red[z * 4 + 0];
    b.rtol[z] = fmin(1e-3, fmax(1e-6, 1e-2 * rc));
  }
}

// zH = sigma (the PAQIF solve of the border column), den = h sum zH
__global__ void __launch_bounds__(kNkBlock) k_nk_border(const LineInst* __restrict__ inst, NkBuf b,
                                                        const double* __restrict__ sigma,
                                                        const int* __restrict__ done, double* __restrict__ rhs,
                                                        int N) {
  const int z = blockIdx.x;
  if (done[z]) return;
  __shared__ double sh[kNkBlock];
  const int n = N - 2, n1 = n + 1;
  double s = 0.0;
  for (int r = threadIdx.x; r < n; r += kNkBlock) {
    const double v = sigma[(size_t)z * n + r];
    b.zH[(size_t)z * n + r] = v;
    s += v;
  }
  s = block_sum(s, sh) * inst[z].h;
  if (threadIdx.x == 0) b.den[z] = fabs(s) > 1e-300 ? s : 1e-300;
  // the first preconditioner input: v_0[0:n]
  const double* v0 = b.V + (size_t)z * (b.m + 1) * n1;
  for (int r = threadIdx.x; r < n; r += kNkBlock) rhs[(size_t)z * n + r] = v0[r];
}

// z_j = M^-1 v_j from z1 = Jb^-1 v_j[0:n]: xi = (h sum z1 - v_j[n]) / den, z = z1 - xi zH
// (jd != null: the Krylov index is read from device memory, the loop counter of a device-driven solve)
__device__ __forceinline__ void nk_prec(const LineInst* inst, const NkBuf& b, int j, const double* sigma, int N, int z,
                                        double* sh) {
  const int n = N - 2, n1 = n + 1;
  double s = 0.0;
  for (int r = threadIdx.x; r < n; r += kNkBlock) s += sigma[(size_t)z * n + r];
  s = block_sum(s, sh) * inst[z].h;
  const double* vj = b.V + ((size_t)z * (b.m + 1) + j) * n1;
  const double xi = (s - vj[n]) / b.den[z];
  double* Zj = b.Z + ((size_t)z * b.m + j) * n1;
  double* zn = b.znode + (size_t)z * N;
  for (int r = threadIdx.x; r < n; r += kNkBlock) {
    const double v = sigma[(size_t)z * n + r] - xi * b.zH[(size_t)z * n + r];
    Zj[r] = v;
    zn[r + 1] = v;
  }
  if (threadIdx.x == 0) {
    Zj[n] = xi;
    zn[0] = 0.0;
    zn[N - 1] = 0.0;
    b.zh0[z] = xi;
  }
}

__global__ void __launch_bounds__(kNkBlock) k_nk_prec(const LineInst* __restrict__ inst, NkBuf b, int j,
                                                      const double* __restrict__ sigma, const int* __restrict__ skip,
                                                      int N, const int* __restrict__ jd) {
  const int z = blockIdx.x;
  if (skip[z]) return;
  if (jd) j = *jd;
  __shared__ double sh[kNkBlock];
  nk_prec(inst, b, j, sigma, N, z, sh);
}

// Exact directional derivative of R_i: (dR/dP) v + (dR/dH0) v_H0, given the
// nodal direction zn (zero at the boundary nodes) and the film's directional
// derivative dH = -K v + v_H0.
struct JvArgs {
  const double *P, *H, *rho, *drho, *deta_rel, *eps, *psia, *psib, *dH, *zn;
};
__device__ __forceinline__ double line_jv_row(const JvArgs& q, size_t base, int i, double h) {
  auto dU = [&](int j) { return q.rho[base + j] * q.dH[base + j] + q.drho[base + j] * q.H[base + j] * q.zn[base + j]; };
  auto dE = [&](int j) {
    const double e = q.eps[base + j];
    return (3.0 * e / q.H[base + j]) * q.dH[base + j] +
           e * (q.drho[base + j] / q.rho[base + j] - q.deta_rel[base + j]) * q.zn[base + j];
  };
  auto dF = [&](int j) {
    const double d0 = dU(j);
    if (j == 0) return d0;
    return d0 + 0.5 * (q.psia[base + j] * (d0 - dU(j - 1)) + q.psib[base + j] * (dU(j + 1) - d0));
  };
  const double dC = (dF(i) - dF(i - 1)) / h;
  const double ef1 = 0.5 * (q.eps[base + i] + q.eps[base + i + 1]);
  const double ef0 = 0.5 * (q.eps[base + i - 1] + q.eps[base + i]);
  const double Pi = q.P[base + i];
  const double* zn = q.zn + base;
  const double dq = 0.5 * (dE(i) + dE(i + 1)) * (q.P[base + i + 1] - Pi) + ef1 * (zn[i + 1] - zn[i]) -
                    0.5 * (dE(i - 1) + dE(i)) * (Pi - q.P[base + i - 1]) - ef0 * (zn[i] - zn[i - 1]);
  return dC - dq / (h * h);
}

// The coefficients of the directional derivative that do not depend on the
// direction, once per Newton step: jc[j] = (drho_j H_j, 3 eps_j / H_j,
// eps_j (drho_j / rho_j - deta_j), 1 / d_j), so that a Krylov product needs no
// division (the FP64 pipe runs at 1/64 of the FP32 rate).
__global__ void k_nk_jvcoef(const double* __restrict__ rho, const double* __restrict__ drho,
                            const double* __restrict__ deta_rel, const double* __restrict__ eps,
                            const double* __restrict__ H, const double* __restrict__ dg, const int* __restrict__ skip,
                            double* __restrict__ jc, int N) {
  const int z = blockIdx.y;
  if (skip[z]) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const size_t o = (size_t)z * N + j;
  const double e = eps[o], Hj = H[o];
  double* c = jc + 4 * o;
  c[0] = drho[o] * Hj;
  c[1] = 3.0 * e / Hj;
  c[2] = e * (drho[o] / rho[o] - deta_rel[o]);
  c[3] = (j >= 1 && j <= N - 2) ? 1.0 / dg[(size_t)z * (N - 2) + j - 1] : 0.0;
}

// line_jv_row with the per-step coefficients, every nodal derivative formed once
__device__ __forceinline__ double line_jv_row_c(const JvArgs& q, const double* __restrict__ jc, size_t base, int i,
                                                double ih, double ih2) {
  const double* cj = jc + 4 * base;
  auto dU = [&](int j) { return q.rho[base + j] * q.dH[base + j] + cj[4 * j] * q.zn[base + j]; };
  auto dE = [&](int j) { return cj[4 * j + 1] * q.dH[base + j] + cj[4 * j + 2] * q.zn[base + j]; };
  const double um2 = (i >= 2) ? dU(i - 2) : 0.0, um1 = dU(i - 1), u0 = dU(i), up1 = dU(i + 1);
  const double F1 = u0 + 0.5 * (q.psia[base + i] * (u0 - um1) + q.psib[base + i] * (up1 - u0));
  const double F0 =
      (i == 1) ? um1 : um1 + 0.5 * (q.psia[base + i - 1] * (um1 - um2) + q.psib[base + i - 1] * (u0 - um1));
  const double em1 = dE(i - 1), e0 = dE(i), ep1 = dE(i + 1);
  const double ef1 = 0.5 * (q.eps[base + i] + q.eps[base + i + 1]);
  const double ef0 = 0.5 * (q.eps[base + i - 1] + q.eps[base + i]);
  const double Pi = q.P[base + i];
  const double* zn = q.zn + base;
  const double dq = 0.5 * (e0 + ep1) * (q.P[base + i + 1] - Pi) + ef1 * (zn[i + 1] - zn[i]) -
                    0.5 * (em1 + e0) * (Pi - q.P[base + i - 1]) - ef0 * (zn[i] - zn[i - 1]);
  return (F1 - F0) * ih - dq * ih2;
}

// w = J_Phi z at interior node i (the force row is added by the Arnoldi step)
__device__ __forceinline__ void nk_jv(const LineInst* inst, const NkBuf& b, const JvArgs& q, const uint8_t* act, int z,
                                      int i, int N) {
  const int n = N - 2, n1 = n + 1;
  const size_t base = (size_t)z * N;
  const double h = inst[z].h;
  const double jv = line_jv_row_c(q, b.jc, base, i, 1.0 / h, 1.0 / (h * h));
  const size_t o = (size_t)z * n + (i - 1);
  b.w[(size_t)z * n1 + (i - 1)] = act[o] ? q.zn[base + i] : jv * b.jc[4 * (base + i) + 3];
}

// w = J_Phi z for the interior rows (the force row is added in k_nk_arnoldi)
__global__ void k_nk_jv(const LineInst* __restrict__ inst, NkBuf b, JvArgs q, const uint8_t* __restrict__ act,
                        const int* __restrict__ skip, int N) {
  const int z = blockIdx.y;
  if (skip[z]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;  // interior node
  if (i > N - 2) return;
  nk_jv(inst, b, q, act, z, i, N);
}

// out[z][i] = (dR_i/dP) v + (dR_i/dH0) v_H0 at interior nodes, 0 at the boundary
__global__ void k_line_jv_raw(const LineInst* __restrict__ inst, JvArgs q, double* __restrict__ out, int N) {
  const int z = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const size_t base = (size_t)z * N;
  out[base + i] = (i >= 1 && i <= N - 2) ? line_jv_row(q, base, i, inst[z].h) : 0.0;
}

// Arnoldi step j with modified Gram-Schmidt, Givens update, convergence test
__device__ __forceinline__ void nk_arnoldi(const LineInst* inst, const NkBuf& b, int j, double* rhs, int N, int z,
                                           double* sh) {
  const int n = N - 2, n1 = n + 1, m = b.m;
  double* w = b.w + (size_t)z * n1;
  const double* Zj = b.Z + ((size_t)z * m + j) * n1;
  double s = 0.0;
  for (int r = threadIdx.x; r < n; r += kNkBlock) s += Zj[r];
  s = block_sum(s, sh) * inst[z].h;
  if (threadIdx.x == 0) w[n] = s;
  __syncthreads();
  double* H = b.Hh + (size_t)z * (m + 1) * m;  // H[i + j*(m+1)]
  for (int i = 0; i <= j; ++i) {
    const double* Vi = b.V + ((size_t)z * (m + 1) + i) * n1;
    double d = 0.0;
    for (int r = threadIdx.x; r < n1; r += kNkBlock) d += w[r] * Vi[r];
    d = block_sum(d, sh);
    for (int r = threadIdx.x; r < n1; r += kNkBlock) w[r] -= d * Vi[r];
    if (threadIdx.x == 0) H[i + (size_t)j * (m + 1)] = d;
    __syncthreads();
  }
  double nn = 0.0;
  for (int r = threadIdx.x; r < n1; r += kNkBlock) nn += w[r] * w[r];
  nn = sqrt(block_sum(nn, sh));
  double* Vn = b.V + ((size_t)z * (m + 1) + j + 1) * n1;
  const double inv = nn > 0.0 ? 1.0 / nn : 0.0;
  for (int r = threadIdx.x; r < n1; r += kNkBlock) {
    const double v = w[r] * inv;
    Vn[r] = v;
    if (r < n) rhs[(size_t)z * n + r] = v;
  }
  if (threadIdx.x == 0) {
    double* col = H + (size_t)j * (m + 1);
    col[j + 1] = nn;
    double* cs = b.cs + (size_t)z * m;
    double* sn = b.sn + (size_t)z * m;
    for (int i = 0; i < j; ++i) {
      const double t = cs[i] * col[i] + sn[i] * col[i + 1];
      col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
      col[i] = t;
    }
    const double a = col[j], c = col[j + 1];
    const double r = hypot(a, c);
    const double cj = r > 0.0 ? a / r : 1.0, sj = r > 0.0 ? c / r : 0.0;
    cs[j] = cj;
    sn[j] = sj;
    col[j] = r;
    col[j + 1] = 0.0;
    double* g = b.g + (size_t)z * (m + 1);
    g[j + 1] = -sj * g[j];
    g[j] = cj * g[j];
    b.gm_k[z] = j + 1;
    if (fabs(g[j + 1]) <= b.rtol[z] * b.beta0[z] || j + 1 == m || nn == 0.0) b.gm_conv[z] = 1;
  }
}

__global__ void __launch_bounds__(kNkBlock) k_nk_arnoldi(const LineInst* __restrict__ inst, NkBuf b, int j,
                                                         const int* __restrict__ skip, double* __restrict__ rhs,
                                                         int N, const int* __restrict__ jd) {
  const int z = blockIdx.x;
  if (skip[z]) return;
  if (jd) j = *jd;
  __shared__ double sh[kNkBlock];
  nk_arnoldi(inst, b, j, rhs, N, z, sh);
}

// One Krylov step of an instance of at most kNkSmallN nodes in one CTA: the preconditioned
// vector z_j (k_nk_prec), the film's directional derivative dH = -K z + xi in double-float
// (k_line_deform's chunks of kDefChunk sources, summed as k_line_film sums them), w = J z
// (k_nk_jv) and the Arnoldi step (k_nk_arnoldi), with block barriers in place of the kernel
// boundaries: the same operations in the same order, in one launch instead of five.  Compiled
// into one kernel they round differently in the last bits (a converged solve agrees with the
// stage kernels' to about 1e-11).
constexpr int kNkSmallN = 257;
constexpr int kDefChunk = 128;  // sources per chunk of k_line_deform
// (It skips an instance that is done or whose GMRES has converged itself, so no skip kernel
// runs before it.)
__global__ void __launch_bounds__(kNkBlock) k_nk_krylov_small(const LineInst* __restrict__ inst, NkBuf b, int j,
                                                              const double* __restrict__ sigma,
                                                              const int* __restrict__ done, int N,
                                                              const int* __restrict__ jd,
                                                              const float2* __restrict__ gtab, JvArgs q,
                                                              double* dH, const uint8_t* __restrict__ act,
                                                              double* __restrict__ rhs) {
  const int z = blockIdx.x;
  if (done[z] || b.gm_conv[z]) return;
  if (jd) j = *jd;
  __shared__ double sh[kNkBlock];
  nk_prec(inst, b, j, sigma, N, z, sh);
  __syncthreads();
  const size_t base = (size_t)z * N;
  const double xi = b.zh0[z];
  const bool elastic = inst[z].elastic != 0;
  // dH is q.dH (written here, then read by the directional derivative below)
  for (int i = threadIdx.x; i < N; i += kNkBlock) {
    double Dd = 0.0;
    if (elastic) {
      df D = df_zero();
      for (int k0 = 0; k0 < N; k0 += kDefChunk) {
        const float2 p = line_deform_chunk(gtab + base, b.znode + base, i, k0, min(kDefChunk, N - k0));
        D = df_add(D, make_df(p.x, p.y));
      }
      Dd = df_to_double(D);
    }
    dH[base + i] = -Dd + xi;
  }
  __syncthreads();
  for (int i = threadIdx.x + 1; i <= N - 2; i += kNkBlock) nk_jv(inst, b, q, act, z, i, N);
  __syncthreads();
  nk_arnoldi(inst, b, j, rhs, N, z, sh);
}

// y = R^-1 g over the k Arnoldi steps, delta = sum y_j z_j
__global__ void __launch_bounds__(kNkBlock) k_nk_update(const LineInst* __restrict__ inst, NkBuf b,
                                                        const int* __restrict__ done, int N) {
  const int z = blockIdx.x;
  if (done[z]) return;
  const int n = N - 2, n1 = n + 1, m = b.m;
  const int k = b.gm_k[z];
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
  double* dl = b.delta + (size_t)z * n1;
  for (int r = threadIdx.x; r < n1; r += kNkBlock) {
    double s = 0.0;
    for (int q = 0; q < k; ++q) s += y[q] * b.Z[((size_t)z * m + q) * n1 + r];
    dl[r] = s;
  }
  if (threadIdx.x == 0) {
    b.tstep[z] = 1.0;
    b.lsdone[z] = 0;
    b.lsphase[z] = 0;
  }
}

// trial point P_t = P + t dP, projected on P_t >= 0 in the first phase; H0_t = H0 + t dH0
__global__ void k_nk_trial(NkBuf b, const double* __restrict__ P, const double* __restrict__ H0,
                           const int* __restrict__ skip, int N) {
  const int z = blockIdx.y;
  if (skip[z]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int n1 = N - 1;
  const double t = b.tstep[z];
  double v = 0.0;
  if (i >= 1 && i <= N - 2) {
    v = P[(size_t)z * N + i] + t * b.delta[(size_t)z * n1 + (i - 1)];
    if (b.lsphase[z] == 0) v = v > 0.0 ? v : 0.0;
  }
  b.Pt[(size_t)z * N + i] = v;
  if (i == 0) b.H0t[z] = H0[z] + t * b.delta[(size_t)z * n1 + (N - 2)];
}

// Merit of the trial point; accept (copy into P, H0) or shorten the step.
// Backtracking on ||Phi||_2 with sufficient decrease 1e-4 t.  Projected
// trials run down to t = 2^-10; the projection max(0, .) can destroy the
// descent of the Newton direction where the step drives many pressures below
// zero, so the search then restarts at t = 1 without it (Phi = min(P, R/d) is
// defined for P < 0) and accepts its last trial once t < 1e-10.
__global__ void __launch_bounds__(kNkBlock) k_nk_merit(const LineInst* __restrict__ inst, NkBuf b,
                                                       const double* __restrict__ R, const double* __restrict__ red,
                                                       const double* __restrict__ dg, const int* __restrict__ skip,
                                                       double* __restrict__ P, double* __restrict__ H0, int N) {
  const int z = blockIdx.x;
  if (skip[z]) return;
  __shared__ double sh[kNkBlock];
  __shared__ int accept;
  const int n = N - 2;
  double ss = 0.0;
  bool finite = true;
  for (int r = threadIdx.x; r < n; r += kNkBlock) {
    const double pt = b.Pt[(size_t)z * N + r + 1];
    const double rt = R[(size_t)z * N + r + 1] / dg[(size_t)z * n + r];
    const double ph = pt < rt ? pt : rt;
    if (!(ph == ph) || isinf(ph)) finite = false;
    ss += ph * ph;
  }
  ss = block_sum(ss, sh);
  const int nf = __syncthreads_or(finite ? 0 : 1);
  const double f = red[z * 4 + 1];
  const double nrm = sqrt(ss + f * f);
  const double t = b.tstep[z];
  const int phase = b.lsphase[z];
  if (threadIdx.x == 0)
    accept = (!nf && nrm == nrm && nrm <= (1.0 - 1e-4 * t) * b.phinorm[z]) || (phase == 1 && t < 1e-10);
  __syncthreads();
  if (accept) {
    for (int i = threadIdx.x; i < N; i += kNkBlock) P[(size_t)z * N + i] = b.Pt[(size_t)z * N + i];
    if (threadIdx.x == 0) {
      H0[z] = b.H0t[z];
      b.lsdone[z] = 1;
    }
  } else if (threadIdx.x == 0) {
    if (phase == 0 && 0.5 * t < 0x1p-10) {
      b.lsphase[z] = 1;
      b.tstep[z] = 1.0;
    } else {
      b.tstep[z] = 0.5 * t;
    }
  }
}

// ----------------------------------------------------------------- host side
cudaError_t line_jacobian_apply(LineCtx* c, const double* P, const double* H0, const double* rough, const double* v,
                                const double* v_h0, double* out) {
  cudaError_t e = line_state(c, P, H0, rough, nullptr, nullptr);
  // the film's change through the Krylov products' deformation (the arithmetic `precision` selects)
  if (e == cudaSuccess) e = line_krylov_deform(c, v, v_h0, nullptr);
  if (e != cudaSuccess) return e;
  JvArgs q{P, c->H, c->rho, c->drho, c->deta_rel, c->eps, c->psia, c->psib, c->dH, v};
  const dim3 gn((c->N + 255) / 256, c->n_inst);
  k_line_jv_raw<<<gn, 256, 0, c->st>>>(c->inst, q, out, c->N);
  note_launch();
  return cudaGetLastError();
}

void line_nk_free(LineCtx* c) {
  delete (NkBuf*)c->nk;
  c->nk = nullptr;
}

cudaError_t line_nk_alloc(LineCtx* c) {
  NkBuf* b = new NkBuf();
  c->nk = b;
  const int m = c->krylov_dim, n1 = c->n + 1, ni = c->n_inst;
  b->m = m;
  b->n1 = n1;
  const size_t NN = (size_t)ni * c->N;
  struct A {
    void** p;
    size_t bytes;
  } al[] = {{(void**)&b->V, sizeof(double) * ni * (m + 1) * (size_t)n1},
            {(void**)&b->Z, sizeof(double) * ni * (size_t)m * n1},
            {(void**)&b->Hh, sizeof(double) * ni * (m + 1) * (size_t)m},
            {(void**)&b->cs, sizeof(double) * ni * (size_t)m},
            {(void**)&b->sn, sizeof(double) * ni * (size_t)m},
            {(void**)&b->g, sizeof(double) * ni * (size_t)(m + 1)},
            {(void**)&b->phi, sizeof(double) * ni * (size_t)n1},
            {(void**)&b->phinorm, sizeof(double) * ni},
            {(void**)&b->zH, sizeof(double) * ni * (size_t)c->n},
            {(void**)&b->den, sizeof(double) * ni},
            {(void**)&b->delta, sizeof(double) * ni * (size_t)n1},
            {(void**)&b->Pt, sizeof(double) * NN},
            {(void**)&b->H0t, sizeof(double) * ni},
            {(void**)&b->tstep, sizeof(double) * ni},
            {(void**)&b->rtol, sizeof(double) * ni},
            {(void**)&b->beta0, sizeof(double) * ni},
            {(void**)&b->znode, sizeof(double) * NN},
            {(void**)&b->zh0, sizeof(double) * ni},
            {(void**)&b->w, sizeof(double) * ni * (size_t)n1},
            {(void**)&b->jc, sizeof(double) * 4 * NN},
            {(void**)&b->gm_k, sizeof(int) * ni},
            {(void**)&b->gm_conv, sizeof(int) * ni},
            {(void**)&b->lsdone, sizeof(int) * ni},
            {(void**)&b->lsphase, sizeof(int) * ni},
            {(void**)&b->skip, sizeof(int) * ni},
            {(void**)&b->loop, sizeof(int) * kLoopSlots},
            {(void**)&b->fstore, paqif_factor_store_bytes(ni * c->pq_parts, c->n / c->pq_parts, c->beta, c->pq_r)}};
  for (auto& x : al) {
    cudaError_t e = ctx_alloc(c, x.p, x.bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// PAQIF on the scaled band.  Its cavitated rows are already identity rows, and
// the preconditioner must return v_i on them, so no active mask is passed (a
// mask would pin those unknowns to zero).  factor = true factors the band once
// per Newton step (solving for rhs as well); otherwise the stored factors are
// reused for a new right-hand side.
static cudaError_t paqif_on(LineCtx* c, const double* rhs, double* x, bool factor) {
  NkBuf& b = *(NkBuf*)c->nk;
  PaqifLaunch L;
  // pq_parts diagonal blocks per band, consecutive rows: the band rows of block p
  // start at row p n/r, and entries that couple to other blocks fall outside the
  // block's matrix, so PAQIF ignores them (block Jacobi)
  L.n_sys = c->n_inst * c->pq_parts;
  L.n = c->n / c->pq_parts;
  L.parts = c->pq_r;
  L.beta = c->beta;
  L.mode = 0;
  L.band = c->band;
  L.rhs = rhs;
  L.act = nullptr;
  L.stack = c->pq_ws;
  L.x = x;
  L.iters = nullptr;
  L.info = c->pq_info;
  L.f32 = c->precision > 0;  // the mixed-precision path also runs its preconditioner in float32
  return factor ? launch_paqif_factor(L, b.fstore, c->st) : launch_paqif_resolve(L, b.fstore, c->st);
}

static bool krylov_fused(const LineCtx* c) { return c->fuse && c->precision == 0 && c->N <= kNkSmallN; }

// Krylov step j (or the index at jd, in a device-driven solve) after the preconditioner's
// PAQIF solve: z_j, the film derivative, w = J z and the Arnoldi step; one CTA per instance for
// small plain-precision instances, else the skip flags and the stage kernels.
static cudaError_t krylov_step(LineCtx* c, const double* P, int j, const int* jd) {
  NkBuf& b = *(NkBuf*)c->nk;
  const int ni = c->n_inst, N = c->N;
  JvArgs q{P, c->H, c->rho, c->drho, c->deta_rel, c->eps, c->psia, c->psib, c->dH, b.znode};
  if (krylov_fused(c)) {
    k_nk_krylov_small<<<ni, kNkBlock, 0, c->st>>>(c->inst, b, j, c->sigma, c->done, N, jd, c->gtab, q, c->dH,
                                                  c->act, c->rhs);
    note_launch();
    return cudaGetLastError();
  }
  k_nk_skip<<<(ni + 127) / 128, 128, 0, c->st>>>(c->done, b.gm_conv, b.skip, ni);
  note_launch();
  k_nk_prec<<<ni, kNkBlock, 0, c->st>>>(c->inst, b, j, c->sigma, b.skip, N, jd);
  note_launch();
  cudaError_t e = line_krylov_deform(c, b.znode, b.zh0, b.skip);
  if (e != cudaSuccess) return e;
  k_nk_jv<<<dim3((N + 255) / 256, ni), 256, 0, c->st>>>(c->inst, b, q, c->act, b.skip, N);
  note_launch();
  k_nk_arnoldi<<<ni, kNkBlock, 0, c->st>>>(c->inst, b, j, b.skip, c->rhs, N, jd);
  note_launch();
  return cudaGetLastError();
}

static bool all_set(LineCtx* c, const int* a, const int* b2, cudaError_t& e) {
  std::vector<int> ha(c->n_inst), hb(c->n_inst);
  e = cudaMemcpyAsync(ha.data(), a, sizeof(int) * c->n_inst, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hb.data(), b2, sizeof(int) * c->n_inst, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  for (int k = 0; k < c->n_inst; ++k)
    if (!ha[k] && !hb[k]) return false;
  return true;
}

// Line-search trials [t0, t1): trial point, its residual, merit and acceptance;
// with check, stop as soon as every instance is done or has accepted.
static cudaError_t line_nk_trials(LineCtx* c, double* P, double* H0, const double* rough, int t0, int t1,
                                  bool check) {
  NkBuf& b = *(NkBuf*)c->nk;
  const int ni = c->n_inst, N = c->N;
  const dim3 gn((N + 255) / 256, ni);
  cudaError_t e = cudaSuccess;
  for (int trial = t0; trial < t1; ++trial) {
    k_nk_skip<<<(ni + 127) / 128, 128, 0, c->st>>>(c->done, b.lsdone, b.skip, ni);
    note_launch();
    k_nk_trial<<<gn, 256, 0, c->st>>>(b, P, H0, b.skip, N);
    note_launch();
    e = line_state(c, b.Pt, b.H0t, rough, b.skip, nullptr);
    if (e == cudaSuccess) e = line_finalize(c, nullptr, nullptr);
    if (e != cudaSuccess) return e;
    k_nk_merit<<<ni, kNkBlock, 0, c->st>>>(c->inst, b, c->R, c->red, c->dg, b.skip, P, H0, N);
    note_launch();
    if (check) {
      if (all_set(c, c->done, b.lsdone, e)) {
        // every instance accepted its last evaluated trial: the state arrays are at the new iterate
        c->state_current = true;
        break;
      }
      if (e != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

cudaError_t line_nk_finish(LineCtx* c, double* P, double* H0, const double* rough, int first_trial) {
  NkBuf& b = *(NkBuf*)c->nk;
  cudaError_t e = cudaSuccess;
  if (all_set(c, c->done, b.lsdone, e) || e != cudaSuccess) return e;
  return line_nk_trials(c, P, H0, rough, first_trial, 64, true);
}

// One Newton step for every instance that is not done.
cudaError_t line_nk_step(LineCtx* c, double* P, double* H0, const double* rough) {
  NkBuf& b = *(NkBuf*)c->nk;
  const int ni = c->n_inst, N = c->N;
  cudaError_t e = cudaSuccess;
  // the state at (P, H0) was left by the accepted line-search trials of the last step,
  // unless this step is captured into a graph (which must compute it on every replay)
  if (c->capturing || !c->state_current) e = line_state(c, P, H0, rough, c->done, nullptr);
  c->state_current = false;
  if (e == cudaSuccess) e = line_finalize(c, c->done, c->iters);
  if (e == cudaSuccess) e = line_jac_band(c, P, 1, c->band, c->act, c->jh, c->dg, c->done);
  if (e != cudaSuccess) return e;
  k_nk_setup<<<ni, kNkBlock, 0, c->st>>>(c->inst, b, P, c->R, c->red, c->act, c->dg, c->jh, c->done, c->band,
                                         c->rhs, N, c->beta);
  note_launch();
  k_nk_jvcoef<<<dim3((N + 255) / 256, ni), 256, 0, c->st>>>(c->rho, c->drho, c->deta_rel, c->eps, c->H, c->dg,
                                                            c->done, b.jc, N);
  note_launch();
  e = paqif_on(c, c->rhs, c->sigma, true);  // factor, solving for the border column
  if (e != cudaSuccess) return e;
  k_nk_border<<<ni, kNkBlock, 0, c->st>>>(c->inst, b, c->sigma, c->done, c->rhs, N);
  note_launch();
  for (int j = 0; j < b.m; ++j) {
    e = paqif_on(c, c->rhs, c->sigma, false);
    if (e != cudaSuccess) return e;
    e = krylov_step(c, P, j, nullptr);
    if (e != cudaSuccess) return e;
    if (!c->capturing && (j + 1) % 8 == 0 && j + 1 < b.m) {
      if (all_set(c, c->done, b.gm_conv, e)) break;
      if (e != cudaSuccess) return e;
    }
  }
  k_nk_update<<<ni, kNkBlock, 0, c->st>>>(c->inst, b, c->done, N);
  note_launch();
  if (c->capturing) return line_nk_trials(c, P, H0, rough, 0, kGraphTrials, false);
  std::vector<int> tk, tc;
  std::vector<double> tphin, trtol;
  if (c->trace) {
    const int nt = c->trace < ni ? c->trace : ni;
    tk.resize(nt);
    tc.resize(nt);
    tphin.resize(nt);
    trtol.resize(nt);
    e = cudaMemcpyAsync(tk.data(), b.gm_k, sizeof(int) * nt, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tc.data(), b.gm_conv, sizeof(int) * nt, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(tphin.data(), b.phinorm, sizeof(double) * nt, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(trtol.data(), b.rtol, sizeof(double) * nt, cudaMemcpyDeviceToHost, c->st);
    if (e != cudaSuccess) return e;
  }
  e = line_nk_trials(c, P, H0, rough, 0, 64, true);
  if (e != cudaSuccess) return e;
  if (c->trace) {
    const int nt = (int)tk.size();
    std::vector<double> tt(nt), tred(4 * nt);
    std::vector<int> tph(nt), tdone(nt), tit(nt);
    e = cudaMemcpyAsync(tt.data(), b.tstep, sizeof(double) * nt, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tph.data(), b.lsphase, sizeof(int) * nt, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tdone.data(), c->done, sizeof(int) * nt, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tit.data(), c->iters, sizeof(int) * nt, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return e;
    for (int z = 0; z < nt; ++z)
      if (!tdone[z])
        fprintf(stderr, "ehl nk N=%d inst %d it %d |Phi| %.3e rtol %.1e gmres %d conv %d t %.3e phase %d\n", N, z,
                tit[z], tphin[z], trtol[z], tk[z], tc[z], tt[z], tph[z]);
  }
  return cudaGetLastError();
}

// ===================================================== device-driven solve (graph mode 2)
// The outer Newton iteration, the GMRES iteration and the line search run as while-loops of one
// CUDA graph: each loop's condition is set on the device (cudaGraphSetConditional) by k_nk_loop
// from the instances' done / converged / accepted flags and an iteration cap, so a whole solve
// of a grid is one graph launch with no host round trip.

// any instance with done[z] == 0 and other[z] == 0 (block-wide)
__device__ __forceinline__ bool nk_any_active(const int* done, const int* other, int ni) {
  int a = 0;
  for (int z = threadIdx.x; z < ni && !a; z += blockDim.x) a = !done[z] && !(other && other[z]);
  return __syncthreads_or(a) != 0;
}

// next = 0: counter = 0 (before the loop); next = 1: counter += 1 (end of a pass), total += 1.
// The loop continues while counter < cap and some instance is active.
__global__ void k_nk_loop(cudaGraphConditionalHandle h, int* __restrict__ counter, int* __restrict__ total, int cap,
                          int next, const int* __restrict__ done, const int* __restrict__ other, int ni) {
  const int c = next ? *counter + 1 : 0;
  const bool act = nk_any_active(done, other, ni);  // a block barrier: every thread has read *counter
  if (threadIdx.x == 0) {
    *counter = c;
    if (next && total) *total += 1;
    cudaGraphSetConditional(h, (c < cap && act) ? 1u : 0u);
  }
}

namespace {

cudaError_t nk_loop(LineCtx* c, cudaGraphConditionalHandle h, int slot, int total_slot, int cap, int next,
                    const int* other) {
  NkBuf& b = *(NkBuf*)c->nk;
  k_nk_loop<<<1, 256, 0, c->st>>>(h, b.loop + slot, total_slot >= 0 ? b.loop + total_slot : nullptr, cap, next,
                                  c->done, other, c->n_inst);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t line_nk_capture_solve(LineCtx* c, double* P, double* H0, const double* rough, cudaStream_t s1,
                                  cudaStream_t s2, SolveGraphCounts& n) {
  NkBuf& b = *(NkBuf*)c->nk;
  const int ni = c->n_inst, N = c->N;
  const cudaStream_t s0 = c->st;
  const dim3 gn((N + 255) / 256, ni);
  c->capturing = true;
  cudaError_t e = cudaSuccess;
  unsigned long long l0 = thread_launches();
  // as iterate(): fresh flags, no residual seen yet (bytes 0x7f: 1.4e306), no stall
  e = cudaMemsetAsync(c->done, 0, sizeof(int) * ni, s0);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->iters, 0, sizeof(int) * ni, s0);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->best, 0x7f, sizeof(double) * ni, s0);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->stall, 0, sizeof(int) * ni, s0);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.loop, 0, sizeof(int) * kLoopSlots, s0);
  auto krylov_body = [&](cudaGraphConditionalHandle hk) -> cudaError_t {
    cudaError_t ee = paqif_on(c, c->rhs, c->sigma, false);
    if (ee != cudaSuccess) return ee;
    ee = krylov_step(c, P, 0, b.loop + 1);
    if (ee != cudaSuccess) return ee;
    return nk_loop(c, hk, 1, 3, b.m, 1, b.gm_conv);
  };
  auto trial_body = [&](cudaGraphConditionalHandle ht) -> cudaError_t {
    k_nk_skip<<<(ni + 127) / 128, 128, 0, c->st>>>(c->done, b.lsdone, b.skip, ni);
    note_launch();
    k_nk_trial<<<gn, 256, 0, c->st>>>(b, P, H0, b.skip, N);
    note_launch();
    cudaError_t ee = line_state(c, b.Pt, b.H0t, rough, b.skip, nullptr);
    if (ee == cudaSuccess) ee = line_finalize(c, nullptr, nullptr);
    if (ee != cudaSuccess) return ee;
    k_nk_merit<<<ni, kNkBlock, 0, c->st>>>(c->inst, b, c->R, c->red, c->dg, b.skip, P, H0, N);
    note_launch();
    return nk_loop(c, ht, 2, 4, 64, 1, b.lsdone);
  };
  auto newton_body = [&](cudaGraphConditionalHandle hn) -> cudaError_t {
    const unsigned long long m0 = thread_launches();
    cudaError_t ee = line_state(c, P, H0, rough, c->done, nullptr);
    if (ee == cudaSuccess) ee = line_finalize(c, c->done, c->iters);
    if (ee == cudaSuccess) ee = line_jac_band(c, P, 1, c->band, c->act, c->jh, c->dg, c->done);
    if (ee != cudaSuccess) return ee;
    k_nk_setup<<<ni, kNkBlock, 0, c->st>>>(c->inst, b, P, c->R, c->red, c->act, c->dg, c->jh, c->done, c->band,
                                           c->rhs, N, c->beta);
    note_launch();
    k_nk_jvcoef<<<dim3((N + 255) / 256, ni), 256, 0, c->st>>>(c->rho, c->drho, c->deta_rel, c->eps, c->H, c->dg,
                                                              c->done, b.jc, N);
    note_launch();
    ee = paqif_on(c, c->rhs, c->sigma, true);
    if (ee != cudaSuccess) return ee;
    k_nk_border<<<ni, kNkBlock, 0, c->st>>>(c->inst, b, c->sigma, c->done, c->rhs, N);
    note_launch();
    const cudaStream_t here = c->st;
    ee = capture_while(
        c, here, s2, [&](cudaGraphConditionalHandle hk) { return nk_loop(c, hk, 1, -1, b.m, 0, b.gm_conv); },
        krylov_body, &n.krylov);
    if (ee != cudaSuccess) return ee;
    k_nk_update<<<ni, kNkBlock, 0, c->st>>>(c->inst, b, c->done, N);
    note_launch();
    ee = capture_while(
        c, here, s2, [&](cudaGraphConditionalHandle ht) { return nk_loop(c, ht, 2, -1, 64, 0, b.lsdone); },
        trial_body, &n.trial);
    if (ee != cudaSuccess) return ee;
    ee = nk_loop(c, hn, 0, -1, c->max_iter, 1, nullptr);
    n.newton = (long long)(thread_launches() - m0) - n.krylov - n.trial;
    return ee;
  };
  if (e == cudaSuccess)
    e = capture_while(
        c, s0, s1, [&](cudaGraphConditionalHandle hn) { return nk_loop(c, hn, 0, -1, c->max_iter, 0, nullptr); },
        newton_body, nullptr);
  c->st = s0;
  if (e == cudaSuccess) e = line_state(c, P, H0, rough, nullptr, nullptr);
  if (e == cudaSuccess) e = line_finalize(c, nullptr, nullptr);
  c->capturing = false;
  n.fixed = (long long)(thread_launches() - l0) - n.newton - n.krylov - n.trial;
  return e;
}

// kernels the last replay ran, from the loop totals (read after the replay)
long long line_nk_graph_launches(const SolveGraphCounts& n, const int* loop_host) {
  return n.fixed + (long long)loop_host[0] * n.newton + (long long)loop_host[3] * n.krylov +
         (long long)loop_host[4] * n.trial;
}

const int* line_nk_loop_counters(LineCtx* c) { return ((NkBuf*)c->nk)->loop; }

}  // namespace ehl
