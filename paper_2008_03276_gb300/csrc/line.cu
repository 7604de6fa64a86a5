// line.cu -- line-contact hot path (Sec. 3.3): closed-form kernel table,
// double-float Toeplitz deformation, float64 lubricant model and TVD residual,
// the band Jacobians, and the paper's limiter-based Newton-Raphson relaxation.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>

#include <vector>

#include "df64.cuh"
#include "ehl_internal.h"
#include "line_kernels.cuh"
#include "graph_loop.h"
#include "line.h"
#include "tc_gemm.h"

namespace ehl {

constexpr int kDefTI = 64;    // outputs per deformation CTA
constexpr int kDefSK = 128;   // sources per deformation CTA
constexpr int kNodeBlock = 256;

// max that keeps a NaN operand (fmax would drop it)
__device__ __forceinline__ double nan_max(double a, double b) { return (a > b || a != a) ? a : b; }

// ---------------------------------------------------------------- kernel table
__global__ void k_line_gtab(const LineInst* __restrict__ inst, float2* __restrict__ gtab, double* __restrict__ gtab64,
                            int N) {
  const int z = blockIdx.y;
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= N) return;
  const double g = line_cell_integral(d, inst[z].h) / M_PI;
  const df v = df_from_double(g);
  gtab[(size_t)z * N + d] = make_float2(v.hi, v.lo);
  gtab64[(size_t)z * N + d] = g;
}

// ---------------------------------------------------------------- deformation
// partial[y][z][i] = sum_{k in chunk y} K_{|i-k|} V[z][k]   (double-float, Ogita-Rump-Oishi Dot2 sum)
__global__ void __launch_bounds__(kDefTI) k_line_deform(const LineInst* __restrict__ inst,
                                                        const float2* __restrict__ gtab,
                                                        const double* __restrict__ V, int vstride,
                                                        const int* __restrict__ skip, float2* __restrict__ partial,
                                                        int n_inst, int N) {
  const int z = blockIdx.z;
  if (skip && skip[z]) return;
  const int i0 = blockIdx.x * kDefTI, k0 = blockIdx.y * kDefSK;
  const int tid = threadIdx.x;
  float2* out = partial + ((size_t)blockIdx.y * n_inst + z) * N;
  if (!inst[z].elastic) {
    if (i0 + tid < N) out[i0 + tid] = make_float2(0.f, 0.f);
    return;
  }
  __shared__ float2 Vs[kDefSK];
  __shared__ float2 Gs[kDefTI + kDefSK - 1];
  for (int t = tid; t < kDefSK; t += kDefTI) {
    const int k = k0 + t;
    df v = (k < N) ? df_from_double(V[(size_t)z * vstride + k]) : df_zero();
    Vs[t] = make_float2(v.hi, v.lo);
  }
  const int base_d = i0 - (k0 + kDefSK - 1);
  for (int m = tid; m < kDefTI + kDefSK - 1; m += kDefTI) {
    int d = base_d + m;
    d = d < 0 ? -d : d;
    Gs[m] = (d < N) ? gtab[(size_t)z * N + d] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int i = i0 + tid;
  if (i >= N) return;
  float s = 0.f, c = 0.f;
  const int kmax = min(kDefSK, N - k0);
#pragma unroll 4
  for (int k = 0; k < kmax; ++k) {
    const float2 g = Gs[tid + kDefSK - 1 - k];
    const float2 v = Vs[k];
    const float p = __fmul_rn(g.x, v.x);
    float e = __fmaf_rn(g.x, v.x, -p);
    e = __fmaf_rn(g.x, v.y, e);
    e = __fmaf_rn(g.y, v.x, e);
    float t1, t2;
    two_sum(s, p, t1, t2);
    s = t1;
    c = __fadd_rn(c, __fadd_rn(t2, e));
  }
  float hi, lo;
  fast_two_sum(s, c, hi, lo);
  out[i] = make_float2(hi, lo);
}

// The same sums in float64 (FMA accumulation per CTA chunk, chunks added in
// float64 by the film kernel): the deformation of the residual, whose
// rounding sets how far the outer iteration can drive ||min(P,R)||.  The
// double-float form above (about 48 bits) serves the Krylov products.
__global__ void __launch_bounds__(kDefTI) k_line_deform64(const LineInst* __restrict__ inst,
                                                          const double* __restrict__ gtab64,
                                                          const double* __restrict__ V, int vstride,
                                                          const int* __restrict__ skip, double* __restrict__ partial,
                                                          int n_inst, int N) {
  const int z = blockIdx.z;
  if (skip && skip[z]) return;
  const int i0 = blockIdx.x * kDefTI, k0 = blockIdx.y * kDefSK;
  const int tid = threadIdx.x;
  double* out = partial + ((size_t)blockIdx.y * n_inst + z) * N;
  if (!inst[z].elastic) {
    if (i0 + tid < N) out[i0 + tid] = 0.0;
    return;
  }
  __shared__ double Vs[kDefSK];
  __shared__ double Gs[kDefTI + kDefSK - 1];
  for (int t = tid; t < kDefSK; t += kDefTI) {
    const int k = k0 + t;
    Vs[t] = (k < N) ? V[(size_t)z * vstride + k] : 0.0;
  }
  const int base_d = i0 - (k0 + kDefSK - 1);
  for (int m = tid; m < kDefTI + kDefSK - 1; m += kDefTI) {
    int d = base_d + m;
    d = d < 0 ? -d : d;
    Gs[m] = (d < N) ? gtab64[(size_t)z * N + d] : 0.0;
  }
  __syncthreads();
  const int i = i0 + tid;
  if (i >= N) return;
  const int kmax = min(kDefSK, N - k0);
  // four interleaved accumulators: independent FMA chains
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int k = 0;
  for (; k + 4 <= kmax; k += 4) {
    s0 = fma(Gs[tid + kDefSK - 1 - k], Vs[k], s0);
    s1 = fma(Gs[tid + kDefSK - 2 - k], Vs[k + 1], s1);
    s2 = fma(Gs[tid + kDefSK - 3 - k], Vs[k + 2], s2);
    s3 = fma(Gs[tid + kDefSK - 4 - k], Vs[k + 3], s3);
  }
  for (; k < kmax; ++k) s0 = fma(Gs[tid + kDefSK - 1 - k], Vs[k], s0);
  out[i] = (s0 + s1) + (s2 + s3);
}

// mode 0: H = H0 + X^2/2 - D + rough;  mode 1: out = -D + dh0 (directional derivative of H)
// partial holds float64 chunk sums (p64 = 1), double-float ones (0) or one float32 product (2)
__global__ void k_line_film(const LineInst* __restrict__ inst, const float2* __restrict__ partial, int ksplit,
                            const double* __restrict__ H0, const double* __restrict__ rough, int rstride,
                            const int* __restrict__ skip, double* __restrict__ out, int n_inst, int N, int mode,
                            int p64) {
  const int z = blockIdx.y;
  if (skip && skip[z]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double Dd;
  if (p64 == 2) {  // one float32 product [n_inst][N] (the GEMM of the mixed-precision Krylov products)
    Dd = (double)reinterpret_cast<const float*>(partial)[(size_t)z * N + i];
  } else if (p64 == 3) {  // float32 partial products of the K-splits [ksplit][n_inst][N] (tensor cores)
    const float* pf = reinterpret_cast<const float*>(partial);
    Dd = 0.0;
    for (int y = 0; y < ksplit; ++y) Dd += (double)pf[((size_t)y * n_inst + z) * N + i];
  } else if (p64) {
    const double* pd = reinterpret_cast<const double*>(partial);
    Dd = 0.0;
    for (int y = 0; y < ksplit; ++y) Dd += pd[((size_t)y * n_inst + z) * N + i];
  } else {
    df D = df_zero();
    for (int y = 0; y < ksplit; ++y) {
      const float2 p = partial[((size_t)y * n_inst + z) * N + i];
      D = df_add(D, make_df(p.x, p.y));
    }
    Dd = df_to_double(D);
  }
  if (mode == 0) {
    double H = line_film_h(inst[z], i, H0[z], Dd);
    if (rough) H += rough[(size_t)z * rstride + i];
    out[(size_t)z * N + i] = H;
  } else {
    out[(size_t)z * N + i] = -Dd + (H0 ? H0[z] : 0.0);
  }
}

// ---------------------------------------------------------------- lubricant state
__global__ void k_line_nodes(const LineInst* __restrict__ inst, const double* __restrict__ P,
                             const double* __restrict__ H, const int* __restrict__ skip, double* __restrict__ rho,
                             double* __restrict__ drho, double* __restrict__ deta_rel, double* __restrict__ eps,
                             double* __restrict__ u, int N) {
  const int z = blockIdx.y;
  if (skip && skip[z]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const LineInst q = inst[z];
  line_node(q, (size_t)z * N + i, P, H, rho, drho, deta_rel, eps, u);
}

// face j (0..N-2) at offset o: limited face value and the limiter's derivatives
__device__ __forceinline__ void line_face(const LineInst& q, size_t o, int j, const double* u, double* F,
                                          double* psi, double* psia, double* psib) {
  double ps = 0.0, pa = 0.0, pb = 0.0;
  if (j >= 1) line_limiter(q.limiter, q.kappa, u[o] - u[o - 1], u[o + 1] - u[o], ps, pa, pb);
  F[o] = u[o] + 0.5 * ps;
  psi[o] = ps;
  psia[o] = pa;
  psib[o] = pb;
}

// faces j = 0..N-2: limited face value and limiter derivatives
__global__ void k_line_faces(const LineInst* __restrict__ inst, const double* __restrict__ u,
                             const int* __restrict__ skip, double* __restrict__ F, double* __restrict__ psi,
                             double* __restrict__ psia, double* __restrict__ psib, int N) {
  const int z = blockIdx.y;
  if (skip && skip[z]) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N - 1) return;
  line_face(inst[z], (size_t)z * N + j, j, u, F, psi, psia, psib);
}

// R_i at node i of the instance at offset base (0 at the boundary nodes) and the block's
// reductions of max|min(P,R)|, sum P, min H and the largest term of R into out[0..3] (one
// thread per node, kNodeBlock threads, a tree over the block)
__device__ __forceinline__ void line_residual_block(double h, const double* P, const double* H, const double* eps,
                                                    const double* F, double* R, double* out, size_t base, int i,
                                                    int N) {
  double cres = 0.0, sp = 0.0, hmin = INFINITY, term = 0.0;
  if (i < N) {
    const size_t o = base + i;
    hmin = H[o];
    if (i >= 1 && i <= N - 2) {
      const double C = (F[o] - F[o - 1]) / h;
      const double ef1 = 0.5 * (eps[o] + eps[o + 1]);
      const double ef0 = 0.5 * (eps[o - 1] + eps[o]);
      const double Q = (ef1 * (P[o + 1] - P[o]) - ef0 * (P[o] - P[o - 1])) / (h * h);
      const double r = C - Q;
      R[o] = r;
      cres = fabs(P[o] < r ? P[o] : r);  // NaN in r propagates
      sp = P[o];
      // magnitude of the largest term of R_i (sets the rounding floor of R)
      term = (fabs(F[o]) + fabs(F[o - 1])) / h +
             (fabs(ef1 * (P[o + 1] - P[o])) + fabs(ef0 * (P[o] - P[o - 1]))) / (h * h);
    } else {
      R[o] = 0.0;
    }
  }
  __shared__ double s_c[kNodeBlock], s_s[kNodeBlock], s_h[kNodeBlock], s_t[kNodeBlock];
  s_c[threadIdx.x] = cres;
  s_s[threadIdx.x] = sp;
  s_h[threadIdx.x] = hmin;
  s_t[threadIdx.x] = term;
  __syncthreads();
  for (int w = kNodeBlock / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s_c[threadIdx.x] = nan_max(s_c[threadIdx.x], s_c[threadIdx.x + w]);
      s_s[threadIdx.x] += s_s[threadIdx.x + w];
      s_h[threadIdx.x] = fmin(s_h[threadIdx.x], s_h[threadIdx.x + w]);
      s_t[threadIdx.x] = fmax(s_t[threadIdx.x], s_t[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s_c[0];
    out[1] = s_s[0];
    out[2] = s_h[0];
    out[3] = s_t[0];
  }
}

// residual at interior nodes; block partials of max|min(P,R)|, sum P and min H
__global__ void __launch_bounds__(kNodeBlock) k_line_residual(const LineInst* __restrict__ inst,
                                                              const double* __restrict__ P,
                                                              const double* __restrict__ H,
                                                              const double* __restrict__ eps,
                                                              const double* __restrict__ F,
                                                              const int* __restrict__ skip, double* __restrict__ R,
                                                              double* __restrict__ blk, int nblk, int N) {
  const int z = blockIdx.y;
  if (skip && skip[z]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  line_residual_block(inst[z].h, P, H, eps, F, R, blk + ((size_t)z * nblk + blockIdx.x) * 4, (size_t)z * N, i, N);
}

// line_state of an instance of at most kNodeBlock nodes in one CTA, one thread per node: the
// film from k_line_deform64's float64 chunk sums, the lubricant state, the limited faces and the
// residual with its block reductions.  The arithmetic of k_line_film, k_line_nodes, k_line_faces
// and k_line_residual in the same order (one residual block, nblk = 1), so the same results
// bit for bit, in one launch instead of four.
__global__ void __launch_bounds__(kNodeBlock) k_line_state_small(
    const LineInst* __restrict__ inst, const double* __restrict__ partial, int ksplit, const double* __restrict__ H0,
    const double* __restrict__ rough, const double* __restrict__ P, const int* __restrict__ skip, double* H,
    double* rho, double* drho, double* deta_rel, double* eps, double* u, double* F, double* psi, double* psia,
    double* psib, double* R, double* __restrict__ blk, int n_inst, int N) {
  const int z = blockIdx.x;
  if (skip && skip[z]) return;
  const int i = threadIdx.x;
  const LineInst q = inst[z];
  const size_t base = (size_t)z * N;
  if (i < N) {
    double Dd = 0.0;
    for (int y = 0; y < ksplit; ++y) Dd += partial[((size_t)y * n_inst + z) * N + i];
    double Hv = line_film_h(q, i, H0[z], Dd);
    if (rough) Hv += rough[base + i];
    H[base + i] = Hv;
    line_node(q, base + i, P, H, rho, drho, deta_rel, eps, u);
  }
  __syncthreads();
  if (i < N - 1) line_face(q, base + i, i, u, F, psi, psia, psib);
  __syncthreads();
  line_residual_block(q.h, P, H, eps, F, R, blk + (size_t)z * 4, base, i, N);
}

// red[z] = (max|min(P,R)|, h sum P - pi/2, sum P, min H); convergence flag and iteration count
__global__ void k_line_finalize(const LineInst* __restrict__ inst, const double* __restrict__ blk, int nblk,
                                double* __restrict__ red, int* __restrict__ done, int* __restrict__ iters,
                                double* __restrict__ best, int* __restrict__ stall, int n_inst) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= n_inst) return;
  if (done && done[z]) return;
  double c = 0.0, s = 0.0, hm = INFINITY, tm = 0.0;
  for (int b = 0; b < nblk; ++b) {
    const double* p = blk + ((size_t)z * nblk + b) * 4;
    c = nan_max(c, p[0]);
    s += p[1];
    hm = fmin(hm, p[2]);
    tm = fmax(tm, p[3]);
  }
  const double force = inst[z].h * s - 0.5 * M_PI;
  red[z * 4 + 0] = c;
  red[z * 4 + 1] = force;
  red[z * 4 + 2] = s;
  red[z * 4 + 3] = hm;
  if (done) {
    const double tol = inst[z].tol;
    if (c <= tol && fabs(force) <= tol) {
      done[z] = 1;
      return;
    }
    if (!(c == c) || !(force == force)) {
      done[z] = 2;  // non-finite: stop this instance
      return;
    }
    // Rounding-floor stop: the residual has not halved for five outer
    // iterations and lies within 1e3 roundoff units of the largest term of R.
    if (best && stall) {
      if (c < 0.5 * best[z]) {
        best[z] = c;
        stall[z] = 0;
      } else {
        stall[z] += 1;
      }
      const double floor_r = 1e3 * DBL_EPSILON * tm;
      if (stall[z] >= 5 && c <= fmax(tol, floor_r) && fabs(force) <= tol) {
        done[z] = 1;
        return;
      }
    }
    if (iters) iters[z] += 1;
  }
}

// ---------------------------------------------------------------- band Jacobians
struct LineRowCtx {
  const double *rho, *drho, *deta_rel, *eps, *u, *H, *P, *psi, *psia, *psib;
  const float2* gtab;
  size_t base;  // z * N
  int N;
  double h;
  __device__ double K(int d) const {
    d = d < 0 ? -d : d;
    if (d >= N) return 0.0;
    const float2 g = gtab[base + d];
    return (double)g.x + (double)g.y;
  }
  // frozen limiter factor phi_j = psi_j / (u_j - u_{j-1})
  __device__ double phi(int j) const {
    if (j < 1) return 0.0;
    const double a = u[base + j] - u[base + j - 1];
    return a != 0.0 ? psi[base + j] / a : 0.0;
  }
  // frozen face derivative dF_{j+1/2}/dP_m (rho, phi, eps frozen); with a hybrid splitting
  // (cs > 0) the face carries cs rho_j dH_j, so that dC_i = cs (du_i - du_{i-1}) / h
  __device__ double dF_frozen(int j, int m, double cs) const {
    if (cs > 0.0) return -cs * rho[base + j] * K(j - m);
    if (j == 0) return -rho[base] * K(0 - m);
    const double ph = phi(j);
    return -rho[base + j] * (1.0 + 0.5 * ph) * K(j - m) + 0.5 * ph * rho[base + j - 1] * K(j - 1 - m);
  }
  __device__ double J_frozen(int i, int m, double ef0, double ef1, double cs) const {
    double dC = (dF_frozen(i, m, cs) - dF_frozen(i - 1, m, cs)) / h;
    double dQ = 0.0;
    if (m == i + 1) dQ = ef1 / (h * h);
    if (m == i) dQ = -(ef1 + ef0) / (h * h);
    if (m == i - 1) dQ = ef0 / (h * h);
    return dC - dQ;
  }
  // exact derivatives of the nodal u = rho H and eps with respect to P_m (m interior)
  __device__ double dU(int j, int m) const {
    double v = -rho[base + j] * K(j - m);
    if (j == m) v += drho[base + j] * H[base + j];
    return v;
  }
  __device__ double dE(int j, int m) const {
    const double e = eps[base + j];
    double v = -(3.0 * e / H[base + j]) * K(j - m);
    if (j == m) v += e * (drho[base + j] / rho[base + j] - deta_rel[base + j]);
    return v;
  }
  __device__ double dF_exact(int j, int m) const {
    const double d0 = dU(j, m);
    if (j == 0) return d0;
    return d0 + 0.5 * (psia[base + j] * (d0 - dU(j - 1, m)) + psib[base + j] * (dU(j + 1, m) - d0));
  }
  __device__ double J_exact(int i, int m, double ef0, double ef1) const {
    const double dC = (dF_exact(i, m) - dF_exact(i - 1, m)) / h;
    const double def1 = 0.5 * (dE(i, m) + dE(i + 1, m));
    const double def0 = 0.5 * (dE(i - 1, m) + dE(i, m));
    const double Pi = P[base + i];
    const double dq = def1 * (P[base + i + 1] - Pi) + ef1 * ((m == i + 1) - (m == i)) -
                      def0 * (Pi - P[base + i - 1]) - ef0 * ((m == i) - (m == i - 1));
    return dC - dq / (h * h);
  }
  // The 2b+1 band entries of row i of the exact Jacobian in double-float (the
  // same terms as J_exact, on the FP32 pipes): the nodal quantities of the
  // stencil nodes i-2..i+1 are read once per row, the kernel values once per
  // entry.  Entries whose column leaves the interior are 0.
  __device__ void J_exact_row(int i, int beta, double ef0, double ef1, double* out) const {
    df a[4], ud[4], e3[4], ed[4];  // nodes j = i-2+t: -rho_j, drho_j H_j, -3 eps_j/H_j, eps_j (drho/rho - deta)_j
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int j = i - 2 + t;
      if (j < 0) {
        a[t] = ud[t] = e3[t] = ed[t] = df_zero();
        continue;
      }
      const double rj = rho[base + j], Hj = H[base + j], ej = eps[base + j];
      a[t] = df_from_double(-rj);
      ud[t] = df_from_double(drho[base + j] * Hj);
      e3[t] = df_from_double(-3.0 * ej / Hj);
      ed[t] = df_from_double(ej * (drho[base + j] / rj - deta_rel[base + j]));
    }
    const df pa1 = df_from_double(psia[base + i]), pb1 = df_from_double(psib[base + i]);
    const df pa0 = df_from_double(i - 1 >= 1 ? psia[base + i - 1] : 0.0);
    const df pb0 = df_from_double(i - 1 >= 1 ? psib[base + i - 1] : 0.0);
    const double Pi = P[base + i];
    const df dp1 = df_from_double(P[base + i + 1] - Pi), dp0 = df_from_double(Pi - P[base + i - 1]);
    const df f1 = df_from_double(ef1), f0 = df_from_double(ef0);
    const df ih = df_from_double(1.0 / h), ih2 = df_from_double(1.0 / (h * h));
    const df half = make_df(0.5f, 0.f);
    const int n = N - 2;
    for (int e = 0; e <= 2 * beta; ++e) {
      const int m = i - beta + e;  // node of the column
      if (m < 1 || m > n) {
        out[e] = 0.0;
        continue;
      }
      df u[4], ee[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int j = i - 2 + t;
        int d = j - m;
        d = d < 0 ? -d : d;
        const df k = (j >= 0 && d < N) ? f2df_(gtab[base + d]) : df_zero();
        u[t] = df_mul(a[t], k);
        ee[t] = df_mul(e3[t], k);
        if (j == m) {
          u[t] = df_add(u[t], ud[t]);
          ee[t] = df_add(ee[t], ed[t]);
        }
      }
      // face derivatives dF_i, dF_{i-1} (limited; the first face is upwind only)
      const df F1 = df_add(u[2], df_mul(half, df_add(df_mul(pa1, df_sub(u[2], u[1])), df_mul(pb1, df_sub(u[3], u[2])))));
      const df F0 = (i - 1 == 0)
                        ? u[1]
                        : df_add(u[1], df_mul(half, df_add(df_mul(pa0, df_sub(u[1], u[0])), df_mul(pb0, df_sub(u[2], u[1])))));
      const df dC = df_mul(df_sub(F1, F0), ih);
      const df def1 = df_mul(half, df_add(ee[2], ee[3])), def0 = df_mul(half, df_add(ee[1], ee[2]));
      df dq = df_sub(df_mul(def1, dp1), df_mul(def0, dp0));
      const int s1 = (m == i + 1) - (m == i), s0 = (m == i) - (m == i - 1);
      if (s1) dq = s1 > 0 ? df_add(dq, f1) : df_sub(dq, f1);
      if (s0) dq = s0 > 0 ? df_sub(dq, f0) : df_add(dq, f0);
      out[e] = df_to_double(df_sub(dC, df_mul(dq, ih2)));
    }
  }
  __device__ static df f2df_(float2 v) { return make_df(v.x, v.y); }
  // exact and frozen dR_i/dH0
  __device__ double JH_exact(int i, double ef0, double ef1) const {
    auto dUh = [&](int j) { return rho[base + j]; };
    auto dEh = [&](int j) { return 3.0 * eps[base + j] / H[base + j]; };
    auto dFh = [&](int j) {
      const double d0 = dUh(j);
      if (j == 0) return d0;
      return d0 + 0.5 * (psia[base + j] * (d0 - dUh(j - 1)) + psib[base + j] * (dUh(j + 1) - d0));
    };
    const double dC = (dFh(i) - dFh(i - 1)) / h;
    const double Pi = P[base + i];
    const double dq = 0.5 * (dEh(i) + dEh(i + 1)) * (P[base + i + 1] - Pi) -
                      0.5 * (dEh(i - 1) + dEh(i)) * (Pi - P[base + i - 1]);
    return dC - dq / (h * h);
  }
  __device__ double JH_frozen(int i, double cs) const {
    auto dFh = [&](int j) {
      if (cs > 0.0) return cs * rho[base + j];
      if (j == 0) return rho[base];
      const double ph = phi(j);
      return rho[base + j] * (1.0 + 0.5 * ph) - 0.5 * ph * rho[base + j - 1];
    };
    return (dFh(i) - dFh(i - 1)) / h;
  }
};

// kind 1: band of the exact Jacobian, rows with P_i <= R_i / |J_ii| -> identity (kind 0, the
// paper's frozen and distributed matrix, is k_line_jac_band0 below).  One thread per row; also
// writes the exact dR/dH0 (jh) and the row scale (dg) per row.
__global__ void k_line_jac_band(const LineInst* __restrict__ inst, LineRowCtx c, const double* __restrict__ R,
                                const int* __restrict__ skip, int beta, double* __restrict__ band,
                                uint8_t* __restrict__ act, double* __restrict__ jh, double* __restrict__ dg) {
  const int z = blockIdx.y;
  if (skip && skip[z]) return;
  const int N = c.N, n = N - 2;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  LineRowCtx q = c;
  q.base = (size_t)z * N;
  q.h = inst[z].h;
  const int i = r + 1;
  const int bw = 2 * beta + 1;
  double* row = band + ((size_t)z * n + r) * bw;
  const double ef1 = 0.5 * (c.eps[q.base + i] + c.eps[q.base + i + 1]);
  const double ef0 = 0.5 * (c.eps[q.base + i - 1] + c.eps[q.base + i]);
  const double Pi = c.P[q.base + i], Ri = R[q.base + i];
  // row scale d = max(|J_ii|, |J_i|_max / 10) over the band: |J_ii| alone can pass
  // through zero in the Hertzian zone, where the row is carried by its neighbours
  double rmax = 0.0, jii = 0.0;
  q.J_exact_row(i, beta, ef0, ef1, row);
  for (int j = 0; j < bw; ++j) {
    const double v = row[j];
    rmax = fmax(rmax, fabs(v));
    if (j == beta) jii = v;
  }
  double d = fmax(fabs(jii), 0.1 * rmax);
  d = d > 0.0 ? d : 1.0;
  const bool a = Pi <= Ri / d;
  if (a)
    for (int j = 0; j < bw; ++j) row[j] = (j == beta ? 1.0 : 0.0);
  if (jh) jh[(size_t)z * n + r] = a ? 0.0 : q.JH_exact(i, ef0, ef1);
  if (dg) dg[(size_t)z * n + r] = d;
  act[(size_t)z * n + r] = a ? 1 : 0;
}

// kind 0 with one thread per band entry: a row's 2b+1 entries, each with its distributed
// neighbours, are independent chains of float64 divisions (FP64 latency, not throughput, sets
// the time of a row), so each entry gets its own thread; the entries are computed by the same
// code as in k_line_jac_band.  The thread of the diagonal entry also writes the row's dR/dH0
// and flag and, when asked, the paper iteration's right-hand side and PAQIF's int32 flag.
__global__ void k_line_jac_band0(const LineInst* __restrict__ inst, LineRowCtx c, const double* __restrict__ R,
                                 const int* __restrict__ skip, int beta, double* __restrict__ band,
                                 uint8_t* __restrict__ act, double* __restrict__ jh, double* __restrict__ rhs_out,
                                 int* __restrict__ act32) {
  const int z = blockIdx.y;
  if (skip && skip[z]) return;
  const int N = c.N, n = N - 2;
  const int bw = 2 * beta + 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * bw) return;
  const int r = t / bw, j = t % bw;
  LineRowCtx q = c;
  q.base = (size_t)z * N;
  q.h = inst[z].h;
  const int i = r + 1;
  const double ef1 = 0.5 * (c.eps[q.base + i] + c.eps[q.base + i + 1]);
  const double ef0 = 0.5 * (c.eps[q.base + i - 1] + c.eps[q.base + i]);
  const double Pi = c.P[q.base + i], Ri = R[q.base + i];
  const bool a = (Pi <= 0.0) && (Ri > 0.0);
  const double w = inst[z].dist_w, sw = inst[z].switch_eps_h;
  const double cs = line_split_coef(inst[z]);
  const int col = r - beta + j;  // interior column index, node col + 1
  double v = 0.0;
  if (col >= 0 && col < n) {
    const int m = col + 1;
    v = q.J_frozen(i, m, ef0, ef1, cs);
    if (c.eps[q.base + m] / q.h <= sw) {
      if (m - 1 >= 1) v -= w * q.J_frozen(i, m - 1, ef0, ef1, cs);
      if (m + 1 <= N - 2) v -= w * q.J_frozen(i, m + 1, ef0, ef1, cs);
    }
  }
  band[((size_t)z * n + r) * bw + j] = a ? (j == beta ? 1.0 : 0.0) : v;
  if (j != beta) return;
  const size_t o = (size_t)z * n + r;
  if (jh) jh[o] = a ? 0.0 : q.JH_frozen(i, cs);
  act[o] = a ? 1 : 0;
  if (rhs_out) rhs_out[o] = a ? 0.0 : -Ri;
  if (act32) act32[o] = a ? 1 : 0;
}

// ---------------------------------------------------------------- paper relaxation
__global__ void k_line_paper_rhs(const double* __restrict__ R, const uint8_t* __restrict__ act,
                                 const int* __restrict__ skip, double* __restrict__ rhs, int N) {
  const int z = blockIdx.y, n = N - 2;
  if (skip && skip[z]) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  rhs[(size_t)z * n + r] = act[(size_t)z * n + r] ? 0.0 : -R[(size_t)z * N + r + 1];
}

// H0 - c (pi/2 - h s), s = h-less sum of P (Sec. 3.3.4, Eq. eqn75 with the line-contact load)
__device__ __forceinline__ double line_h0_step(const LineInst& q, double H0, double s) {
  return H0 - q.c_h0 * (0.5 * M_PI - q.h * s);
}

// P <- max(0, P + omega D sigma) (Sec. 3.3.4, Eq. eqn69); block partial sums of the new P
// (one thread per node, the same blocks as k_line_residual)
__global__ void __launch_bounds__(kNodeBlock) k_line_paper_update(const LineInst* __restrict__ inst,
                                                                  const double* __restrict__ sigma,
                                                                  const double* __restrict__ eps,
                                                                  const int* __restrict__ skip,
                                                                  double* __restrict__ P, double* __restrict__ blk,
                                                                  int nblk, int N, double* __restrict__ H0) {
  const int z = blockIdx.y, n = N - 2;
  if (skip && skip[z]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = i - 1;  // interior index
  const LineInst q = inst[z];
  double pn = 0.0;
  if (r >= 0 && r < n) {
    const size_t so = (size_t)z * n;
    double dp = sigma[so + r];
    for (int cc = r - 1; cc <= r + 1; cc += 2) {
      if (cc < 0 || cc >= n) continue;
      if (eps[(size_t)z * N + cc + 1] / q.h <= q.switch_eps_h) dp -= q.dist_w * sigma[so + cc];
    }
    const size_t o = (size_t)z * N + i;
    pn = P[o] + q.omega * dp;
    pn = pn > 0.0 ? pn : 0.0;
    P[o] = pn;
  }
  __shared__ double s[kNodeBlock];
  s[threadIdx.x] = pn;
  __syncthreads();
  for (int w = kNodeBlock / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) blk[((size_t)z * nblk + blockIdx.x) * 4 + 1] = s[0];
  // one block holds the whole sum: the H0 update of k_line_h0_update here
  if (H0 && nblk == 1 && threadIdx.x == 0) {
    double t = 0.0;
    t += s[0];
    H0[z] = line_h0_step(q, H0[z], t);
  }
}

// H0 <- H0 - c (pi/2 - h sum P)   (Sec. 3.3.4, Eq. eqn75 with the line-contact load)
__global__ void k_line_h0_update(const LineInst* __restrict__ inst, const double* __restrict__ blk, int nblk,
                                 const int* __restrict__ skip, double* __restrict__ H0, int n_inst) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= n_inst || (skip && skip[z])) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += blk[((size_t)z * nblk + b) * 4 + 1];
  H0[z] = line_h0_step(inst[z], H0[z], s);
}

// ---------------------------------------------------------------- start
__global__ void k_line_hertz(const LineInst* __restrict__ inst, double* __restrict__ P, int N) {
  const int z = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double X = inst[z].xa + i * inst[z].h;
  double v = 1.0 - X * X;
  P[(size_t)z * N + i] = (i == 0 || i == N - 1 || v <= 0.0) ? 0.0 : sqrt(v);
}

__global__ void k_line_set_h0(const LineInst* __restrict__ inst, const double* __restrict__ blk, int nblk,
                              double* __restrict__ H0, int n_inst) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= n_inst) return;
  double hm = INFINITY;
  for (int b = 0; b < nblk; ++b) hm = fmin(hm, blk[((size_t)z * nblk + b) * 4 + 2]);
  H0[z] = inst[z].h_init - hm;  // the film was evaluated with H0 = 0
}

// ================================================================= host side
cudaError_t ctx_alloc(LineCtx* c, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 16);
  if (e == cudaSuccess) c->allocs.push_back(*p);
  return e;
}

LineRowCtx line_row_ctx(LineCtx* c) {
  LineRowCtx q;
  q.rho = c->rho;
  q.drho = c->drho;
  q.deta_rel = c->deta_rel;
  q.eps = c->eps;
  q.u = c->u;
  q.H = c->H;
  q.P = nullptr;
  q.psi = c->psi;
  q.psia = c->psia;
  q.psib = c->psib;
  q.gtab = c->gtab;
  q.base = 0;
  q.N = c->N;
  q.h = 0.0;
  return q;
}

// deformation of the nodal vectors V [n_inst][vstride] -> c->partial
cudaError_t line_deform(LineCtx* c, const double* V, int vstride, const int* skip) {
  dim3 g((c->N + kDefTI - 1) / kDefTI, c->ksplit, c->n_inst);
  k_line_deform<<<g, kDefTI, 0, c->st>>>(c->inst, c->gtab, V, vstride, skip, c->partial, c->n_inst, c->N);
  note_launch();
  return cudaGetLastError();
}

// film + lubricant state + faces + residual + reductions at (P, H0)
cudaError_t line_deform64(LineCtx* c, const double* V, int vstride, const int* skip) {
  dim3 g((c->N + kDefTI - 1) / kDefTI, c->ksplit, c->n_inst);
  k_line_deform64<<<g, kDefTI, 0, c->st>>>(c->inst, c->gtab64, V, vstride, skip,
                                           reinterpret_cast<double*>(c->partial), c->n_inst, c->N);
  note_launch();
  return cudaGetLastError();
}

cudaError_t line_state(LineCtx* c, const double* P, const double* H0, const double* rough, const int* skip,
                       int* iters_done_flag_mode) {
  cudaError_t e = line_deform64(c, P, c->N, skip);
  if (e != cudaSuccess) return e;
  if (c->fuse && c->N <= kNodeBlock) {
    k_line_state_small<<<c->n_inst, kNodeBlock, 0, c->st>>>(
        c->inst, reinterpret_cast<const double*>(c->partial), c->ksplit, H0, rough, P, skip, c->H, c->rho, c->drho,
        c->deta_rel, c->eps, c->u, c->F, c->psi, c->psia, c->psib, c->R, c->blk, c->n_inst, c->N);
    note_launch();
    return cudaGetLastError();
  }
  dim3 gn((c->N + kNodeBlock - 1) / kNodeBlock, c->n_inst);
  k_line_film<<<gn, kNodeBlock, 0, c->st>>>(c->inst, c->partial, c->ksplit, H0, rough, c->N, skip, c->H,
                                             c->n_inst, c->N, 0, 1);
  note_launch();
  k_line_nodes<<<gn, kNodeBlock, 0, c->st>>>(c->inst, P, c->H, skip, c->rho, c->drho, c->deta_rel, c->eps, c->u,
                                              c->N);
  note_launch();
  k_line_faces<<<gn, kNodeBlock, 0, c->st>>>(c->inst, c->u, skip, c->F, c->psi, c->psia, c->psib, c->N);
  note_launch();
  k_line_residual<<<gn, kNodeBlock, 0, c->st>>>(c->inst, P, c->H, c->eps, c->F, skip, c->R, c->blk, c->nblk, c->N);
  note_launch();
  (void)iters_done_flag_mode;
  return cudaGetLastError();
}

cudaError_t line_finalize(LineCtx* c, int* done, int* iters) {
  k_line_finalize<<<(c->n_inst + 127) / 128, 128, 0, c->st>>>(
      c->inst, c->blk, c->nblk, c->red, done, iters, done ? c->best : nullptr, done ? c->stall : nullptr, c->n_inst);
  note_launch();
  return cudaGetLastError();
}

cudaError_t line_jac_band(LineCtx* c, const double* P, int kind, double* band, uint8_t* act, double* jh,
                          double* dg, const int* skip, double* rhs_out, int* act32) {
  LineRowCtx q = line_row_ctx(c);
  q.P = P;
  if (kind == 0) {  // one thread per band entry
    const long long entries = (long long)c->n * (2 * c->beta + 1);
    dim3 g((unsigned)((entries + 127) / 128), c->n_inst);
    k_line_jac_band0<<<g, 128, 0, c->st>>>(c->inst, q, c->R, skip, c->beta, band, act, jh, rhs_out, act32);
    note_launch();
    return cudaGetLastError();
  }
  dim3 g((c->n + 127) / 128, c->n_inst);
  k_line_jac_band<<<g, 128, 0, c->st>>>(c->inst, q, c->R, skip, c->beta, band, act, jh, dg);
  note_launch();
  return cudaGetLastError();
}

cudaError_t line_start(LineCtx* c, double* P, double* H0, const double* rough) {
  dim3 gn((c->N + kNodeBlock - 1) / kNodeBlock, c->n_inst);
  k_line_hertz<<<gn, kNodeBlock, 0, c->st>>>(c->inst, P, c->N);
  note_launch();
  cudaError_t e = cudaMemsetAsync(H0, 0, sizeof(double) * c->n_inst, c->st);
  if (e != cudaSuccess) return e;
  e = line_state(c, P, H0, rough, nullptr, nullptr);
  if (e != cudaSuccess) return e;
  k_line_set_h0<<<(c->n_inst + 127) / 128, 128, 0, c->st>>>(c->inst, c->blk, c->nblk, H0, c->n_inst);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------ grid sequence
__global__ void k_line_inject(const double* __restrict__ src, int Nf, double* __restrict__ dst, int Nc, int stride) {
  const int z = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < Nc) dst[(size_t)z * Nc + i] = src[(size_t)z * Nf + (size_t)i * stride];
}

cudaError_t line_inject(const double* src, int Nf, double* dst, int Nc, int n_inst, cudaStream_t st) {
  if (Nc < 2 || (Nf - 1) % (Nc - 1) != 0) return cudaErrorInvalidValue;
  dim3 g((Nc + 255) / 256, n_inst);
  k_line_inject<<<g, 256, 0, st>>>(src, Nf, dst, Nc, (Nf - 1) / (Nc - 1));
  note_launch();
  return cudaGetLastError();
}

// fine node 2i = coarse node i; fine node 2i+1 = mean of coarse nodes i, i+1
__global__ void k_line_prolong(const double* __restrict__ Pc, const double* __restrict__ H0c,
                               const int* __restrict__ cdone, int Nc, double* __restrict__ Pf,
                               double* __restrict__ H0f) {
  const int z = blockIdx.y;
  if (cdone && cdone[z] != 1) return;  // only a converged coarse solve seeds the finer grid
  const int Nf = 2 * Nc - 1;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Nf) return;
  const double* pc = Pc + (size_t)z * Nc;
  const int i = j >> 1;
  Pf[(size_t)z * Nf + j] = (j & 1) ? 0.5 * (pc[i] + pc[i + 1]) : pc[i];
  if (j == 0) H0f[z] = H0c[z];
}

cudaError_t line_prolong(const double* Pc, const double* H0c, const int* cdone, int Nc, double* Pf, double* H0f,
                         int n_inst, cudaStream_t st) {
  const int Nf = 2 * Nc - 1;
  dim3 g((Nf + 255) / 256, n_inst);
  k_line_prolong<<<g, 256, 0, st>>>(Pc, H0c, cdone, Nc, Pf, H0f);
  note_launch();
  return cudaGetLastError();
}

// the paper's iteration: band Newton step with the frozen / distributed Jacobian,
// PAQIF solve, projected distributed update, H0 relaxation
cudaError_t line_paper_iteration(LineCtx* c, double* P, double* H0, const double* rough) {
  cudaError_t e = line_state(c, P, H0, rough, c->done, nullptr);
  if (e != cudaSuccess) return e;
  e = line_finalize(c, c->done, c->iters);
  if (e != cudaSuccess) return e;
  int* act32 = (int*)((unsigned char*)c->pq_ws + align_up(paqif_stack_bytes(c->n_inst, c->n, c->beta), kWorkspaceAlign));
  // with fuse the band kernel also writes the right-hand side and PAQIF's row flags, and the
  // update kernel of a one-block instance updates H0 (the same values, three launches fewer)
  e = line_jac_band(c, P, 0, c->band, c->act, nullptr, nullptr, c->done, c->fuse ? c->rhs : nullptr,
                    c->fuse ? act32 : nullptr);
  if (e != cudaSuccess) return e;
  if (!c->fuse) {
    dim3 g((c->n + 127) / 128, c->n_inst);
    k_line_paper_rhs<<<g, 128, 0, c->st>>>(c->R, c->act, c->done, c->rhs, c->N);
    note_launch();
  }
  PaqifLaunch L;
  L.n_sys = c->n_inst;
  L.n = c->n;
  L.beta = c->beta;
  L.mode = 0;
  L.band = c->band;
  L.rhs = c->rhs;
  L.act = act32;
  L.stack = c->pq_ws;
  L.x = c->sigma;
  L.iters = nullptr;
  L.info = c->pq_info;
  if (!c->fuse) {
    e = launch_expand_active(c->act, L.act, (size_t)c->n_inst * c->n, c->st);
    if (e != cudaSuccess) return e;
  }
  e = launch_paqif(L, c->st);
  if (e != cudaSuccess) return e;
  const bool h0_here = c->fuse && c->nblk == 1;
  dim3 gu((c->N + kNodeBlock - 1) / kNodeBlock, c->n_inst);
  k_line_paper_update<<<gu, kNodeBlock, 0, c->st>>>(c->inst, c->sigma, c->eps, c->done, P, c->blk, c->nblk, c->N,
                                                     h0_here ? H0 : nullptr);
  note_launch();
  if (!h0_here) {
    k_line_h0_update<<<(c->n_inst + 127) / 128, 128, 0, c->st>>>(c->inst, c->blk, c->nblk, c->done, H0, c->n_inst);
    note_launch();
  }
  return cudaGetLastError();
}

// The paper's iteration of one grid as one graph: a while-node whose body is one pass of
// line_paper_iteration and whose condition k_nk_loop sets on the device (some instance not done
// and fewer than max_iter passes), then the state and reductions at the final iterate, as the
// host-driven loop ends.  Same kernels, same order, so the same iterates.
cudaError_t line_paper_capture_solve(LineCtx* c, double* P, double* H0, const double* rough, cudaStream_t s1,
                                     SolveGraphCounts& n) {
  const int ni = c->n_inst;
  const cudaStream_t s0 = c->st;
  c->capturing = true;
  const unsigned long long l0 = thread_launches();
  // fresh flags, no residual seen yet (bytes 0x7f: 1.4e306), no stall, pass counter 0
  cudaError_t e = cudaMemsetAsync(c->done, 0, sizeof(int) * ni, s0);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->iters, 0, sizeof(int) * ni, s0);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->best, 0x7f, sizeof(double) * ni, s0);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->stall, 0, sizeof(int) * ni, s0);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->loop0, 0, sizeof(int) * 8, s0);
  auto loop = [&](cudaGraphConditionalHandle h, int next) -> cudaError_t {
    k_nk_loop<<<1, 256, 0, c->st>>>(h, c->loop0, nullptr, c->max_iter, next, c->done, nullptr, ni);
    note_launch();
    return cudaGetLastError();
  };
  long long body = 0;
  if (e == cudaSuccess)
    e = capture_while(
        c, s0, s1, [&](cudaGraphConditionalHandle h) { return loop(h, 0); },
        [&](cudaGraphConditionalHandle h) {
          cudaError_t ee = line_paper_iteration(c, P, H0, rough);
          return ee == cudaSuccess ? loop(h, 1) : ee;
        },
        &body);
  c->st = s0;
  if (e == cudaSuccess) e = line_state(c, P, H0, rough, nullptr, nullptr);
  if (e == cudaSuccess) e = line_finalize(c, nullptr, nullptr);
  c->capturing = false;
  n = SolveGraphCounts();
  n.newton = body;
  n.fixed = (long long)(thread_launches() - l0) - body;
  return e;
}

}  // namespace ehl

namespace ehl {
// ------------------------------------------------ mixed-precision Krylov products
// K as a dense float32 matrix (column-major, symmetric) from the float64 table of instance 0
__global__ void k_line_kfull(const double* __restrict__ gtab64, float* __restrict__ Kf, int N) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)N * N) return;
  const int i = (int)(t % N), k = (int)(t / N);
  Kf[t] = (float)gtab64[i > k ? i - k : k - i];
}

__global__ void k_line_to_f32(const double* __restrict__ V, int vstride, float* __restrict__ Vf, int N) {
  const int z = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) Vf[(size_t)z * N + i] = (float)V[(size_t)z * vstride + i];
}

cudaError_t line_mixed_init(LineCtx* c, int precision) {
  c->precision = 0;
  if (precision <= 0) return cudaSuccess;
  // one K for the bucket: every instance must share the grid spacing
  for (const LineInst& q : c->h_inst)
    if (q.h != c->h_inst[0].h || q.elastic != c->h_inst[0].elastic) return cudaSuccess;
  if (!c->h_inst[0].elastic) return cudaSuccess;
  if (precision == 5) return line_tc_init(c);
  const size_t NN = (size_t)c->N * c->N, NI = (size_t)c->N * c->n_inst;
  cudaError_t e = ctx_alloc(c, (void**)&c->Kf, sizeof(float) * NN);
  if (e == cudaSuccess) e = ctx_alloc(c, (void**)&c->Vf, sizeof(float) * NI);
  if (e == cudaSuccess) e = ctx_alloc(c, (void**)&c->Df, sizeof(float) * NI);
  if (e != cudaSuccess) return e;
  if (cublasCreate(&c->blas) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
  cublasSetStream(c->blas, c->st);
  // a workspace of its own, so that no GEMM allocates (also inside a graph capture)
  void* ws = nullptr;
  const size_t wsb = (size_t)32 << 20;
  e = ctx_alloc(c, &ws, wsb);
  if (e != cudaSuccess) return e;
  cublasSetWorkspace(c->blas, ws, wsb);
  cublasSetMathMode(c->blas, CUBLAS_DEFAULT_MATH);
  // precision 2 asks for the BF16x9 tensor-core emulation with the eager strategy (cuBLAS
  // still runs SIMT SGEMM kernels for these shapes, N x n_inst x N with odd N)
  if (precision == 2) cublasSetEmulationStrategy(c->blas, CUBLAS_EMULATION_STRATEGY_EAGER);
  k_line_kfull<<<(unsigned)((NN + 255) / 256), 256, 0, c->st>>>(c->gtab64, c->Kf, c->N);
  note_launch();
  c->precision = precision;
  return cudaGetLastError();
}

void line_mixed_free(LineCtx* c) {
  if (c->blas) cublasDestroy(c->blas);
  c->blas = nullptr;
  delete reinterpret_cast<TcGemm*>(c->tc);
  c->tc = nullptr;
}

// precision 5: K [N][ld] and the vectors [n_inst][ld] as tf32 hi / lo parts, the tcgen05 plan and
// K-splits enough to give the 152 SMs about one tile each
cudaError_t line_tc_init(LineCtx* c) {
  const int N = c->N, ni = c->n_inst, ld = tc_ld(N);
  const int tiles = ((N + 127) / 128) * ((ni + 127) / 128);
  const int ktiles = (N + 31) / 32;
  int splits = kSmCount / (tiles > 0 ? tiles : 1);
  splits = splits < 1 ? 1 : (splits > ktiles ? ktiles : splits);
  cudaError_t e = ctx_alloc(c, (void**)&c->Khi, sizeof(float) * (size_t)N * ld);
  if (e == cudaSuccess) e = ctx_alloc(c, (void**)&c->Klo, sizeof(float) * (size_t)N * ld);
  if (e == cudaSuccess) e = ctx_alloc(c, (void**)&c->Vhi, sizeof(float) * (size_t)ni * ld);
  if (e == cudaSuccess) e = ctx_alloc(c, (void**)&c->Vlo, sizeof(float) * (size_t)ni * ld);
  if (e == cudaSuccess) e = ctx_alloc(c, (void**)&c->Df, sizeof(float) * (size_t)splits * ni * N);
  if (e == cudaSuccess) e = ctx_alloc(c, (void**)&c->tc_err, sizeof(int));
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(c->tc_err, 0, sizeof(int), c->st);
  // the padding columns N..ld-1 are never read (the tensor maps end at column N)
  if (e == cudaSuccess) e = tc_toeplitz(c->gtab64, N, c->Khi, c->Klo, ld, c->st);
  if (e != cudaSuccess) return e;
  TcGemm* g = new TcGemm();
  e = tc_gemm_init(*g, c->Khi, c->Klo, c->Vhi, c->Vlo, N, ni, N, ld, ld, c->Df, N, splits);
  if (e != cudaSuccess) {
    delete g;
    return e;
  }
  c->tc = g;
  c->tc_splits = g->splits;
  c->precision = 5;
  return cudaSuccess;
}

// dH = -K v + zh0 for the Krylov vectors: the double-float Toeplitz kernel, or
// with precision > 0 one float32-output GEMM K [N x N] . V [N x n_inst] of the
// whole bucket (precision 1 float32, 2 float32 with the BF16x9 emulation
// requested -- cuBLAS runs SIMT SGEMM kernels for these shapes --, 3 TF32, 4 BF16).
cudaError_t line_krylov_deform(LineCtx* c, const double* V, const double* zh0, const int* skip) {
  if (c->precision <= 0) {
    cudaError_t e = line_deform(c, V, c->N, skip);
    if (e == cudaSuccess) e = line_film_dir(c, zh0, skip);
    return e;
  }
  const int N = c->N, ni = c->n_inst;
  if (c->precision == 5) {
    // TF32x3 on the tensor cores: D[s][z][i] partial sums of K V over the K-splits
    const TcGemm& tg = *reinterpret_cast<const TcGemm*>(c->tc);
    cudaError_t e = tc_split(V, N, ni, N, c->Vhi, c->Vlo, tc_ld(N), c->st);
    if (e == cudaSuccess) e = tc_gemm_run(tg, c->tc_err, c->st);
    if (e != cudaSuccess) return e;
    dim3 gn((N + kNodeBlock - 1) / kNodeBlock, ni);
    k_line_film<<<gn, kNodeBlock, 0, c->st>>>(c->inst, reinterpret_cast<const float2*>(c->Df), tg.splits, zh0, nullptr,
                                               N, skip, c->dH, ni, N, 1, 3);
    note_launch();
    return cudaGetLastError();
  }
  dim3 g((N + 255) / 256, ni);
  k_line_to_f32<<<g, 256, 0, c->st>>>(V, N, c->Vf, N);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cublasComputeType_t ct = CUBLAS_COMPUTE_32F;
  if (c->precision == 2) ct = CUBLAS_COMPUTE_32F_EMULATED_16BFX9;
  if (c->precision == 3) ct = CUBLAS_COMPUTE_32F_FAST_TF32;
  if (c->precision == 4) ct = CUBLAS_COMPUTE_32F_FAST_16BF;
  const float one = 1.0f, zero = 0.0f;
  if (cublasGemmEx(c->blas, CUBLAS_OP_N, CUBLAS_OP_N, N, ni, N, &one, c->Kf, CUDA_R_32F, N, c->Vf, CUDA_R_32F, N,
                   &zero, c->Df, CUDA_R_32F, N, ct, CUBLAS_GEMM_DEFAULT) != CUBLAS_STATUS_SUCCESS)
    return cudaErrorUnknown;
  dim3 gn((N + kNodeBlock - 1) / kNodeBlock, ni);
  k_line_film<<<gn, kNodeBlock, 0, c->st>>>(c->inst, reinterpret_cast<const float2*>(c->Df), 1, zh0, nullptr, N,
                                             skip, c->dH, ni, N, 1, 2);
  note_launch();
  return cudaGetLastError();
}

cudaError_t line_film_dir(LineCtx* c, const double* zh0, const int* skip, bool p64) {
  dim3 gn((c->N + kNodeBlock - 1) / kNodeBlock, c->n_inst);
  k_line_film<<<gn, kNodeBlock, 0, c->st>>>(c->inst, c->partial, c->ksplit, zh0, nullptr, c->N, skip, c->dH,
                                             c->n_inst, c->N, 1, p64 ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

cudaError_t line_init_tables(LineCtx* c) {
  dim3 g((c->N + 255) / 256, c->n_inst);
  k_line_gtab<<<g, 256, 0, c->st>>>(c->inst, c->gtab, c->gtab64, c->N);
  note_launch();
  return cudaGetLastError();
}
}  // namespace ehl
