// paqif3.cu -- batched PAQIF (projected alternate quadrant interlocking factorization).
//
// Method (Sec. 2.2.1-2.2.3; projection of Sec. 2.2.2 / Sec. 2.2.4 Steps 5
// and 7 after the solve, one partition per system): for n = 2s, level
// k = 1..s pivots on rows/columns (s-k+1, s+k) of the Schur complement
// L0^(k); the Z0 rows are the pivot rows, the W0 columns solve
//   z_pp w_ip + z_qp w_iq = l_ip,   z_pq w_ip + z_qq w_iq = l_iq,
// and L0^(k+1) = L0^(k) - w_p z_p^T - w_q z_q^T.  W0 Y = F runs in the same
// middle-out sweep; Z0 U = Y runs from both ends towards the middle with one
// 2x2 solve per level.
//
// GB300 mapping:
//  * for half-band b only the window of the Schur complement on rows/columns
//    {p-b..p} u {q..q+b} is non-trivial.  It lives in shared memory with the
//    right-hand side appended as one more column, so the W0 Y = F sweep is
//    part of the rank-2 update.  Rows/columns form a ring per side (index
//    mod (b+1)); the ring offset advances by one each level.
//  * a group of LS lanes serves one system (32/LS systems per warp).  Per
//    level the lanes share one task list: the 2b outer-row multipliers and
//    the 2b+1 folded outer columns Pi^-1 [z_p; z_q] (the last one is Pi^-1 y),
//    then the (2b) x (2b+1) rank-2 update, then the two incoming rows and
//    columns -- the same instruction stream on every lane.
//  * band rows stream from HBM with cp.async into a 32-row ring per side,
//    16 levels ahead, and are converted float64 -> double-float once, in
//    place, by the lane that copied them;
//  * the folded columns go to a per-system stack; the Z0 sweep reads it back
//    in reverse and pushes each solved pair of unknowns into accumulators of
//    the b levels below, so a level costs one double-float FMA per lane;
//  * arithmetic is double-float (df64.cuh); float64 only at the interface.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "df64.cuh"
#include "ehl_internal.h"

namespace ehl {

template <int B>
struct C3 {
  static constexpr int W = B + 1;        // ring slots per side
  static constexpr int NS = 2 * W;       // window rows
  static constexpr int NC = NS + 1;      // window columns (rhs appended)
  static constexpr int BW = 2 * B + 1;   // band row width
  static constexpr int NO = 2 * B;       // outer rows per level
  static constexpr int NOC = NO + 1;     // outer columns per level (rhs included)
  static constexpr int LS = (B == 1) ? 4 : (B <= 3 ? 8 : (B <= 6 ? 16 : 32));
  static constexpr int G = 32 / LS;      // systems per warp
  static constexpr int RB = 32;          // ring rows per side
  static constexpr int CH = 8;           // rows per chunk
  static constexpr int SL = NOC;         // float4 per stack level: (Mp, Mq) per outer column
  static constexpr int FL = NO + 2;      // float4 per factor-store level: (w_p, w_q) per outer row, Pi^-1
  static constexpr int NT1 = NO + NOC;   // multiplier + folded-column tasks
  static constexpr int R1 = (NT1 + LS - 1) / LS;
  static constexpr int NUP = NO * NOC;   // update entries
  static constexpr int RU = (NUP + LS - 1) / LS;
  static constexpr int NNEW = 2 * (NC + NS);  // entries of the two incoming rows and columns
  static constexpr int RN = (NNEW + LS - 1) / LS;
  static constexpr int WARPS = 4;
};

template <int B>
struct __align__(16) Sm3 {
  using C = C3<B>;
  float2 S[C::NS][C::NC];  // window (double-float), column NS is the rhs
  float2 w[C::NO][2];      // multipliers (w_ip, w_iq) of the outer rows
  float2 acc[C::W][2];     // phase 2: accumulators of the next b levels per side
  float2 xpq[2];           // phase 2: the pair solved last
  int kind[C::NS];         // row kind of each window slot (0 outside, 1 real, 2 identity)
  union {
    double ring[2][C::RB][C::BW];  // band rows: float64 as copied, double-float after conversion
    float4 stk[C::RB][C::SL];      // phase 2: stack levels
    float4 fr[C::RB][C::FL];       // solve-only W0 sweep: factor-store levels
  } u;
  double rrhs[2][C::RB];
  int ract[2][C::RB];
};

struct Paqif3Args {
  int n_sys, n, s, mode;
  const double* band;
  const double* rhs;
  int* act;
  float4* stack;   // [pad_sys][s][SL]
  float4* fstore;  // [pad_sys][s][FL]: outer-row multipliers and Pi^-1 (factor once, solve many), or null
  double* x;
  int* iters;
  int* info;
};

__device__ __forceinline__ void cpa8(void* smem, const void* gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cpa16cg(void* smem, const void* gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ df f2df(float2 v) { return make_df(v.x, v.y); }
__device__ __forceinline__ float2 df2f(df v) { return make_float2(v.hi, v.lo); }

// Arithmetic of the sweeps: double-float (F32 = false, about 48 bits) or plain
// float32 in the hi word (F32 = true: the Krylov preconditioner of the mixed-
// precision path, whose accuracy GMRES absorbs).  Storage is double-float in
// both cases (lo = 0 for float32).
template <bool F32>
struct Ar {
  static __device__ __forceinline__ df det2(df a, df d, df b, df c) { return df_det2(a, d, b, c); }
  static __device__ __forceinline__ df mul(df a, df b) { return df_mul(a, b); }
  static __device__ __forceinline__ df rcp(df a) { return df_rcp(a); }
  static __device__ __forceinline__ df sub_two_prods(df s, df w0, df z0, df w1, df z1) {
    return df_sub_two_prods(s, w0, z0, w1, z1);
  }
  static __device__ __forceinline__ df sub(df a, df b) { return df_sub(a, b); }
  static __device__ __forceinline__ df fma(df a, df b, df c) { return df_fma(a, b, c); }
  static __device__ __forceinline__ df from_double(double x) { return df_from_double(x); }
  static __device__ __forceinline__ double to_double(df a) { return df_to_double(a); }
};
template <>
struct Ar<true> {
  static __device__ __forceinline__ df det2(df a, df d, df b, df c) {
    return make_df(__fmaf_rn(a.hi, d.hi, -__fmul_rn(b.hi, c.hi)), 0.f);
  }
  static __device__ __forceinline__ df mul(df a, df b) { return make_df(__fmul_rn(a.hi, b.hi), 0.f); }
  static __device__ __forceinline__ df rcp(df a) { return make_df(__frcp_rn(a.hi), 0.f); }
  static __device__ __forceinline__ df sub_two_prods(df s, df w0, df z0, df w1, df z1) {
    return make_df(__fmaf_rn(-w1.hi, z1.hi, __fmaf_rn(-w0.hi, z0.hi, s.hi)), 0.f);
  }
  static __device__ __forceinline__ df sub(df a, df b) { return make_df(__fsub_rn(a.hi, b.hi), 0.f); }
  static __device__ __forceinline__ df fma(df a, df b, df c) { return make_df(__fmaf_rn(a.hi, b.hi, c.hi), 0.f); }
  static __device__ __forceinline__ df from_double(double x) { return make_df((float)x, 0.f); }
  static __device__ __forceinline__ double to_double(df a) { return (double)a.hi; }
};

template <int B, bool F32>
struct P3 {
  using C = C3<B>;
  using A = Ar<F32>;

  static __device__ __forceinline__ int row_of(int side, int t, int s) { return side ? s + t : s - 1 - t; }
  static __device__ __forceinline__ int wrap(int x) { return x >= C::W ? x - C::W : x; }

  // Copy (CONVERT = false) or convert in place (CONVERT = true) chunk c of
  // both sides; the lane of rank u handles elements u, u + LS, ...
  template <bool CONVERT>
  static __device__ __forceinline__ void chunk(Sm3<B>& sm, const Paqif3Args& a, int dsys, int c, int u) {
    const int s = a.s, n = a.n;
    const double* bsys = a.band + (size_t)dsys * n * C::BW;
    const double* rsys = a.rhs + (size_t)dsys * n;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int t0 = c * C::CH;
      int r_lo = side ? s + t0 : s - 1 - (t0 + C::CH - 1);
      int r_hi = side ? s + t0 + C::CH - 1 : s - 1 - t0;
      r_lo = max(r_lo, 0);
      r_hi = min(r_hi, n - 1);
      if (r_lo > r_hi) continue;
      const int nel = (r_hi - r_lo + 1) * C::BW;
      for (int e = u; e < nel; e += C::LS) {
        const int r = r_lo + e / C::BW, col = e % C::BW;
        const int t = side ? r - s : s - 1 - r;
        double* dst = &sm.u.ring[side][t & (C::RB - 1)][col];
        if (CONVERT) {
          const df v = A::from_double(*dst);
          *reinterpret_cast<float2*>(dst) = make_float2(v.hi, v.lo);
        } else {
          cpa8(dst, bsys + (size_t)r * C::BW + col);
        }
      }
      for (int r = r_lo + u; r <= r_hi; r += C::LS) {
        const int t = side ? r - s : s - 1 - r;
        double* dst = &sm.rrhs[side][t & (C::RB - 1)];
        if (CONVERT) {
          const df v = A::from_double(*dst);
          *reinterpret_cast<float2*>(dst) = make_float2(v.hi, v.lo);
          sm.ract[side][t & (C::RB - 1)] = a.act ? __ldcg(a.act + (size_t)dsys * n + r) : 0;
        } else {
          cpa8(dst, rsys + r);
        }
      }
    }
  }

  // 0: outside the matrix, 1: a real row, 2: an identity row (padding or active)
  static __device__ __forceinline__ int row_kind(const Sm3<B>& sm, int side, int t, int s, int n) {
    const int i = row_of(side, t, s);
    if (i < 0 || i >= 2 * s) return 0;
    if (i >= n) return 2;
    return sm.ract[side][t & (C::RB - 1)] ? 2 : 1;
  }

  // A[(side, tr)][(side, tc)] for a row and a column on the same side (|tr - tc| <= b)
  static __device__ __forceinline__ float2 same_side(const Sm3<B>& sm, int side, int tr, int tc, int kind, int s,
                                                     int n) {
    if (kind == 0) return make_float2(0.f, 0.f);
    if (kind == 2) return (tr == tc) ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f);
    const int jcol = row_of(side, tc, s);
    if (jcol < 0 || jcol >= n) return make_float2(0.f, 0.f);
    const int d = side ? (tc - tr) : (tr - tc);  // column index - row index
    return *reinterpret_cast<const float2*>(&sm.u.ring[side][tr & (C::RB - 1)][B + d]);
  }
  // A[(sr, tr)][(sc, tc)] for any pair (used for the initial window, where the
  // middle rows of the two sides are within the band of each other)
  static __device__ __forceinline__ float2 any_entry(const Sm3<B>& sm, int sr, int tr, int sc, int tc, int kind,
                                                     int s, int n) {
    if (kind == 0) return make_float2(0.f, 0.f);
    const int i = row_of(sr, tr, s), jcol = row_of(sc, tc, s);
    if (kind == 2) return (i == jcol) ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f);
    if (jcol < 0 || jcol >= n) return make_float2(0.f, 0.f);
    const int d = jcol - i;
    if (d < -B || d > B) return make_float2(0.f, 0.f);
    return *reinterpret_cast<const float2*>(&sm.u.ring[sr][tr & (C::RB - 1)][B + d]);
  }
  static __device__ __forceinline__ float2 rhs_of(const Sm3<B>& sm, int side, int t, int kind) {
    if (kind != 1) return make_float2(0.f, 0.f);
    return *reinterpret_cast<const float2*>(&sm.rrhs[side][t & (C::RB - 1)]);
  }

  // ---------------------------------------------------------------- phase 1
  static __device__ void factor(Sm3<B>& sm, const Paqif3Args& a, int dsys, int ssys, int u, int& flag) {
    const int s = a.s, n = a.n;
    float4* stk = a.stack + (size_t)ssys * s * C::SL;
    float4* fst = a.fstore ? a.fstore + (size_t)ssys * s * C::FL : nullptr;
    // prologue: chunks 0..3 issued, 0 and 1 converted; afterwards chunks
    // [0, conv) are double-float and chunks up to conv+1 are issued
    chunk<false>(sm, a, dsys, 0, u);
    cpa_commit();
    chunk<false>(sm, a, dsys, 1, u);
    cpa_commit();
    chunk<false>(sm, a, dsys, 2, u);
    cpa_commit();
    chunk<false>(sm, a, dsys, 3, u);
    cpa_commit();
    cpa_wait<2>();
    chunk<true>(sm, a, dsys, 0, u);
    chunk<true>(sm, a, dsys, 1, u);
    __syncwarp();
    int conv = 2;
    // initial window: stream indices [0, b] on both sides, slot = side*W + t
    for (int e = u; e < C::NS * C::NC; e += C::LS) {
      const int r = e / C::NC, c = e % C::NC;
      const int sr = r / C::W, tr = r % C::W;
      const int kind = row_kind(sm, sr, tr, s, n);
      sm.S[r][c] = (c == C::NS) ? rhs_of(sm, sr, tr, kind) : any_entry(sm, sr, tr, c / C::W, c % C::W, kind, s, n);
      if (c == 0) sm.kind[r] = kind;
    }
    __syncwarp();

    // static update coordinates of this lane
    int upd_r[C::RU], upd_c[C::RU];
#pragma unroll
    for (int m = 0; m < C::RU; ++m) {
      const int e = u + m * C::LS;
      upd_r[m] = e / C::NOC;
      upd_c[m] = e % C::NOC;
    }
    int base = 1;  // (k + 1) mod W
    for (int k = 0; k < s; ++k) {
      const int pslot = base == 0 ? C::W - 1 : base - 1;  // k mod W
      const int sp = pslot, sq = C::W + pslot;
      // slot of outer index o (o < b: left row/column, b <= o < 2b: right, o = 2b: rhs column)
      auto oslot = [&](int o) {
        return o < B ? wrap(base + o) : (o < C::NO ? C::W + wrap(base + o - B) : C::NS);
      };
      const df pa = f2df(sm.S[sp][sp]), pb = f2df(sm.S[sp][sq]);
      const df pc = f2df(sm.S[sq][sp]), pd = f2df(sm.S[sq][sq]);
      df det = A::det2(pa, pd, pb, pc);
      const float scale = fabsf(pa.hi * pd.hi) + fabsf(pb.hi * pc.hi);
      if (!(fabsf(det.hi) > 1e-13f * scale) || !(scale > 0.f)) {
        if (flag == 0) flag = EHL_INFO_SINGULAR;
        if (!(fabsf(det.hi) > 0.f)) det = make_df(1e-30f, 0.f);
      }
      const df inv = A::rcp(det);
      if (fst && u == 0) {  // Pi^-1 = inv [[d, -b], [-c, a]]
        const df i00 = A::mul(pd, inv), i01 = df_neg(A::mul(pb, inv));
        const df i10 = df_neg(A::mul(pc, inv)), i11 = A::mul(pa, inv);
        fst[(size_t)k * C::FL + C::NO] = make_float4(i00.hi, i00.lo, i01.hi, i01.lo);
        fst[(size_t)k * C::FL + C::NO + 1] = make_float4(i10.hi, i10.lo, i11.hi, i11.lo);
      }
      // tasks t < 2b: multipliers of outer row t, [w_ip, w_iq] = [l_ip, l_iq] Pi^-1;
      //       t >= 2b: folded outer column o = t - 2b, Pi^-1 [z_p,o; z_q,o].
      // All loads first, then the arithmetic, then the stores (no shared-memory
      // store sits between the loads, so the rounds overlap).
      df tx1[C::R1], tx2[C::R1];
#pragma unroll
      for (int m = 0; m < C::R1; ++m) {
        const int t = min(u + m * C::LS, C::NT1 - 1);
        const bool rowtask = t < C::NO;
        const int so = oslot(rowtask ? t : t - C::NO);
        tx1[m] = f2df(rowtask ? sm.S[so][sp] : sm.S[sp][so]);
        tx2[m] = f2df(rowtask ? sm.S[so][sq] : sm.S[sq][so]);
      }
      df tr1[C::R1], tr2[C::R1];
#pragma unroll
      for (int m = 0; m < C::R1; ++m) {
        const bool rowtask = (u + m * C::LS) < C::NO;
        // row:    w_p = inv (x1 d - x2 c),  w_q = inv (x2 a - x1 b)
        // column: m_p = inv (x1 d - x2 b),  m_q = inv (x2 a - x1 c)
        tr1[m] = A::mul(A::det2(tx1[m], pd, tx2[m], rowtask ? pc : pb), inv);
        tr2[m] = A::mul(A::det2(tx2[m], pa, tx1[m], rowtask ? pb : pc), inv);
      }
#pragma unroll
      for (int m = 0; m < C::R1; ++m) {
        const int t = u + m * C::LS;
        if (t < C::NO) {
          sm.w[t][0] = df2f(tr1[m]);
          sm.w[t][1] = df2f(tr2[m]);
          if (fst) fst[(size_t)k * C::FL + t] = make_float4(tr1[m].hi, tr1[m].lo, tr2[m].hi, tr2[m].lo);
        } else if (t < C::NT1) {
          stk[(size_t)k * C::SL + (t - C::NO)] = make_float4(tr1[m].hi, tr1[m].lo, tr2[m].hi, tr2[m].lo);
        }
      }
      __syncwarp();
      // rank-2 update of the outer block (rhs column included): L <- L - w_p z_p - w_q z_q
      {
        float2 uS[C::RU], uW0[C::RU], uW1[C::RU], uZp[C::RU], uZq[C::RU];
        int uslot[C::RU];
#pragma unroll
        for (int m = 0; m < C::RU; ++m) {
          const int ro = min(upd_r[m], C::NO - 1);
          const int r = oslot(ro), c = oslot(upd_c[m]);
          uslot[m] = r * C::NC + c;
          uS[m] = sm.S[r][c];
          uW0[m] = sm.w[ro][0];
          uW1[m] = sm.w[ro][1];
          uZp[m] = sm.S[sp][c];
          uZq[m] = sm.S[sq][c];
        }
        float2 uN[C::RU];
#pragma unroll
        for (int m = 0; m < C::RU; ++m)
          uN[m] = df2f(A::sub_two_prods(f2df(uS[m]), f2df(uW0[m]), f2df(uZp[m]), f2df(uW1[m]), f2df(uZq[m])));
#pragma unroll
        for (int m = 0; m < C::RU; ++m)
          if (upd_r[m] < C::NO) (&sm.S[0][0])[uslot[m]] = uN[m];
      }
      // rows entering at the end of this level have stream index tn on both sides
      const int tn = k + B + 1;
      if ((tn >> 3) >= conv) {
        // issue chunk conv+2 into the slots of chunk conv-2 (rows t < 8 conv - 8 <= tn - b,
        // no longer referenced); then at most the two newest groups are pending
        chunk<false>(sm, a, dsys, conv + 2, u);
        cpa_commit();
        cpa_wait<2>();
        chunk<true>(sm, a, dsys, conv, u);
        ++conv;
      }
      __syncwarp();
      // the two incoming rows and columns go into the pivot slots; in the new
      // window slot q of a side holds stream index k + 1 + ((q - base) mod W).
      // An incoming row/column is at least 2k + b + 3 > b away from every index
      // of the other side, so its cross-side entries are zero.
      // Closed forms: in the new window slot q of a side holds stream index
      // t_q = k + 1 + wq with wq = (q - base) mod W, so tn - t_q = b - wq.  The
      // incoming row's entry in column q is band[row][2b - wq] on the left and
      // band[row][wq] on the right; a window row r's entry in the incoming
      // column is band[r][wq_r] on the left and band[r][2b - wq_r] on the right.
      const int kind_l = row_kind(sm, 0, tn, s, n), kind_r = row_kind(sm, 1, tn, s, n);
      const bool gval_l = kind_l != 0, gval_r = (s + tn) < n;  // incoming column index inside [0, n)
      {
        float2 nv[C::RN];
        int nslot[C::RN];
#pragma unroll
        for (int m = 0; m < C::RN; ++m) {
          const int e = min(u + m * C::LS, C::NNEW - 1);
          const int side = e / (C::NC + C::NS);
          const int rem = e % (C::NC + C::NS);
          const int sn = side ? sq : sp;
          float2 v = make_float2(0.f, 0.f);
          if (rem < C::NC) {  // entry (incoming row, column rem)
            const int kind_n = side ? kind_r : kind_l;
            nslot[m] = sn * C::NC + rem;
            if (rem == C::NS) {
              if (kind_n == 1) v = *reinterpret_cast<const float2*>(&sm.rrhs[side][tn & (C::RB - 1)]);
            } else if (rem / C::W == side) {
              const int wq = wrap((rem % C::W) - base + C::W);
              if (kind_n == 1)
                v = *reinterpret_cast<const float2*>(&sm.u.ring[side][tn & (C::RB - 1)][side ? wq : 2 * B - wq]);
              else if (kind_n == 2 && rem == sn)
                v = make_float2(1.f, 0.f);
            }
          } else {  // entry (window row r, incoming column); the diagonal belongs to the row part
            const int r = rem - C::NC;
            nslot[m] = (r == sn) ? -1 : r * C::NC + sn;
            if (r / C::W == side && r != sn && (side ? gval_r : gval_l) && sm.kind[r] == 1) {
              const int wq = wrap((r % C::W) - base + C::W);
              const int tr = k + 1 + wq;
              v = *reinterpret_cast<const float2*>(&sm.u.ring[side][tr & (C::RB - 1)][side ? 2 * B - wq : wq]);
            }
          }
          nv[m] = v;
        }
        __syncwarp();  // every lane has read sm.kind before the pivot slots change kind
#pragma unroll
        for (int m = 0; m < C::RN; ++m)
          if (u + m * C::LS < C::NNEW && nslot[m] >= 0) (&sm.S[0][0])[nslot[m]] = nv[m];
        if (u == 0) {
          sm.kind[sp] = kind_l;
          sm.kind[sq] = kind_r;
        }
      }
      __syncwarp();
      base = wrap(base + 1);
    }
    cpa_wait<0>();
    __threadfence_block();
    __syncwarp();
  }


  // ---------------------------------------------------------------- solve only
  // W0 Y = F for a new right-hand side with the multipliers of a stored
  // factorization: middle-out, y_p,q are read off the pivot slots, the outer
  // rows take F_o -= w_o,p y_p + w_o,q y_q, and Pi^-1 (y_p, y_q) replaces the
  // folded rhs column of the stack level for the Z0 sweep.
  static __device__ void w_sweep(Sm3<B>& sm, const Paqif3Args& a, int dsys, int ssys, int u) {
    const int s = a.s, n = a.n;
    float4* stk = a.stack + (size_t)ssys * s * C::SL;
    const float4* fst = a.fstore + (size_t)ssys * s * C::FL;
    const double* rsys = a.rhs + (size_t)dsys * n;
    // rhs and flags by chunk of 8 stream indices per side, staged in rrhs/ract;
    // factor-store levels staged in the (unused) band ring as float4 [RB][FL]
    float4 (*fring)[C::FL] = sm.u.fr;
    auto issue = [&](int c) {
      const int t0 = c * C::CH;
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        int r_lo = side ? s + t0 : s - 1 - (t0 + C::CH - 1);
        int r_hi = side ? s + t0 + C::CH - 1 : s - 1 - t0;
        r_lo = max(r_lo, 0);
        r_hi = min(r_hi, n - 1);
        for (int r = r_lo + u; r <= r_hi; r += C::LS)
          cpa8(&sm.rrhs[side][(side ? r - s : s - 1 - r) & (C::RB - 1)], rsys + r);
      }
      const int k0 = t0, k1 = min(t0 + C::CH, s);
      for (int e = u; e < (k1 - k0) * C::FL; e += C::LS) {
        const int lvl = k0 + e / C::FL, off = e % C::FL;
        if (lvl < s) cpa16cg(&fring[lvl & (C::RB - 1)][off], fst + (size_t)lvl * C::FL + off);
      }
    };
    auto convert = [&](int c) {
      const int t0 = c * C::CH;
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        int r_lo = side ? s + t0 : s - 1 - (t0 + C::CH - 1);
        int r_hi = side ? s + t0 + C::CH - 1 : s - 1 - t0;
        r_lo = max(r_lo, 0);
        r_hi = min(r_hi, n - 1);
        for (int r = r_lo + u; r <= r_hi; r += C::LS) {
          const int t = (side ? r - s : s - 1 - r) & (C::RB - 1);
          double* dst = &sm.rrhs[side][t];
          const df v = A::from_double(*dst);
          *reinterpret_cast<float2*>(dst) = make_float2(v.hi, v.lo);
          sm.ract[side][t] = a.act ? __ldcg(a.act + (size_t)dsys * n + r) : 0;
        }
      }
    };
    // chunk c = rhs of stream indices [8c, 8c+8) and factor-store levels [8c, 8c+8).
    // Level k reads levels of chunk k/8 and rhs up to stream k + b + 1 <= k + 9,
    // so at k = 8c chunks c..c+2 must be complete and chunk c-1 is free.
    issue(0);
    cpa_commit();
    issue(1);
    cpa_commit();
    issue(2);
    cpa_commit();
    issue(3);
    cpa_commit();
    cpa_wait<1>();
    convert(0);
    convert(1);
    convert(2);
    __syncwarp();
    float2* F = &sm.S[0][C::NS];  // reuse the window's rhs column, stride NC
    for (int e = u; e < C::NS; e += C::LS) {
      const int side = e / C::W, t = e % C::W;
      F[e * C::NC] = rhs_of(sm, side, t, row_kind(sm, side, t, s, n));
    }
    __syncwarp();
    int base = 1;
    for (int k = 0; k < s; ++k) {
      const int pslot = base == 0 ? C::W - 1 : base - 1;
      const int sp = pslot, sq = C::W + pslot;
      const int tn = k + B + 1;
      if ((k & 7) == 0 && k > 0) {
        // issue chunk c+3 into the slots of chunk c-1, then all but the newest
        // group are complete: chunk c+2 can be converted
        issue((k >> 3) + 3);
        cpa_commit();
        cpa_wait<1>();
        convert((k >> 3) + 2);
        __syncwarp();
      }
      const df yp = f2df(F[sp * C::NC]), yq = f2df(F[sq * C::NC]);
      const float4* lv = fring[k & (C::RB - 1)];
      if (u < C::NO) {
        const int so = u < B ? wrap(base + u) : C::W + wrap(base + u - B);
        const float4 wv = lv[u];
        F[so * C::NC] = df2f(A::sub_two_prods(f2df(F[so * C::NC]), make_df(wv.x, wv.y), yp, make_df(wv.z, wv.w), yq));
      } else if (u == C::NO) {
        const float4 r0 = lv[C::NO], r1 = lv[C::NO + 1];
        const df cp = A::sub_two_prods(df_zero(), df_neg(make_df(r0.x, r0.y)), yp, df_neg(make_df(r0.z, r0.w)), yq);
        const df cq = A::sub_two_prods(df_zero(), df_neg(make_df(r1.x, r1.y)), yp, df_neg(make_df(r1.z, r1.w)), yq);
        stk[(size_t)k * C::SL + C::NO] = make_float4(cp.hi, cp.lo, cq.hi, cq.lo);
      }
      __syncwarp();
      if (u < 2) F[(u ? sq : sp) * C::NC] = rhs_of(sm, u, tn, row_kind(sm, u, tn, s, n));
      __syncwarp();
      base = wrap(base + 1);
    }
    cpa_wait<0>();
    __threadfence_block();
    __syncwarp();
  }

  // ---------------------------------------------------------------- phase 2
  // Z0 U = Y for k = s-1 .. 0: x_p,q = Pi^-1 y - sum_o (Pi^-1 z_o) x_o.  The
  // sum is accumulated ahead: when a level solves its pair, each of the b
  // levels below adds that pair's terms to its accumulators.
  static __device__ void z_solve(Sm3<B>& sm, const Paqif3Args& a, int dsys, int ssys, bool real, int u,
                                 int& flag) {
    const int s = a.s, n = a.n;
    const float4* stk = a.stack + (size_t)ssys * s * C::SL;
    double* xs = a.x + (size_t)dsys * n;
    for (int e = u; e < 2 * C::W; e += C::LS) sm.acc[e >> 1][e & 1] = make_float2(0.f, 0.f);
    auto issue = [&](int c) {  // levels with v = s-1-k in [8c, 8c+8)
      const int v0 = c * C::CH, v1 = min(v0 + C::CH, s);
      if (v0 >= v1) return;
      const int k_lo = s - v1;
      const int nvec = (v1 - v0) * C::SL;
      const float4* src = stk + (size_t)k_lo * C::SL;
      for (int e = u; e < nvec; e += C::LS) {
        const int lvl = k_lo + e / C::SL, off = e % C::SL;
        cpa16cg(&sm.u.stk[(s - 1 - lvl) & (C::RB - 1)][off], src + e);
      }
    };
    issue(0);
    cpa_commit();
    issue(1);
    cpa_commit();
    issue(2);
    cpa_commit();
    cpa_wait<1>();  // chunks 0 and 1: the accumulations look up to b levels ahead
    __syncwarp();
    int issued = 3;
    df pend_x = df_zero();
    int pend_row = -1;
    auto store_x = [&](df xv, int row) {
      double d = A::to_double(xv);
      if (!isfinite(d) && flag == 0) flag = EHL_INFO_NONFINITE;
      if (a.mode == 1) d = d > 0.0 ? d : 0.0;
      if (real && row < n) xs[row] = d;
    };
    for (int k = s - 1; k >= 0; --k) {
      const int v = s - 1 - k;
      if ((v & 7) == 0 && v > 0) {
        // at v = 8c: chunk c+2 replaces chunk c-2, then chunks <= c+1 are complete
        issue(issued);
        cpa_commit();
        ++issued;
        cpa_wait<1>();
        __syncwarp();
      }
      const int km = k % C::W;
      if (u < 2) {
        const float4 cv = sm.u.stk[v & (C::RB - 1)][C::NO];  // folded rhs column: Pi^-1 y
        const df c = u ? make_df(cv.z, cv.w) : make_df(cv.x, cv.y);
        const df xv = A::sub(c, f2df(sm.acc[km][u]));
        sm.xpq[u] = df2f(xv);
        sm.acc[km][u] = make_float2(0.f, 0.f);
        // the float64 conversion and store of the previous level run here, off
        // the path that the next level waits on
        if (pend_row >= 0) store_x(pend_x, pend_row);
        pend_x = xv;
        pend_row = (u ? s + k : s - 1 - k);
      }
      __syncwarp();
      // push (x_p, x_q) of level k into the accumulators of levels k-1 .. k-b
      if (u < 2 * B) {
        const int dl = 1 + (u >> 1), side = u & 1;
        const int kn = k - dl;
        if (kn >= 0) {
          const float4* lv = sm.u.stk[(s - 1 - kn) & (C::RB - 1)];
          const float4 ml = lv[dl - 1], mr = lv[B + dl - 1];  // columns of x_p and x_q at level kn
          const df m1 = side ? make_df(ml.z, ml.w) : make_df(ml.x, ml.y);
          const df m2 = side ? make_df(mr.z, mr.w) : make_df(mr.x, mr.y);
          const int slot = kn % C::W;
          const df acc = f2df(sm.acc[slot][side]);
          sm.acc[slot][side] =
              df2f(A::sub_two_prods(acc, df_neg(m1), f2df(sm.xpq[0]), df_neg(m2), f2df(sm.xpq[1])));
        }
      }
      __syncwarp();
    }
    if (u < 2 && pend_row >= 0) store_x(pend_x, pend_row);
    cpa_wait<0>();
    __threadfence_block();
    __syncwarp();
  }

  static __device__ bool active_set_update(const Paqif3Args& a, int dsys, bool real, int u) {
    const int n = a.n;
    const double* bsys = a.band + (size_t)dsys * n * C::BW;
    const double* xs = a.x + (size_t)dsys * n;
    int* as = a.act + (size_t)dsys * n;
    int changed = 0;
    if (real) {
      for (int i = u; i < n; i += C::LS) {
        df w = df_neg(A::from_double(a.rhs[(size_t)dsys * n + i]));
#pragma unroll
        for (int q = 0; q < C::BW; ++q) {
          const int c = i - B + q;
          if (c >= 0 && c < n)
            w = A::fma(A::from_double(__ldg(bsys + (size_t)i * C::BW + q)), A::from_double(__ldcg(xs + c)), w);
        }
        const int old = __ldcg(as + i);
        const double xi = __ldcg(xs + i);
        const int nw = old ? (w.hi > 0.f ? 1 : 0) : (xi < 0.0 ? 1 : 0);
        if (nw != old) {
          changed = 1;
          __stcg(as + i, nw);
        }
      }
    }
#pragma unroll
    for (int off = C::LS / 2; off > 0; off >>= 1) changed |= __shfl_xor_sync(0xffffffffu, changed, off, C::LS);
    __threadfence_block();
    __syncwarp();
    return changed != 0;
  }
};

// Groups past n_sys replay a real system's loads with their own stack slot and
// no other global stores, so every warp barrier and shuffle sees a full warp.
// Mode 2 runs active-set steps until no group of the warp changes its set (a
// converged group re-solves with the same set, reproducing the same x).
template <int B, bool F32>
__global__ void __launch_bounds__(32 * C3<B>::WARPS, 4) paqif3_kernel(Paqif3Args a) {
  using C = C3<B>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / C::LS, u = lane % C::LS;
  Sm3<B>& sm = reinterpret_cast<Sm3<B>*>(smem_raw)[warp * C::G + grp];
  const int ssys = (blockIdx.x * C::WARPS + warp) * C::G + grp;
  const bool real = ssys < a.n_sys;
  const int dsys = real ? ssys : a.n_sys - 1;
  if (__all_sync(0xffffffffu, !real)) return;
  int flag = 0, solves = 0;
  bool more = real;
  const int max_solves = (a.mode == 2) ? kPaqifMaxActiveSetSteps : 1;
  for (int it = 0; it < max_solves; ++it) {
    P3<B, F32>::factor(sm, a, dsys, ssys, u, flag);
    P3<B, F32>::z_solve(sm, a, dsys, ssys, real, u, flag);
    if (more) ++solves;
    if (a.mode != 2) break;
    if (!P3<B, F32>::active_set_update(a, dsys, real, u)) more = false;
    if (!__any_sync(0xffffffffu, more)) break;
  }
  // the first nonzero flag among the group's lanes
  int f = flag;
#pragma unroll
  for (int off = C::LS / 2; off > 0; off >>= 1) {
    const int o = __shfl_xor_sync(0xffffffffu, f, off, C::LS);
    if (f == 0) f = o;
  }
  if (a.mode == 2 && more && f == 0) f = EHL_INFO_NOCONV;
  if (real && u == 0) {
    if (a.iters) a.iters[dsys] = solves;
    if (a.info) a.info[dsys] = f;
  }
}

// Solve only, with the factorization stored by a factor launch (same systems,
// same band): the W0 sweep for the new rhs, then the Z0 sweep.
template <int B, bool F32>
__global__ void __launch_bounds__(32 * C3<B>::WARPS, 4) paqif3_solve_kernel(Paqif3Args a) {
  using C = C3<B>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / C::LS, u = lane % C::LS;
  Sm3<B>& sm = reinterpret_cast<Sm3<B>*>(smem_raw)[warp * C::G + grp];
  const int ssys = (blockIdx.x * C::WARPS + warp) * C::G + grp;
  const bool real = ssys < a.n_sys;
  const int dsys = real ? ssys : a.n_sys - 1;
  if (__all_sync(0xffffffffu, !real)) return;
  int flag = 0;
  P3<B, F32>::w_sweep(sm, a, dsys, ssys, u);
  P3<B, F32>::z_solve(sm, a, dsys, ssys, real, u, flag);
  int f = flag;
#pragma unroll
  for (int off = C::LS / 2; off > 0; off >>= 1) {
    const int o = __shfl_xor_sync(0xffffffffu, f, off, C::LS);
    if (f == 0) f = o;
  }
  if (real && u == 0 && a.info && f != 0) a.info[dsys] = f;
}

template <int B>
static size_t p3_smem() {
  return sizeof(Sm3<B>) * (size_t)(C3<B>::WARPS * C3<B>::G);
}
template <int B>
static int p3_per_cta() {
  return C3<B>::WARPS * C3<B>::G;
}

size_t paqif_stack_bytes(int n_sys, int n, int beta) {
  const int s = (n + 1) / 2;
  int per = 0;
  switch (beta) {
    case 1: per = p3_per_cta<1>(); break;
    case 2: per = p3_per_cta<2>(); break;
    case 3: per = p3_per_cta<3>(); break;
    case 4: per = p3_per_cta<4>(); break;
    case 5: per = p3_per_cta<5>(); break;
    case 6: per = p3_per_cta<6>(); break;
    case 7: per = p3_per_cta<7>(); break;
    case 8: per = p3_per_cta<8>(); break;
    default: return 0;
  }
  const size_t padded = (size_t)((n_sys + per - 1) / per) * per;
  return padded * (size_t)s * (size_t)(2 * beta + 1) * sizeof(float4);
}

template <int B>
static int p3_fl() {
  return C3<B>::FL;
}

size_t paqif_factor_store_bytes(int n_sys, int n, int beta) {
  const int s = (n + 1) / 2;
  int per = 0, fl = 0;
  switch (beta) {
#define EHL_CASE(BB)          \
  case BB:                    \
    per = p3_per_cta<BB>();   \
    fl = p3_fl<BB>();         \
    break;
    EHL_CASE(1) EHL_CASE(2) EHL_CASE(3) EHL_CASE(4) EHL_CASE(5) EHL_CASE(6) EHL_CASE(7) EHL_CASE(8)
#undef EHL_CASE
    default:
      return 0;
  }
  const size_t padded = (size_t)((n_sys + per - 1) / per) * per;
  return padded * (size_t)s * (size_t)fl * sizeof(float4);
}

// the dynamic shared-memory size of both kernels, set once per device
template <int B>
static cudaError_t p3_attrs() {
  static std::atomic<unsigned long long> set{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (set.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  const int smem = (int)p3_smem<B>();
  e = cudaFuncSetAttribute(paqif3_kernel<B, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(paqif3_solve_kernel<B, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(paqif3_kernel<B, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(paqif3_solve_kernel<B, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess && bit) set.fetch_or(bit, std::memory_order_release);
  return e;
}

cudaError_t paqif_prepare(int beta) {
  switch (beta) {
    case 1: return p3_attrs<1>();
    case 2: return p3_attrs<2>();
    case 3: return p3_attrs<3>();
    case 4: return p3_attrs<4>();
    case 5: return p3_attrs<5>();
    case 6: return p3_attrs<6>();
    case 7: return p3_attrs<7>();
    case 8: return p3_attrs<8>();
    default: return cudaErrorInvalidValue;
  }
}

template <int B>
static cudaError_t launch3(const PaqifLaunch& L, cudaStream_t st, void* fstore, bool solve_only) {
  Paqif3Args a;
  a.n_sys = L.n_sys;
  a.n = L.n;
  a.s = (L.n + 1) / 2;
  a.mode = L.mode;
  a.band = L.band;
  a.rhs = L.rhs;
  a.act = L.act;
  a.stack = reinterpret_cast<float4*>(L.stack);
  a.fstore = reinterpret_cast<float4*>(fstore);
  a.x = L.x;
  a.iters = L.iters;
  a.info = L.info;
  const size_t smem = p3_smem<B>();
  const int per = p3_per_cta<B>();
  const int grid = (L.n_sys + per - 1) / per;
  cudaError_t e = p3_attrs<B>();
  if (e != cudaSuccess) return e;
  const bool f32 = L.f32 && L.mode != 2;
  if (solve_only) {
    if (f32)
      paqif3_solve_kernel<B, true><<<grid, 32 * C3<B>::WARPS, smem, st>>>(a);
    else
      paqif3_solve_kernel<B, false><<<grid, 32 * C3<B>::WARPS, smem, st>>>(a);
    note_launch();
  } else {
    if (f32)
      paqif3_kernel<B, true><<<grid, 32 * C3<B>::WARPS, smem, st>>>(a);
    else
      paqif3_kernel<B, false><<<grid, 32 * C3<B>::WARPS, smem, st>>>(a);
    note_launch();
  }
  return cudaGetLastError();
}

// int8 mask -> int32 flags in the workspace (mode 2 rewrites them in place).
__global__ void expand_active3_kernel(const uint8_t* __restrict__ in, int* __restrict__ out, size_t total) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < total; i += stride) out[i] = in ? (in[i] ? 1 : 0) : 0;
}

cudaError_t launch_expand_active(const uint8_t* in, int* out, size_t total, cudaStream_t st) {
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  expand_active3_kernel<<<blocks, 256, 0, st>>>(in, out, total);
  note_launch();
  return cudaGetLastError();
}

static cudaError_t dispatch3(const PaqifLaunch& L, cudaStream_t st, void* fstore, bool solve_only) {
  switch (L.beta) {
    case 1: return launch3<1>(L, st, fstore, solve_only);
    case 2: return launch3<2>(L, st, fstore, solve_only);
    case 3: return launch3<3>(L, st, fstore, solve_only);
    case 4: return launch3<4>(L, st, fstore, solve_only);
    case 5: return launch3<5>(L, st, fstore, solve_only);
    case 6: return launch3<6>(L, st, fstore, solve_only);
    case 7: return launch3<7>(L, st, fstore, solve_only);
    case 8: return launch3<8>(L, st, fstore, solve_only);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_paqif(const PaqifLaunch& L, cudaStream_t st) { return dispatch3(L, st, nullptr, false); }

cudaError_t launch_paqif_factor(const PaqifLaunch& L, void* fstore, cudaStream_t st) {
  if (L.mode == 2 || !fstore) return cudaErrorInvalidValue;
  return dispatch3(L, st, fstore, false);
}

cudaError_t launch_paqif_resolve(const PaqifLaunch& L, void* fstore, cudaStream_t st) {
  if (L.mode == 2 || !fstore) return cudaErrorInvalidValue;
  return dispatch3(L, st, fstore, true);
}

}  // namespace ehl
