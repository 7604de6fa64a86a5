// paqif4.cu -- batched PAQIF (projected alternate quadrant interlocking factorization),
// one lane per row of the elimination window.
//
// Method (Sec. 2.2.1-2.2.3; projection of Sec. 2.2.2 / Sec. 2.2.4 Steps 5
// and 7 after the solve, one partition per system): for n = 2s, level
// k = 0..s-1 pivots on the rows/columns at stream index k of the two sides
// (rows s-1-k and s+k) of the Schur complement L0^(k); the Z0 rows are the
// pivot rows, the W0 columns solve
//   z_pp w_ip + z_qp w_iq = l_ip,   z_pq w_ip + z_qq w_iq = l_iq,
// and L0^(k+1) = L0^(k) - w_p z_p^T - w_q z_q^T.  W0 Y = F runs in the same
// middle-out sweep; Z0 U = Y runs from both ends towards the middle with one
// 2x2 solve per level.
//
// GB300 mapping:
//  * for half-band b only the window of the Schur complement on the stream
//    indices k..k+b of both sides is non-trivial: 2(b+1) rows and columns plus
//    the right-hand side as one more column.  Lane (side, j) of a group of
//    2(b+1) lanes owns the window row of stream index t = j (mod b+1) on its
//    side and keeps it in registers, its columns ordered by distance from the
//    pivot (a register shift per level), so the rank-2 update needs no shared
//    memory but the two pivot rows, broadcast once per level.
//  * every lane runs the same instruction stream: an outer row computes its
//    multipliers w = [l_p, l_q] Pi^-1 and updates its entries, a pivot row
//    forms its side of the folded outer columns Pi^-1 [z_p; z_q] for the stack,
//    both as  out = base - (alpha z_p + beta z_q).
//  * band rows stream from HBM with cp.async into a 32-row ring per side,
//    16 levels ahead, converted float64 -> double-float once, in place, by
//    the lane that copied them.
//  * the Z0 and W0 sweeps rotate roles instead of data: the lane that owns a
//    row slot accumulates the terms of the level that slot holds next, and the
//    solved pair of each level is broadcast with warp shuffles.
//  * arithmetic is double-float (df64.cuh); float64 only at the interface.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "df64.cuh"
#include "ehl_internal.h"

namespace ehl {

template <int B>
struct C4 {
  static constexpr int W = B + 1;       // row slots per side (stream indices k..k+b)
  static constexpr int GS = 2 * W;      // lanes per system, one per window row
  static constexpr int G = 32 / GS;     // systems per warp
  static constexpr int NC = GS + 1;     // window columns: (side, distance) then the rhs
  static constexpr int RHS = GS;        // column index of the rhs
  static constexpr int BW = 2 * B + 1;  // band row width
  static constexpr int SL = 2 * B + 1;  // stack float4 per level: (M_p, M_q) per outer column, rhs last
  static constexpr int FL = GS;         // factor-store float4 per level: one per row slot
  static constexpr int RB = 32;         // ring rows per side
  static constexpr int CH = 8;          // rows per chunk
  static constexpr int WARPS = kPaqifWarpsPerCta;
};

template <int B>
struct __align__(16) Sm4 {
  using C = C4<B>;
  float4 zb[2][C::NC];  // the two pivot rows of a level (z_p, z_q) per column, double-buffered
  union {
    double ring[2][C::RB][C::BW];  // band rows: float64 as copied, double-float after conversion
    float4 stk[C::RB][C::SL];      // Z0 sweep: stack levels
    float4 fr[C::RB][C::FL];       // W0 sweep of a resolve: factor-store levels
  } u;
  double rrhs[2][C::RB];
  int ract[2][C::RB];
};

struct Paqif4Args {
  int n_sys, n, s, mode;
  const double* band;
  const double* rhs;
  int* act;
  float4* stack;   // [pad_sys][s][SL]
  float4* fstore;  // [pad_sys][s][FL]: multipliers and Pi^-1 rows (factor once, solve many), or null
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
__device__ __forceinline__ df shfl_df(df v, int src) {
  return make_df(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
}

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

// Lane roles.  Lanes past the last whole group ("phantoms") mirror a lane of
// the last group, so every warp barrier and shuffle sees the full warp; they
// write nothing to shared or global memory.
template <int B>
struct Lane4 {
  int u;      // rank in the group: side * W + j
  int side;   // 0: rows s-1-t (left), 1: rows s+t (right)
  int j;      // row slot: the window row of stream index t = j (mod W)
  int gbase;  // warp lane of rank 0 of the group
  int grp;    // group within the warp
  bool live;  // not a phantom
  __device__ __forceinline__ Lane4() {
    using C = C4<B>;
    const int lane = threadIdx.x & 31;
    const int g0 = lane / C::GS;
    live = g0 < C::G;
    grp = live ? g0 : C::G - 1;
    u = live ? lane - g0 * C::GS : (lane - C::G * C::GS) % C::GS;
    side = u / C::W;
    j = u - side * C::W;
    gbase = grp * C::GS;
  }
};

template <int B, bool F32>
struct P4 {
  using C = C4<B>;
  using A = Ar<F32>;
  using L = Lane4<B>;

  static __device__ __forceinline__ int row_of(int side, int t, int s) { return side ? s + t : s - 1 - t; }

  // Copy (CONVERT = false) or convert in place (CONVERT = true) chunk c of
  // both sides; the lane of rank u handles elements u, u + GS, ...
  template <bool CONVERT>
  static __device__ __forceinline__ void chunk(Sm4<B>& sm, const Paqif4Args& a, int dsys, int c, const L& ln) {
    if (!ln.live) return;
    const int s = a.s, n = a.n, u = ln.u;
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
      for (int e = u; e < nel; e += C::GS) {
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
      for (int r = r_lo + u; r <= r_hi; r += C::GS) {
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
  static __device__ __forceinline__ int row_kind(const Sm4<B>& sm, int side, int t, int s, int n) {
    const int i = row_of(side, t, s);
    if (i < 0 || i >= 2 * s) return 0;
    if (i >= n) return 2;
    return sm.ract[side][t & (C::RB - 1)] ? 2 : 1;
  }
  // column (side, stream t) inside [0, n)
  static __device__ __forceinline__ bool col_in(int side, int t, int s, int n) {
    return side ? (s + t < n) : (t <= s - 1);
  }
  static __device__ __forceinline__ df band_at(const Sm4<B>& sm, int side, int t, int q) {
    return f2df(*reinterpret_cast<const float2*>(&sm.u.ring[side][t & (C::RB - 1)][q]));
  }
  // A[(sr, tr)][(sc, tc)] for any pair (the initial window, where the middle
  // rows of the two sides are within the band of each other)
  static __device__ __forceinline__ df any_entry(const Sm4<B>& sm, int sr, int tr, int sc, int tc, int kind, int s,
                                                 int n) {
    if (kind == 0) return df_zero();
    const int i = row_of(sr, tr, s), jcol = row_of(sc, tc, s);
    if (kind == 2) return (i == jcol) ? make_df(1.f, 0.f) : df_zero();
    if (jcol < 0 || jcol >= n) return df_zero();
    const int d = jcol - i;
    if (d < -B || d > B) return df_zero();
    return band_at(sm, sr, tr, B + d);
  }
  static __device__ __forceinline__ df rhs_of(const Sm4<B>& sm, int side, int t, int kind) {
    if (kind != 1) return df_zero();
    return f2df(*reinterpret_cast<const float2*>(&sm.rrhs[side][t & (C::RB - 1)]));
  }
  // stack index of window column c (c != pivot columns): outer column (side, distance d) or rhs
  static __device__ __forceinline__ constexpr int sidx(int c) {
    return c == C::RHS ? 2 * B : (c / C::W) * B + (c % C::W) - 1;
  }

  // ---------------------------------------------------------------- factor
  // Levels 0..s-1 of L0 = W0 Z0 with the rhs column (W0 Y = F) along; the
  // folded outer columns of every level go to the stack.
  static __device__ void factor(Sm4<B>& sm, const Paqif4Args& a, int dsys, int ssys, const L& ln, int& flag) {
    const int s = a.s, n = a.n;
    const int sg = ln.side, j = ln.j;
    float4* stk = a.stack + (size_t)ssys * s * C::SL;
    float4* fst = a.fstore ? a.fstore + (size_t)ssys * s * C::FL : nullptr;
    // prologue: chunks 0..3 issued, 0 and 1 converted; afterwards chunks
    // [0, conv) are double-float and chunks up to conv+1 are issued
    chunk<false>(sm, a, dsys, 0, ln);
    cpa_commit();
    chunk<false>(sm, a, dsys, 1, ln);
    cpa_commit();
    chunk<false>(sm, a, dsys, 2, ln);
    cpa_commit();
    chunk<false>(sm, a, dsys, 3, ln);
    cpa_commit();
    cpa_wait<2>();
    chunk<true>(sm, a, dsys, 0, ln);
    chunk<true>(sm, a, dsys, 1, ln);
    __syncwarp();
    int conv = 2;
    // the window of level 0: this lane's row is stream index j; column
    // (side c / W, distance c % W) is stream index c % W
    df R[C::NC];
    int kind = row_kind(sm, sg, j, s, n);
#pragma unroll
    for (int c = 0; c < C::NC; ++c)
      R[c] = (c == C::RHS) ? rhs_of(sm, sg, j, kind) : any_entry(sm, sg, j, c / C::W, c % C::W, kind, s, n);

    int pj = 0;  // k mod W: the row slot of the pivots
    for (int k = 0; k < s; ++k) {
      const bool piv = (j == pj);
      float4* zb = sm.zb[k & 1];
      // the two pivot rows to shared memory (double-buffered: one barrier a level)
      if (piv && ln.live) {
#pragma unroll
        for (int c = 0; c < C::NC; ++c) reinterpret_cast<float2*>(&zb[c])[sg] = df2f(R[c]);
      }
      __syncwarp();
      const float4 c0 = zb[0], c1 = zb[C::W];  // pivot columns: (z_p, z_q) at distance 0
      const df pa = make_df(c0.x, c0.y), pc = make_df(c0.z, c0.w);
      const df pb = make_df(c1.x, c1.y), pd = make_df(c1.z, c1.w);
      df det = A::det2(pa, pd, pb, pc);
      const float scale = fabsf(pa.hi * pd.hi) + fabsf(pb.hi * pc.hi);
      if (!(fabsf(det.hi) > 1e-13f * scale) || !(scale > 0.f)) {
        if (flag == 0) flag = EHL_INFO_SINGULAR;
        if (!(fabsf(det.hi) > 0.f)) det = make_df(1e-30f, 0.f);
      }
      const df inv = A::rcp(det);
      const df i00 = A::mul(pd, inv), i01 = df_neg(A::mul(pb, inv));
      const df i10 = df_neg(A::mul(pc, inv)), i11 = A::mul(pa, inv);
      // outer rows: w = [l_p, l_q] Pi^-1; pivot rows: minus their row of Pi^-1
      const df lp = R[0], lq = R[C::W];
      const df wp = A::sub_two_prods(df_zero(), df_neg(lp), i00, df_neg(lq), i10);
      const df wq = A::sub_two_prods(df_zero(), df_neg(lp), i01, df_neg(lq), i11);
      const df al = piv ? df_neg(sg ? i10 : i00) : wp;
      const df be = piv ? df_neg(sg ? i11 : i01) : wq;
      if (fst && ln.live) fst[(size_t)k * C::FL + ln.u] = make_float4(al.hi, al.lo, be.hi, be.lo);
      // rank-2 update of an outer row / folded outer columns of a pivot row
#pragma unroll
      for (int c = 0; c < C::NC; ++c) {
        if (c == 0 || c == C::W) continue;
        const float4 z = zb[c];
        const df o = A::sub_two_prods(piv ? df_zero() : R[c], al, make_df(z.x, z.y), be, make_df(z.z, z.w));
        if (piv) {
          if (ln.live) reinterpret_cast<float2*>(stk + (size_t)k * C::SL + sidx(c))[sg] = df2f(o);
        } else {
          R[c] = o;
        }
      }
      // the columns move one step towards the pivot
#pragma unroll
      for (int sd = 0; sd < 2; ++sd)
#pragma unroll
        for (int d = 1; d <= B; ++d) R[sd * C::W + d - 1] = R[sd * C::W + d];
      // rows entering at the end of this level have stream index tn on both sides
      const int tn = k + C::W;
      if ((tn >> 3) >= conv) {
        // issue chunk conv+2 into the slots of chunk conv-2 (stream indices
        // below 8 conv - 8 <= tn - b, no longer referenced); then at most the
        // two newest groups are pending
        chunk<false>(sm, a, dsys, conv + 2, ln);
        cpa_commit();
        cpa_wait<2>();
        chunk<true>(sm, a, dsys, conv, ln);
        ++conv;
        __syncwarp();
      }
      if (piv) {
        // the incoming row of this side (stream tn) takes the pivot slot.  In
        // the new window column (side, d) is stream k + 1 + d, at distance
        // b - d from the row: band[2b - d] on the left, band[d] on the
        // right; the other side's columns are more than b away.
        const int kn = row_kind(sm, sg, tn, s, n);
#pragma unroll
        for (int c = 0; c < C::NC; ++c) {
          df v = df_zero();
          if (c == C::RHS) {
            v = rhs_of(sm, sg, tn, kn);
          } else if (c / C::W == sg) {
            const int d = c % C::W;
            if (kn == 1) {
              if (col_in(sg, k + 1 + d, s, n)) v = band_at(sm, sg, tn, sg ? d : 2 * B - d);
            } else if (kn == 2 && d == B) {
              v = make_df(1.f, 0.f);
            }
          }
          R[c] = v;
        }
        kind = kn;
      } else {
        // the incoming column of this side (stream tn) at distance b: the
        // row (stream tr = tn - dd) meets it at band[b - dd] on the left,
        // band[b + dd] on the right
        const int dd = C::W - (j - pj + C::W) % C::W;
        df v = df_zero();
        if (kind == 1 && col_in(sg, tn, s, n)) v = band_at(sm, sg, tn - dd, sg ? B + dd : B - dd);
        R[B] = sg ? df_zero() : v;
        R[C::W + B] = sg ? v : df_zero();
      }
      pj = (pj == B) ? 0 : pj + 1;
    }
    cpa_wait<0>();
    __threadfence_block();
    __syncwarp();
  }

  // ---------------------------------------------------------------- solve only
  // W0 Y = F for a new right-hand side with the multipliers of a stored
  // factorization: the pivot pair (y_p, y_q) of a level is broadcast, the
  // outer rows take F_o -= w_o,p y_p + w_o,q y_q, and Pi^-1 (y_p, y_q)
  // replaces the folded rhs column of the stack level for the Z0 sweep.
  static __device__ void w_sweep(Sm4<B>& sm, const Paqif4Args& a, int dsys, int ssys, const L& ln) {
    const int s = a.s, n = a.n;
    const int sg = ln.side, j = ln.j, u = ln.u;
    float4* stk = a.stack + (size_t)ssys * s * C::SL;
    const float4* fst = a.fstore + (size_t)ssys * s * C::FL;
    const double* rsys = a.rhs + (size_t)dsys * n;
    // rhs and flags by chunk of 8 stream indices per side, staged in rrhs/ract;
    // factor-store levels staged in the (unused) band ring as float4 [RB][FL]
    float4 (*fring)[C::FL] = sm.u.fr;
    auto issue = [&](int c) {
      if (!ln.live) return;
      const int t0 = c * C::CH;
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        int r_lo = side ? s + t0 : s - 1 - (t0 + C::CH - 1);
        int r_hi = side ? s + t0 + C::CH - 1 : s - 1 - t0;
        r_lo = max(r_lo, 0);
        r_hi = min(r_hi, n - 1);
        for (int r = r_lo + u; r <= r_hi; r += C::GS)
          cpa8(&sm.rrhs[side][(side ? r - s : s - 1 - r) & (C::RB - 1)], rsys + r);
      }
      const int k0 = t0, k1 = min(t0 + C::CH, s);
      for (int e = u; e < (k1 - k0) * C::FL; e += C::GS) {
        const int lvl = k0 + e / C::FL, off = e % C::FL;
        cpa16cg(&fring[lvl & (C::RB - 1)][off], fst + (size_t)lvl * C::FL + off);
      }
    };
    auto convert = [&](int c) {
      if (!ln.live) return;
      const int t0 = c * C::CH;
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        int r_lo = side ? s + t0 : s - 1 - (t0 + C::CH - 1);
        int r_hi = side ? s + t0 + C::CH - 1 : s - 1 - t0;
        r_lo = max(r_lo, 0);
        r_hi = min(r_hi, n - 1);
        for (int r = r_lo + u; r <= r_hi; r += C::GS) {
          const int t = (side ? r - s : s - 1 - r) & (C::RB - 1);
          double* dst = &sm.rrhs[side][t];
          const df v = A::from_double(*dst);
          *reinterpret_cast<float2*>(dst) = make_float2(v.hi, v.lo);
          sm.ract[side][t] = a.act ? __ldcg(a.act + (size_t)dsys * n + r) : 0;
        }
      }
    };
    // chunk c = rhs of stream indices [8c, 8c+8) and factor-store levels [8c, 8c+8).
    // Level k reads level k and the rhs of stream k + b + 1 <= k + 9, so at
    // k = 8c chunks c..c+2 must be complete and chunk c-1 is free.
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
    df F = rhs_of(sm, sg, j, row_kind(sm, sg, j, s, n));
    int pj = 0;
    for (int k = 0; k < s; ++k) {
      if ((k & 7) == 0 && k > 0) {
        // issue chunk c+3 into the slots of chunk c-1, then all but the newest
        // group are complete: chunk c+2 can be converted
        issue((k >> 3) + 3);
        cpa_commit();
        cpa_wait<1>();
        convert((k >> 3) + 2);
        __syncwarp();
      }
      const df yp = shfl_df(F, ln.gbase + pj), yq = shfl_df(F, ln.gbase + C::W + pj);
      const float4 f = fring[k & (C::RB - 1)][u];
      const bool piv = (j == pj);
      const df o = A::sub_two_prods(piv ? df_zero() : F, make_df(f.x, f.y), yp, make_df(f.z, f.w), yq);
      if (piv) {
        if (ln.live) reinterpret_cast<float2*>(stk + (size_t)k * C::SL + 2 * B)[sg] = df2f(o);
        const int tn = k + C::W;
        F = rhs_of(sm, sg, tn, row_kind(sm, sg, tn, s, n));
      } else {
        F = o;
      }
      pj = (pj == B) ? 0 : pj + 1;
    }
    cpa_wait<0>();
    __threadfence_block();
    __syncwarp();
  }

  // ---------------------------------------------------------------- Z0 sweep
  // Z0 U = Y for k = s-1 .. 0: x_p,q = Pi^-1 y - sum_o (Pi^-1 z_o) x_o.  The
  // lane of row slot j accumulates the sum for the next level of that slot
  // (k - d, d = (k - j) mod W): when a level solves its pair, the pair is
  // broadcast and every lane adds its terms.
  static __device__ void z_solve(Sm4<B>& sm, const Paqif4Args& a, int dsys, int ssys, bool real, const L& ln,
                                 int& flag) {
    const int s = a.s, n = a.n;
    const int sg = ln.side, j = ln.j, u = ln.u;
    const float4* stk = a.stack + (size_t)ssys * s * C::SL;
    double* xs = a.x + (size_t)dsys * n;
    auto issue = [&](int c) {  // levels with v = s-1-k in [8c, 8c+8)
      if (!ln.live) return;
      const int v0 = c * C::CH, v1 = min(v0 + C::CH, s);
      if (v0 >= v1) return;
      const int k_lo = s - v1;
      const int nvec = (v1 - v0) * C::SL;
      const float4* src = stk + (size_t)k_lo * C::SL;
      for (int e = u; e < nvec; e += C::GS) {
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
    df acc = df_zero();
    df pend_x = df_zero();
    int pend_row = -1;
    auto store_x = [&](df xv, int row) {
      double d = A::to_double(xv);
      if (!isfinite(d) && flag == 0) flag = EHL_INFO_NONFINITE;
      if (a.mode == 1) d = d > 0.0 ? d : 0.0;
      if (real && ln.live && row < n) xs[row] = d;
    };
    int pj = (s - 1) % C::W;
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
      const int d = (pj - j + C::W) % C::W;  // this lane's next level is k - d
      df xv = df_zero();
      if (d == 0) {
        const float4 cv = sm.u.stk[v & (C::RB - 1)][2 * B];  // folded rhs column: Pi^-1 y
        xv = A::sub(sg ? make_df(cv.z, cv.w) : make_df(cv.x, cv.y), acc);
        acc = df_zero();
      }
      const df xp = shfl_df(xv, ln.gbase + pj), xq = shfl_df(xv, ln.gbase + C::W + pj);
      if (d == 0) {
        // the float64 conversion and store of the previous level run here, off
        // the path that the next level waits on
        if (pend_row >= 0) store_x(pend_x, pend_row);
        pend_x = xv;
        pend_row = sg ? s + k : s - 1 - k;
      } else if (k - d >= 0) {
        // terms of (x_p, x_q) of level k in level k - d: columns (left, d) and (right, d)
        const float4* lv = sm.u.stk[(v + d) & (C::RB - 1)];
        const float4 ml = lv[d - 1], mr = lv[B + d - 1];
        const df m1 = sg ? make_df(ml.z, ml.w) : make_df(ml.x, ml.y);
        const df m2 = sg ? make_df(mr.z, mr.w) : make_df(mr.x, mr.y);
        acc = A::sub_two_prods(acc, df_neg(m1), xp, df_neg(m2), xq);
      }
      pj = (pj == 0) ? B : pj - 1;
    }
    if (pend_row >= 0) store_x(pend_x, pend_row);
    cpa_wait<0>();
    __threadfence_block();
    __syncwarp();
  }

  static __device__ bool active_set_update(const Paqif4Args& a, int dsys, bool real, const L& ln) {
    const int n = a.n;
    const double* bsys = a.band + (size_t)dsys * n * C::BW;
    const double* xs = a.x + (size_t)dsys * n;
    int* as = a.act + (size_t)dsys * n;
    int changed = 0;
    if (real && ln.live) {
      for (int i = ln.u; i < n; i += C::GS) {
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
    const unsigned gmask = ((1u << C::GS) - 1u) << ln.gbase;
    const unsigned any = __ballot_sync(0xffffffffu, changed) & gmask;
    __threadfence_block();
    __syncwarp();
    return any != 0;
  }

  // the first nonzero flag among the group's lanes
  static __device__ int group_flag(int flag, const L& ln) {
    int f = 0;
#pragma unroll
    for (int i = 0; i < C::GS; ++i) {
      const int o = __shfl_sync(0xffffffffu, flag, ln.gbase + i);
      if (f == 0) f = o;
    }
    return f;
  }
};

// Groups past n_sys replay a real system's loads with their own stack slot and
// no other global stores, so every warp barrier and shuffle sees a full warp.
// Mode 2 runs active-set steps until no group of the warp changes its set (a
// converged group re-solves with the same set, reproducing the same x).
template <int B, bool F32>
__global__ void __launch_bounds__(32 * C4<B>::WARPS, 4) paqif4_kernel(Paqif4Args a) {
  using C = C4<B>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Lane4<B> ln;
  const int warp = threadIdx.x >> 5;
  Sm4<B>& sm = reinterpret_cast<Sm4<B>*>(smem_raw)[warp * C::G + ln.grp];
  const int ssys = (blockIdx.x * C::WARPS + warp) * C::G + ln.grp;
  const bool real = ssys < a.n_sys;
  const int dsys = real ? ssys : a.n_sys - 1;
  if (__all_sync(0xffffffffu, !real)) return;
  int flag = 0, solves = 0;
  bool more = real;
  const int max_solves = (a.mode == 2) ? kPaqifMaxActiveSetSteps : 1;
  for (int it = 0; it < max_solves; ++it) {
    P4<B, F32>::factor(sm, a, dsys, ssys, ln, flag);
    P4<B, F32>::z_solve(sm, a, dsys, ssys, real, ln, flag);
    if (more) ++solves;
    if (a.mode != 2) break;
    if (!P4<B, F32>::active_set_update(a, dsys, real, ln)) more = false;
    if (!__any_sync(0xffffffffu, more)) break;
  }
  int f = P4<B, F32>::group_flag(flag, ln);
  if (a.mode == 2 && more && f == 0) f = EHL_INFO_NOCONV;
  if (real && ln.live && ln.u == 0) {
    if (a.iters) a.iters[dsys] = solves;
    if (a.info) a.info[dsys] = f;
  }
}

// Solve only, with the factorization stored by a factor launch (same systems,
// same band): the W0 sweep for the new rhs, then the Z0 sweep.
template <int B, bool F32>
__global__ void __launch_bounds__(32 * C4<B>::WARPS, 4) paqif4_solve_kernel(Paqif4Args a) {
  using C = C4<B>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Lane4<B> ln;
  const int warp = threadIdx.x >> 5;
  Sm4<B>& sm = reinterpret_cast<Sm4<B>*>(smem_raw)[warp * C::G + ln.grp];
  const int ssys = (blockIdx.x * C::WARPS + warp) * C::G + ln.grp;
  const bool real = ssys < a.n_sys;
  const int dsys = real ? ssys : a.n_sys - 1;
  if (__all_sync(0xffffffffu, !real)) return;
  int flag = 0;
  P4<B, F32>::w_sweep(sm, a, dsys, ssys, ln);
  P4<B, F32>::z_solve(sm, a, dsys, ssys, real, ln, flag);
  const int f = P4<B, F32>::group_flag(flag, ln);
  if (real && ln.live && ln.u == 0 && a.info && f != 0) a.info[dsys] = f;
}

template <int B>
static size_t p4_smem() {
  return sizeof(Sm4<B>) * (size_t)(C4<B>::WARPS * C4<B>::G);
}
template <int B>
static int p4_per_cta() {
  return C4<B>::WARPS * C4<B>::G;
}
template <int B>
static int p4_fl() {
  return C4<B>::FL;
}

#define EHL_BETA_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8)

static bool p4_layout(int beta, int& per, int& fl) {
  switch (beta) {
#define EHL_CASE(BB)        \
  case BB:                  \
    per = p4_per_cta<BB>(); \
    fl = p4_fl<BB>();       \
    return true;
    EHL_BETA_CASES(EHL_CASE)
#undef EHL_CASE
    default:
      return false;
  }
}

size_t paqif_stack_bytes(int n_sys, int n, int beta) {
  int per = 0, fl = 0;
  if (!p4_layout(beta, per, fl)) return 0;
  const int s = (n + 1) / 2;
  const size_t padded = (size_t)((n_sys + per - 1) / per) * per;
  return padded * (size_t)s * (size_t)(2 * beta + 1) * sizeof(float4);
}

size_t paqif_factor_store_bytes(int n_sys, int n, int beta) {
  int per = 0, fl = 0;
  if (!p4_layout(beta, per, fl)) return 0;
  const int s = (n + 1) / 2;
  const size_t padded = (size_t)((n_sys + per - 1) / per) * per;
  return padded * (size_t)s * (size_t)fl * sizeof(float4);
}

// the dynamic shared-memory size of both kernels, set once per device
template <int B>
static cudaError_t p4_attrs() {
  static std::atomic<unsigned long long> set{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (set.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  const int smem = (int)p4_smem<B>();
  e = cudaFuncSetAttribute(paqif4_kernel<B, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(paqif4_solve_kernel<B, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(paqif4_kernel<B, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(paqif4_solve_kernel<B, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess && bit) set.fetch_or(bit, std::memory_order_release);
  return e;
}

cudaError_t paqif_prepare(int beta) {
  switch (beta) {
#define EHL_CASE(BB) \
  case BB:           \
    return p4_attrs<BB>();
    EHL_BETA_CASES(EHL_CASE)
#undef EHL_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <int B>
static cudaError_t launch4(const PaqifLaunch& L, cudaStream_t st, void* fstore, bool solve_only) {
  Paqif4Args a;
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
  const size_t smem = p4_smem<B>();
  const int per = p4_per_cta<B>();
  const int grid = (L.n_sys + per - 1) / per;
  cudaError_t e = p4_attrs<B>();
  if (e != cudaSuccess) return e;
  const bool f32 = L.f32 && L.mode != 2;
  if (solve_only) {
    if (f32)
      paqif4_solve_kernel<B, true><<<grid, 32 * C4<B>::WARPS, smem, st>>>(a);
    else
      paqif4_solve_kernel<B, false><<<grid, 32 * C4<B>::WARPS, smem, st>>>(a);
  } else {
    if (f32)
      paqif4_kernel<B, true><<<grid, 32 * C4<B>::WARPS, smem, st>>>(a);
    else
      paqif4_kernel<B, false><<<grid, 32 * C4<B>::WARPS, smem, st>>>(a);
  }
  note_launch();
  return cudaGetLastError();
}

// int8 mask -> int32 flags in the workspace (mode 2 rewrites them in place).
__global__ void expand_active_kernel(const uint8_t* __restrict__ in, int* __restrict__ out, size_t total) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < total; i += stride) out[i] = in ? (in[i] ? 1 : 0) : 0;
}

cudaError_t launch_expand_active(const uint8_t* in, int* out, size_t total, cudaStream_t st) {
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  expand_active_kernel<<<blocks, 256, 0, st>>>(in, out, total);
  note_launch();
  return cudaGetLastError();
}

static cudaError_t dispatch4(const PaqifLaunch& L, cudaStream_t st, void* fstore, bool solve_only) {
  switch (L.beta) {
#define EHL_CASE(BB) \
  case BB:           \
    return launch4<BB>(L, st, fstore, solve_only);
    EHL_BETA_CASES(EHL_CASE)
#undef EHL_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_paqif(const PaqifLaunch& L, cudaStream_t st) { return dispatch4(L, st, nullptr, false); }

cudaError_t launch_paqif_factor(const PaqifLaunch& L, void* fstore, cudaStream_t st) {
  if (L.mode == 2 || !fstore) return cudaErrorInvalidValue;
  return dispatch4(L, st, fstore, false);
}

cudaError_t launch_paqif_resolve(const PaqifLaunch& L, void* fstore, cudaStream_t st) {
  if (L.mode == 2 || !fstore) return cudaErrorInvalidValue;
  return dispatch4(L, st, fstore, true);
}

}  // namespace ehl
