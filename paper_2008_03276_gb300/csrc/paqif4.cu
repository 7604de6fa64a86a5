// paqif4.cu -- batched PAQIF (projected alternate quadrant interlocking factorization),
// one lane per row of the elimination window, r partitions per system.
//
// Method (Sec. 2.2.1-2.2.3): for a block of order 2s, level k = 0..s-1 pivots
// on the rows/columns at stream index k of the two sides (rows s-1-k and s+k)
// of the Schur complement L0^(k); the Z0 rows are the pivot rows, the W0
// columns solve
//   z_pp w_ip + z_qp w_iq = l_ip,   z_pq w_ip + z_qq w_iq = l_iq,
// and L0^(k+1) = L0^(k) - w_p z_p^T - w_q z_q^T.  W0 Y = F runs in the same
// middle-out sweep; Z0 U = Y runs from both ends towards the middle with one
// 2x2 solve per level.
//
// Partitioning (Sec. 2.1, Eq. eqnn16; Sec. 2.2.4 Steps 1-7): a system is cut
// into r diagonal blocks L0^(m) of order n_p.  Each block is factored and
// swept only over its interior levels (Steps 1, 2); because the middle-out
// order eliminates the interior first, what is left in the window is the
// Schur complement of the block on its first and last b unknowns, with the
// transformed right-hand side.  Those 2b r unknowns satisfy a reduced system:
// the Schur complements on the block diagonal, and the untouched band
// entries that couple the last b rows of a block with the first b columns of
// the next one (and vice versa) off it (Steps 3, 4: the paper's reduced
// system premultiplied by the inverse of W0's outer block, same solution).
// It is block tridiagonal with b x b blocks and is solved by block
// elimination without pivoting (instead of the paper's normal equations,
// which square its conditioning).  The Z0 sweep of each block then starts
// from the known outer unknowns (Step 6).  The projection onto U >= 0
// (Steps 5, 7) is applied once, after the full solve, so the result does not
// depend on r.
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
//  * band rows stream from HBM with cp.async into a ring per side, converted
//    float64 -> double-float once, in place, by the lane that copied them.
//  * the Z0 and W0 sweeps rotate roles instead of data: the lane that owns a
//    row slot accumulates the terms of the level that slot holds next, and the
//    solved pair of each level is broadcast with warp shuffles.
//  * the r blocks of a system are r groups of one CTA; the reduced system is
//    assembled in shared memory and solved by the group of block 0 between two
//    CTA barriers.
//  * arithmetic is double-float (df64.cuh); float64 only at the interface.
#include <cuda_runtime.h>
#include <stdint.h>

#include <math.h>

#include <atomic>

#include "df64.cuh"
#include "ehl_internal.h"
#include "paqif_pair.h"

namespace ehl {

template <int B>
struct C4 {
  static constexpr int W = B + 1;             // row slots per side (stream indices k..k+b)
  static constexpr int GS = 2 * W;            // lanes per block, one per window row
  static constexpr int G = 32 / GS;           // groups per warp
  static constexpr int NC = GS + 1;           // window columns: (side, distance) then the rhs
  static constexpr int RHS = GS;              // column index of the rhs
  static constexpr int BW = 2 * B + 1;        // band row width
  static constexpr int SL = 2 * B + 1;        // stack float4 per level: (M_p, M_q) per outer column, rhs last
  static constexpr int FL = GS;               // factor-store float4 per level: one per row slot
  static constexpr int RB = (B <= 4) ? 16 : 32;  // ring rows per side
  static constexpr int CH = RB / 4;           // rows per chunk (b <= CH keeps the live window in the ring)
  // warps per CTA: 8 at b = 8 (one group per warp), so that a system can be cut into up to
  // 8 blocks within one CTA; 4 below
  static constexpr int WARPS = (B == 8) ? 8 : 4;
  static constexpr int GPC = WARPS * G;       // groups per CTA
  static constexpr int BB = B * B;
  // resident CTAs per SM the register budget is set for: 5 x 4 warps up to b = 4 (shared
  // memory allows 5), 4 x 4 warps for b = 5..7, 2 x 8 warps at b = 8
  static constexpr int MINB = (B <= 4) ? 5 : (B == 8 ? 2 : 4);
};

// reduced-system blocks of one partition: blocks 2m (first b rows) and 2m+1
// (last b rows), each with its sub-diagonal, diagonal and super-diagonal b x b block
template <int B>
struct RedBlk {
  float2 T[2][3][B * B];
};

template <int B>
struct __align__(16) Sm4 {
  using C = C4<B>;
  float4 zb[2][C::NC];  // the two pivot rows of a level (z_p, z_q) per column, double-buffered
  union {
    double ring[2][C::RB][C::BW];  // band rows: float64 as copied, double-float after conversion
    float4 stk[C::RB][C::SL];      // Z0 sweep: stack levels
    float4 fr[C::RB][C::FL];       // W0 sweep of a resolve: factor-store levels
    RedBlk<B> red;                 // reduced system, between the sweeps
  } u;
  double rrhs[2][C::RB];
  int ract[2][C::RB];
  float2 fo[2 * B];  // transformed rhs of the block's outer rows (first b rows, then last b)
  float2 xo[2 * B];  // their solution
  int flag;
  int more;
};

struct Paqif4Args {
  int n_sys, n, mode;
  int r, np, sp, sf;  // blocks per system, block order (even), its levels, levels swept per block
  int spc;            // systems per CTA
  const double* band;
  const double* rhs;
  int* act;
  float4* stack;   // [groups][sp][SL]
  float4* fstore;  // [groups][sp][FL]: multipliers and Pi^-1 rows (factor once, solve many), or null
  float2* rstore;  // [systems][2r][3][b^2]: reduced factors L_b, D_b^-1, U_b (with fstore), or null
  double* x;
  int* iters;
  int* info;
};

// one block of one system, as a PAQIF problem of its own
struct Part4 {
  const double* band;  // first row of the block
  const double* rhs;
  const int* act;
  double* x;
  float4* stk;
  float4* fst;
  int n;     // real rows of the block (rows n..2s-1 are identity rows)
  int s;     // levels of the block
  int sf;    // levels swept (s for one block per system, s - b with a reduced system)
  int m, r;  // block index, blocks per system
  int mode;
  int ng;    // order of the system
  int row0;  // first row of the block in the system
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
  static __device__ __forceinline__ void chunk(Sm4<B>& sm, const Part4& p, int c, const L& ln) {
    if (!ln.live) return;
    const int s = p.s, n = p.n, u = ln.u;
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
          cpa8(dst, p.band + (size_t)r * C::BW + col);
        }
      }
      for (int r = r_lo + u; r <= r_hi; r += C::GS) {
        const int t = side ? r - s : s - 1 - r;
        double* dst = &sm.rrhs[side][t & (C::RB - 1)];
        if (CONVERT) {
          const df v = A::from_double(*dst);
          *reinterpret_cast<float2*>(dst) = make_float2(v.hi, v.lo);
          sm.ract[side][t & (C::RB - 1)] = p.act ? __ldcg(p.act + r) : 0;
        } else {
          cpa8(dst, p.rhs + r);
        }
      }
    }
  }

  // 0: outside the block, 1: a real row, 2: an identity row (padding or active)
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
  // index among the block's 2b outer unknowns (first b rows, then last b) of stream t on a side
  static __device__ __forceinline__ int outer_index(int side, int t, int s) {
    return side ? t - s + 2 * B : s - 1 - t;
  }

  // ---------------------------------------------------------------- factor
  // Levels 0..sf-1 of L0 = W0 Z0 with the rhs column (W0 Y = F) along; the
  // folded outer columns of every level go to the stack.  With sf < s the
  // window left over is the block's part of the reduced system.
  static __device__ void factor(Sm4<B>& sm, const Part4& p, const L& ln, int& flag) {
    const int s = p.s, n = p.n;
    const int sg = ln.side, j = ln.j;
    // prologue: chunks 0..3 issued, 0 and 1 converted; afterwards chunks
    // [0, conv) are double-float and chunks up to conv+1 are issued
    chunk<false>(sm, p, 0, ln);
    cpa_commit();
    chunk<false>(sm, p, 1, ln);
    cpa_commit();
    chunk<false>(sm, p, 2, ln);
    cpa_commit();
    chunk<false>(sm, p, 3, ln);
    cpa_commit();
    cpa_wait<2>();
    chunk<true>(sm, p, 0, ln);
    chunk<true>(sm, p, 1, ln);
    __syncwarp();
    int conv = 2;
    // the window of level 0: this lane's row is stream index j; column
    // (side c / W, distance c % W) is stream index c % W
    df R[C::NC];
    int kind = row_kind(sm, sg, j, s, n);
#pragma unroll
    for (int c = 0; c < C::NC; ++c)
      R[c] = (c == C::RHS) ? rhs_of(sm, sg, j, kind) : any_entry(sm, sg, j, c / C::W, c % C::W, kind, s, n);

    int off = j;  // this lane's row is stream index k + off (0: a pivot row)
    for (int k = 0; k < p.sf; ++k) {
      const bool piv = (off == 0);
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
      if (p.fst && ln.live) p.fst[(size_t)k * C::FL + ln.u] = make_float4(al.hi, al.lo, be.hi, be.lo);
      // rank-2 update of an outer row / folded outer columns of a pivot row
#pragma unroll
      for (int c = 0; c < C::NC; ++c) {
        if (c == 0 || c == C::W) continue;
        const float4 z = zb[c];
        const df o = A::sub_two_prods(piv ? df_zero() : R[c], al, make_df(z.x, z.y), be, make_df(z.z, z.w));
        if (piv && ln.live) reinterpret_cast<float2*>(p.stk + (size_t)k * C::SL + sidx(c))[sg] = df2f(o);
        R[c] = o;  // a pivot row's registers are replaced by the incoming row below
      }
      // the columns move one step towards the pivot
#pragma unroll
      for (int sd = 0; sd < 2; ++sd)
#pragma unroll
        for (int d = 1; d <= B; ++d) R[sd * C::W + d - 1] = R[sd * C::W + d];
      // rows entering at the end of this level have stream index tn on both sides; away from
      // the block's ends every column the incoming row and column touch lies inside it
      const int tn = k + C::W;
      const bool inner = (tn < s) && (s + tn < n);
      if (tn >= conv * C::CH) {
        // issue chunk conv+2 into the slots of chunk conv-2 (stream indices
        // below CH (conv-1) <= tn - b, no longer referenced); then at most the
        // two newest groups are pending
        chunk<false>(sm, p, conv + 2, ln);
        cpa_commit();
        cpa_wait<2>();
        chunk<true>(sm, p, conv, ln);
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
              if (inner || col_in(sg, k + 1 + d, s, n)) v = band_at(sm, sg, tn, sg ? d : 2 * B - d);
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
        const int dd = C::W - off;
        df v = df_zero();
        if (kind == 1 && (inner || col_in(sg, tn, s, n))) v = band_at(sm, sg, tn - dd, sg ? B + dd : B - dd);
        R[B] = sg ? df_zero() : v;
        R[C::W + B] = sg ? v : df_zero();
      }
      off = (off == 0) ? B : off - 1;
    }
    cpa_wait<0>();
    __threadfence_block();
    __syncwarp();
    if (p.sf < s) outer_out(sm, p, ln, R, off);
  }

  // The block's part of the reduced system: the 2b x 2b Schur complement left
  // in the window (rows and columns at stream indices sf..s-1 of both sides)
  // and the transformed rhs, then the band entries coupling its first b rows
  // to the last b columns of the previous block and its last b rows to the
  // first b columns of the next.
  static __device__ void outer_out(Sm4<B>& sm, const Part4& p, const L& ln, const df (&R)[C::NC], int off) {
    const int s = p.s, sg = ln.side;
    const int tr = p.sf + off;  // stream index of this lane's row
    if (tr <= s - 1 && ln.live) {
      const int o = outer_index(sg, tr, s);
      const int h = sg, rb = o - h * B;  // block (first / last rows) and row in it
#pragma unroll
      for (int sd = 0; sd < 2; ++sd)
#pragma unroll
        for (int d = 0; d < B; ++d) {
          // column (side sd, distance d) is stream sf + d: outer index B - 1 - d (left), B + d (right)
          const int cb = sd ? d : B - 1 - d;
          const int which = (sd == h) ? 1 : (h == 0 ? 2 : 0);
          sm.u.red.T[h][which][rb * B + cb] = df2f(R[sd * C::W + d]);
        }
      sm.fo[o] = df2f(R[C::RHS]);
    }
    if (ln.live) {
      for (int e = ln.u; e < 2 * C::BB; e += C::GS) {
        const int part = e / C::BB, i = (e / B) % B, jj = e % B;
        df v = df_zero();
        if (part == 0) {
          // row i of the block, column row0 - b + jj of the previous block (band offset jj - i)
          const int lr = i;
          if (p.m > 0 && jj >= i && lr < p.n && !(p.act && __ldcg(p.act + lr)))
            v = A::from_double(__ldg(p.band + (size_t)lr * C::BW + (jj - i)));
        } else {
          // row 2s - b + i of the block, column row0 + 2s + jj of the next block (band offset 2b - i + jj)
          const int lr = 2 * s - B + i;
          if (p.m < p.r - 1 && jj <= i && lr < p.n && p.row0 + 2 * s + jj < p.ng && !(p.act && __ldcg(p.act + lr)))
            v = A::from_double(__ldg(p.band + (size_t)lr * C::BW + (2 * B - i + jj)));
        }
        sm.u.red.T[part][part == 0 ? 0 : 2][i * B + jj] = df2f(v);
      }
    }
    __syncwarp();
  }

  // ---------------------------------------------------------------- solve only
  // W0 Y = F for a new right-hand side with the multipliers of a stored
  // factorization: the pivot pair (y_p, y_q) of a level is broadcast, the
  // outer rows take F_o -= w_o,p y_p + w_o,q y_q, and Pi^-1 (y_p, y_q)
  // replaces the folded rhs column of the stack level for the Z0 sweep.
  static __device__ void w_sweep(Sm4<B>& sm, const Part4& p, const L& ln) {
    const int s = p.s, n = p.n;
    const int sg = ln.side, j = ln.j, u = ln.u;
    // rhs and flags by chunk of CH stream indices per side, staged in rrhs/ract;
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
          cpa8(&sm.rrhs[side][(side ? r - s : s - 1 - r) & (C::RB - 1)], p.rhs + r);
      }
      const int k0 = t0, k1 = min(t0 + C::CH, p.sf);
      for (int e = u; e < (k1 - k0) * C::FL; e += C::GS) {
        const int lvl = k0 + e / C::FL, off = e % C::FL;
        cpa16cg(&fring[lvl & (C::RB - 1)][off], p.fst + (size_t)lvl * C::FL + off);
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
          sm.ract[side][t] = p.act ? __ldcg(p.act + r) : 0;
        }
      }
    };
    // chunk c = rhs of stream indices [CH c, CH c + CH) and factor-store levels
    // of the same range.  Level k reads level k and the rhs of stream
    // k + b + 1 <= k + CH + 1, so at k = CH c chunks c..c+2 must be complete
    // and chunk c-1 is free.
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
    for (int k = 0; k < p.sf; ++k) {
      if (k > 0 && k % C::CH == 0) {
        // issue chunk c+3 into the slots of chunk c-1, then all but the newest
        // group are complete: chunk c+2 can be converted
        issue(k / C::CH + 3);
        cpa_commit();
        cpa_wait<1>();
        convert(k / C::CH + 2);
        __syncwarp();
      }
      const df yp = shfl_df(F, ln.gbase + pj), yq = shfl_df(F, ln.gbase + C::W + pj);
      const float4 f = fring[k & (C::RB - 1)][u];
      const bool piv = (j == pj);
      const df o = A::sub_two_prods(piv ? df_zero() : F, make_df(f.x, f.y), yp, make_df(f.z, f.w), yq);
      if (piv) {
        if (ln.live) reinterpret_cast<float2*>(p.stk + (size_t)k * C::SL + 2 * B)[sg] = df2f(o);
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
    if (p.sf < s) {
      const int tr = p.sf + (j - pj + C::W) % C::W;
      if (tr <= s - 1 && ln.live) sm.fo[outer_index(sg, tr, s)] = df2f(F);
      __syncwarp();
    }
  }

  // ---------------------------------------------------------------- Z0 sweep
  // Z0 U = Y for k = s-1 .. 0: x_p,q = Pi^-1 y - sum_o (Pi^-1 z_o) x_o.  The
  // lane of row slot j accumulates the sum for the next level of that slot
  // (k - d, d = (k - j) mod W): when a level solves its pair, the pair is
  // broadcast and every lane adds its terms.  Levels sf..s-1 (the outer
  // unknowns of a block) come from the reduced system.
  static __device__ void z_solve(Sm4<B>& sm, const Part4& p, bool real, const L& ln, int& flag) {
    const int s = p.s, sf = p.sf, n = p.n;
    const int sg = ln.side, j = ln.j, u = ln.u;
    auto issue = [&](int c) {  // levels with v = sf-1-k in [CH c, CH c + CH)
      if (!ln.live) return;
      const int v0 = c * C::CH, v1 = min(v0 + C::CH, sf);
      if (v0 >= v1) return;
      const int k_lo = sf - v1;
      const int nvec = (v1 - v0) * C::SL;
      const float4* src = p.stk + (size_t)k_lo * C::SL;
      for (int e = u; e < nvec; e += C::GS) {
        const int lvl = k_lo + e / C::SL, off = e % C::SL;
        cpa16cg(&sm.u.stk[(sf - 1 - lvl) & (C::RB - 1)][off], src + e);
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
    // The solution leaves in float64, a conversion on the FP64 pipe (1/64 of the FP32 rate)
    // that costs a warp instruction's full time however few lanes are active.  So the pair
    // solved at level k (sweep position v = s-1-k) is kept in double-float in the rhs ring,
    // free during this sweep, and every RB levels all lanes of the group convert and store
    // the rows it holds: rows v of the left side, 2s-1-v of the right.
    float2(*xb)[C::RB] = reinterpret_cast<float2(*)[C::RB]>(sm.rrhs);
    auto flush = [&](int base, int cnt) {  // positions base .. base+cnt-1 of both sides
      __syncwarp();
      if (ln.live) {
#pragma unroll
        for (int e = u; e < 2 * C::RB; e += C::GS) {
          const int side = e / C::RB, i = e % C::RB;
          if (i < cnt) {
            // the sign and finiteness of hi + lo are those of hi (|lo| <= ulp(hi) / 2)
            const df xv = f2df(xb[side][i]);
            const int row = side ? 2 * s - 1 - (base + i) : base + i;
            if (!isfinite(xv.hi) && flag == 0) flag = EHL_INFO_NONFINITE;
            const double dv = (p.mode == 1 && !(xv.hi > 0.f)) ? 0.0 : A::to_double(xv);
            if (real && row < n) p.x[row] = dv;
          }
        }
      }
      __syncwarp();
    };
    auto keep = [&](int k, int dk, df xv) {  // after the level's pair is known (dk == 0: solved here)
      const int v = s - 1 - k;
      if (dk == 0 && ln.live) xb[sg][v & (C::RB - 1)] = df2f(xv);
      if ((v & (C::RB - 1)) == C::RB - 1) flush(v - (C::RB - 1), C::RB);
    };
    // terms of the pair (x_p, x_q) of level k in level k - d (columns (left, d) and (right, d))
    auto push = [&](int k, int d, df xp, df xq) {
      const float4* lv = sm.u.stk[(sf - 1 - (k - d)) & (C::RB - 1)];
      const float4 ml = lv[d - 1], mr = lv[B + d - 1];
      const df m1 = sg ? make_df(ml.z, ml.w) : make_df(ml.x, ml.y);
      const df m2 = sg ? make_df(mr.z, mr.w) : make_df(mr.x, mr.y);
      acc = A::sub_two_prods(acc, df_neg(m1), xp, df_neg(m2), xq);
    };
    int pj = (s - 1) % C::W;
    int d = (pj - j + C::W) % C::W;  // this lane's next level is k - d
    // the outer levels, known from the reduced system
    for (int k = s - 1; k >= sf; --k) {
      df xv = df_zero();
      if (d == 0) xv = f2df(sm.xo[outer_index(sg, k, s)]);
      const df xp = shfl_df(xv, ln.gbase + pj), xq = shfl_df(xv, ln.gbase + C::W + pj);
      if (d != 0 && k - d >= 0 && k - d < sf) push(k, d, xp, xq);
      keep(k, d, xv);
      pj = (pj == 0) ? B : pj - 1;
      d = (d == 0) ? B : d - 1;
    }
    for (int k = sf - 1; k >= 0; --k) {
      const int v = sf - 1 - k;
      if (v > 0 && v % C::CH == 0) {
        // at v = CH c: chunk c+2 replaces chunk c-2, then chunks <= c+1 are complete
        issue(issued);
        cpa_commit();
        ++issued;
        cpa_wait<1>();
        __syncwarp();
      }
      df xv = df_zero();
      if (d == 0) {
        const float4 cv = sm.u.stk[v & (C::RB - 1)][2 * B];  // folded rhs column: Pi^-1 y
        xv = A::sub(sg ? make_df(cv.z, cv.w) : make_df(cv.x, cv.y), acc);
        acc = df_zero();
      }
      const df xp = shfl_df(xv, ln.gbase + pj), xq = shfl_df(xv, ln.gbase + C::W + pj);
      if (d != 0 && k - d >= 0) push(k, d, xp, xq);
      keep(k, d, xv);
      pj = (pj == 0) ? B : pj - 1;
      d = (d == 0) ? B : d - 1;
    }
    if (((s - 1) & (C::RB - 1)) != C::RB - 1) flush((s - 1) & ~(C::RB - 1), ((s - 1) & (C::RB - 1)) + 1);
    cpa_wait<0>();
    __threadfence_block();
    __syncwarp();
  }

  // ---------------------------------------------------------------- reduced system
  // Block tridiagonal, 2r blocks of b unknowns (block 2m: the first b rows of
  // partition m, block 2m+1: its last b rows), eliminated without pivoting:
  //   L_q = T_q,q-1 D_{q-1}^-1,  D_q = T_q,q - L_q T_q-1,q,
  //   y_q = f_q - L_q y_{q-1},   x_q = D_q^-1 (y_q - T_q,q+1 x_{q+1}).
  // Run by the group of partition 0 of each system; every group of the warp
  // executes the same loops (uniform barriers), only the leaders store.
  static __device__ __forceinline__ float2* blk(Sm4<B>* ss, int q, int which) {
    return ss[q >> 1].u.red.T[q & 1][which];
  }
  static __device__ __forceinline__ float2* vec(Sm4<B>* ss, int q, bool x) {
    return (x ? ss[q >> 1].xo : ss[q >> 1].fo) + (q & 1) * B;
  }
  static constexpr int NE = (C::BB + C::GS - 1) / C::GS;  // matrix entries per lane

  // C = A X (store = true) or C -= A X into dst, entries e = u, u + GS, ...
  static __device__ __forceinline__ void matmul(const float2* Am, const float2* Xm, float2* dst, bool sub, bool st,
                                                const L& ln) {
    df tmp[NE];
#pragma unroll
    for (int t = 0; t < NE; ++t) {
      const int e = min(ln.u + t * C::GS, C::BB - 1);
      const int i = e / B, jj = e % B;
      df a = sub ? f2df(dst[e]) : df_zero();
#pragma unroll
      for (int q = 0; q < B; q += 2) {
        const df a0 = f2df(Am[i * B + q]), x0 = f2df(Xm[q * B + jj]);
        const df a1 = (q + 1 < B) ? f2df(Am[i * B + q + 1]) : df_zero();
        const df x1 = (q + 1 < B) ? f2df(Xm[(q + 1) * B + jj]) : df_zero();
        a = sub ? A::sub_two_prods(a, a0, x0, a1, x1) : A::sub_two_prods(a, df_neg(a0), x0, df_neg(a1), x1);
      }
      tmp[t] = a;
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < NE; ++t) {
      const int e = ln.u + t * C::GS;
      if (st && e < C::BB) dst[e] = df2f(tmp[t]);
    }
    __syncwarp();
  }
  // y = f - A x, row i by the lane pair (2i, 2i+1): each lane takes every other term, the
  // pair adds its halves with one shuffle (the reduced solve's dependent chain is b/2 terms)
  static __device__ __forceinline__ void matvec_sub(const float2* Am, const float2* xv, const float2* fv, float2* dst,
                                                    bool st, const L& ln) {
    const int i = min(ln.u >> 1, B - 1), h = ln.u & 1;
    df a = h ? df_zero() : f2df(fv[i]);
#pragma unroll
    for (int q = 0; q < B; q += 4) {
      const int q0 = q + h, q1 = q + 2 + h;
      const df a0 = (q0 < B) ? f2df(Am[i * B + q0]) : df_zero(), x0 = (q0 < B) ? f2df(xv[q0]) : df_zero();
      const df a1 = (q1 < B) ? f2df(Am[i * B + q1]) : df_zero(), x1 = (q1 < B) ? f2df(xv[q1]) : df_zero();
      a = A::sub_two_prods(a, a0, x0, a1, x1);
    }
    a = df_add(a, make_df(__shfl_xor_sync(0xffffffffu, a.hi, 1), __shfl_xor_sync(0xffffffffu, a.lo, 1)));
    __syncwarp();
    if (st && h == 0 && (ln.u >> 1) < B) dst[ln.u >> 1] = df2f(a);
    __syncwarp();
  }
  // y = A x, by lane pairs as above
  static __device__ __forceinline__ void matvec(const float2* Am, const float2* xv, float2* dst, bool st,
                                                const L& ln) {
    const int i = min(ln.u >> 1, B - 1), h = ln.u & 1;
    df a = df_zero();
#pragma unroll
    for (int q = 0; q < B; q += 4) {
      const int q0 = q + h, q1 = q + 2 + h;
      const df a0 = (q0 < B) ? f2df(Am[i * B + q0]) : df_zero(), x0 = (q0 < B) ? f2df(xv[q0]) : df_zero();
      const df a1 = (q1 < B) ? f2df(Am[i * B + q1]) : df_zero(), x1 = (q1 < B) ? f2df(xv[q1]) : df_zero();
      a = A::sub_two_prods(a, df_neg(a0), x0, df_neg(a1), x1);
    }
    a = df_add(a, make_df(__shfl_xor_sync(0xffffffffu, a.hi, 1), __shfl_xor_sync(0xffffffffu, a.lo, 1)));
    __syncwarp();
    if (st && h == 0 && (ln.u >> 1) < B) dst[ln.u >> 1] = df2f(a);
    __syncwarp();
  }
  // in-place inverse by Gauss-Jordan elimination without pivoting
  static __device__ void invert(float2* M, bool st, const L& ln, int& flag) {
    for (int q = 0; q < B; ++q) {
      const df piv = f2df(M[q * B + q]);
      if (!(fabsf(piv.hi) > 0.f) && st && flag == 0) flag = EHL_INFO_SINGULAR;
      const df ip = A::rcp((fabsf(piv.hi) > 0.f) ? piv : make_df(1e-30f, 0.f));
      df tmp[NE];
#pragma unroll
      for (int t = 0; t < NE; ++t) {
        const int e = min(ln.u + t * C::GS, C::BB - 1);
        const int i = e / B, jj = e % B;
        const df mij = f2df(M[e]), miq = f2df(M[i * B + q]), mqj = f2df(M[q * B + jj]);
        df v;
        if (i == q && jj == q)
          v = ip;
        else if (i == q)
          v = A::mul(mqj, ip);
        else if (jj == q)
          v = df_neg(A::mul(miq, ip));
        else
          v = A::sub_two_prods(mij, A::mul(miq, ip), mqj, df_zero(), df_zero());
        tmp[t] = v;
      }
      __syncwarp();
#pragma unroll
      for (int t = 0; t < NE; ++t) {
        const int e = ln.u + t * C::GS;
        if (st && e < C::BB) M[e] = df2f(tmp[t]);
      }
      __syncwarp();
    }
  }

  // Factor the reduced system of the system whose partitions are ss[0..r-1]
  // (T blocks and fo filled by outer_out), solve it into xo, and keep the
  // factors in rst when given.
  static __device__ void reduced_factor(Sm4<B>* ss, int r, bool leader, float2* rst, const L& ln, int& flag) {
    const bool st = leader && ln.live;
    const int nb = 2 * r;
    for (int q = 0; q < nb; ++q) {
      if (q > 0) {
        matmul(blk(ss, q, 0), blk(ss, q - 1, 1), blk(ss, q, 0), false, st, ln);  // L_q = T_q,q-1 D^-1
        matmul(blk(ss, q, 0), blk(ss, q - 1, 2), blk(ss, q, 1), true, st, ln);   // D_q -= L_q T_q-1,q
      }
      invert(blk(ss, q, 1), st, ln, flag);
    }
    if (rst && st) {
      for (int q = 0; q < nb; ++q)
        for (int w = 0; w < 3; ++w)
          for (int e = ln.u; e < C::BB; e += C::GS) rst[((size_t)q * 3 + w) * C::BB + e] = blk(ss, q, w)[e];
    }
    __syncwarp();
    reduced_substitute(ss, r, leader, ln);
  }
  // forward and backward substitution with the factors in the T blocks
  static __device__ void reduced_substitute(Sm4<B>* ss, int r, bool leader, const L& ln) {
    const bool st = leader && ln.live;
    const int nb = 2 * r;
    // y_0 = f_0 (into xo), y_q = f_q - L_q y_{q-1}
    if (st && ln.u < B) vec(ss, 0, true)[ln.u] = vec(ss, 0, false)[ln.u];
    __syncwarp();
    for (int q = 1; q < nb; ++q) matvec_sub(blk(ss, q, 0), vec(ss, q - 1, true), vec(ss, q, false), vec(ss, q, true), st, ln);
    // x_q = D_q^-1 (y_q - T_q,q+1 x_{q+1}), the bracket staged in fo
    for (int q = nb - 1; q >= 0; --q) {
      if (q < nb - 1)
        matvec_sub(blk(ss, q, 2), vec(ss, q + 1, true), vec(ss, q, true), vec(ss, q, false), st, ln);
      else {
        if (st && ln.u < B) vec(ss, q, false)[ln.u] = vec(ss, q, true)[ln.u];
        __syncwarp();
      }
      matvec(blk(ss, q, 1), vec(ss, q, false), vec(ss, q, true), st, ln);
    }
  }
  // a resolve: the stored factors back into the T blocks, then the substitution
  static __device__ void reduced_resolve(Sm4<B>* ss, int r, bool leader, const float2* rst, const L& ln) {
    const bool st = leader && ln.live;
    const int nb = 2 * r;
    if (st) {
      for (int q = 0; q < nb; ++q)
        for (int w = 0; w < 3; ++w)
          for (int e = ln.u; e < C::BB; e += C::GS) blk(ss, q, w)[e] = __ldcg(rst + ((size_t)q * 3 + w) * C::BB + e);
    }
    __syncwarp();
    reduced_substitute(ss, r, leader, ln);
  }

  // Mode 2: new active set of rows [r_lo, r_hi) of the system from x (all of
  // the system's rows written); returns whether any row of the group changed.
  static __device__ bool active_set_update(const Paqif4Args& a, int dsys, int r_lo, int r_hi, bool real,
                                           const L& ln) {
    const int n = a.n;
    const double* bsys = a.band + (size_t)dsys * n * C::BW;
    const double* xs = a.x + (size_t)dsys * n;
    int* as = a.act + (size_t)dsys * n;
    int changed = 0;
    if (real && ln.live) {
      for (int i = r_lo + ln.u; i < r_hi; i += C::GS) {
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

  static __device__ Part4 part(const Paqif4Args& a, int dsys, int m, int gidx) {
    Part4 p;
    p.row0 = m * a.np;
    p.n = min(max(a.n - p.row0, 0), a.np);
    p.band = a.band + ((size_t)dsys * a.n + p.row0) * C::BW;
    p.rhs = a.rhs + (size_t)dsys * a.n + p.row0;
    p.act = a.act ? a.act + (size_t)dsys * a.n + p.row0 : nullptr;
    p.x = a.x + (size_t)dsys * a.n + p.row0;
    p.stk = a.stack + (size_t)gidx * a.sp * C::SL;
    p.fst = a.fstore ? a.fstore + (size_t)gidx * a.sp * C::FL : nullptr;
    p.s = a.sp;
    p.sf = a.sf;
    p.m = m;
    p.r = a.r;
    p.mode = a.mode;
    p.ng = a.n;
    return p;
  }
};

// One CTA holds spc systems of r partitions each, one group of lanes per
// partition.  Groups of a padding system replay the last real system's loads
// with their own stack slots and no other global stores, so every warp and CTA
// barrier sees all threads.  Mode 2 runs active-set steps until no system of
// the CTA changes its set (a converged system re-solves with the same set,
// reproducing the same x).
template <int B, bool F32>
__global__ void __launch_bounds__(32 * C4<B>::WARPS, C4<B>::MINB) paqif4_kernel(Paqif4Args a) {
  using C = C4<B>;
  using K = P4<B, F32>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Lane4<B> ln;
  const int warp = threadIdx.x >> 5;
  Sm4<B>* smb = reinterpret_cast<Sm4<B>*>(smem_raw);
  const int gc = warp * C::G + ln.grp;
  const int sysl = gc / a.r, m = gc - sysl * a.r;
  Sm4<B>& sm = smb[gc];
  Sm4<B>* ss = smb + sysl * a.r;
  const int sys = blockIdx.x * a.spc + sysl;
  const bool real = sys < a.n_sys;
  const int dsys = real ? sys : a.n_sys - 1;
  if (a.r == 1 && __all_sync(0xffffffffu, !real)) return;  // no CTA barriers with one partition
  const Part4 p = K::part(a, dsys, m, blockIdx.x * C::GPC + gc);
  float2* rst = a.rstore ? a.rstore + (size_t)sys * 2 * a.r * 3 * C::BB : nullptr;
  int flag = 0, solves = 0;
  bool more = real;
  const int max_solves = (a.mode == 2) ? kPaqifMaxActiveSetSteps : 1;
  for (int it = 0; it < max_solves; ++it) {
    K::factor(sm, p, ln, flag);
    if (a.r > 1) {
      __syncthreads();
      K::reduced_factor(ss, a.r, m == 0, real ? rst : nullptr, ln, flag);
      __syncthreads();
    }
    K::z_solve(sm, p, real, ln, flag);
    if (more) ++solves;
    if (a.mode != 2) break;
    if (a.r == 1) {
      if (!K::active_set_update(a, dsys, 0, a.n, real, ln)) more = false;
      if (!__any_sync(0xffffffffu, more)) break;
    } else {
      __syncthreads();  // x of every partition is written
      const bool ch = K::active_set_update(a, dsys, p.row0, p.row0 + p.n, real, ln);
      if (ln.live && ln.u == 0) sm.more = ch ? 1 : 0;
      __syncthreads();
      int any = 0;
      for (int q = 0; q < a.r; ++q) any |= ss[q].more;
      if (!any) more = false;
      if (!__syncthreads_or(more ? 1 : 0)) break;
    }
  }
  int f = K::group_flag(flag, ln);
  if (a.r > 1) {
    if (ln.live && ln.u == 0) sm.flag = f;
    __syncthreads();
    f = 0;
    for (int q = 0; q < a.r; ++q)
      if (f == 0) f = ss[q].flag;
  }
  if (a.mode == 2 && more && f == 0) f = EHL_INFO_NOCONV;
  if (real && ln.live && ln.u == 0 && m == 0) {
    if (a.iters) a.iters[dsys] = solves;
    if (a.info) a.info[dsys] = f;
  }
}

// Solve only, with the factorization stored by a factor launch (same systems,
// same band): the W0 sweep for the new rhs, the reduced system, then the Z0 sweep.
template <int B, bool F32>
__global__ void __launch_bounds__(32 * C4<B>::WARPS, C4<B>::MINB) paqif4_solve_kernel(Paqif4Args a) {
  using C = C4<B>;
  using K = P4<B, F32>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Lane4<B> ln;
  const int warp = threadIdx.x >> 5;
  Sm4<B>* smb = reinterpret_cast<Sm4<B>*>(smem_raw);
  const int gc = warp * C::G + ln.grp;
  const int sysl = gc / a.r, m = gc - sysl * a.r;
  Sm4<B>& sm = smb[gc];
  Sm4<B>* ss = smb + sysl * a.r;
  const int sys = blockIdx.x * a.spc + sysl;
  const bool real = sys < a.n_sys;
  const int dsys = real ? sys : a.n_sys - 1;
  if (a.r == 1 && __all_sync(0xffffffffu, !real)) return;
  const Part4 p = K::part(a, dsys, m, blockIdx.x * C::GPC + gc);
  int flag = 0;
  K::w_sweep(sm, p, ln);
  if (a.r > 1) {
    __syncthreads();
    K::reduced_resolve(ss, a.r, m == 0, a.rstore + (size_t)(real ? sys : 0) * 2 * a.r * 3 * C::BB, ln);
    __syncthreads();
  }
  K::z_solve(sm, p, real, ln, flag);
  int f = K::group_flag(flag, ln);
  if (a.r > 1) {
    if (ln.live && ln.u == 0) sm.flag = f;
    __syncthreads();
    f = 0;
    for (int q = 0; q < a.r; ++q)
      if (f == 0) f = ss[q].flag;
  }
  if (real && ln.live && ln.u == 0 && m == 0 && a.info && f != 0) a.info[dsys] = f;
}

template <int B>
static size_t p4_smem() {
  return sizeof(Sm4<B>) * (size_t)C4<B>::GPC;
}

#define EHL_BETA_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8)

static int groups_per_cta(int beta) {
  switch (beta) {
#define EHL_CASE(BB) \
  case BB:           \
    return C4<BB>::GPC;
    EHL_BETA_CASES(EHL_CASE)
#undef EHL_CASE
    default:
      return 0;
  }
}

// Partition geometry: r blocks of even order np = 2 ceil(n / 2r), each with
// at least one interior level (np >= 2 beta + 2) and at least one real row;
// r divides the groups of a CTA.
struct Geom {
  int r, np, sp, sf, spc, grid;
};
static bool geom_ok(int n_sys, int n, int beta, int r, Geom& g) {
  const int gpc = groups_per_cta(beta);
  if (gpc == 0 || r < 1 || gpc % r != 0) return false;
  g.r = r;
  g.sp = (n + 2 * r - 1) / (2 * r);
  g.np = 2 * g.sp;
  if (r > 1 && (g.np < 2 * beta + 2 || (r - 1) * g.np >= n)) return false;
  g.sf = (r > 1) ? g.sp - beta : g.sp;
  g.spc = gpc / r;
  g.grid = (n_sys + g.spc - 1) / g.spc;
  return true;
}

template <int B>
static int p4_resident_ctas() {  // CTAs per SM: the register budget, then 227 KB of shared memory
  const int by_smem = (int)((227u * 1024u) / p4_smem<B>());
  return by_smem < C4<B>::MINB ? by_smem : C4<B>::MINB;
}
static int resident_ctas(int beta) {
  switch (beta) {
#define EHL_CASE(BB) \
  case BB:           \
    return p4_resident_ctas<BB>();
    EHL_BETA_CASES(EHL_CASE)
#undef EHL_CASE
    default:
      return 1;
  }
}

// The automatic choice: among the admissible r that keep the batch within two
// rounds of resident groups, the one with the shortest chain per group -- its
// sweep levels (sf) plus the 2r block steps of its system's reduced system,
// counted as b levels each -- and on a tie the larger r if the batch still fits
// in one round.  Measured (CUDA events): the standalone batch (4096 x n = 1024,
// b = 4, 20 warps per SM) takes 1.76, 1.21, 1.24, 1.12, 1.21 ms for r = 1, 2,
// 3, 4, 6 (the choice: 4); 512 x n = 1025 at b = 8 (16 warps per SM) 1.46,
// 0.93, 0.68, 0.88 ms for r = 1, 2, 4, 8 (4); 64 x n = 1025 at b = 8 0.50 and
// 0.32 ms for r = 4, 8 (8); one system of n = 4097 at b = 8 5.77, 3.57, 1.83,
// 0.99 ms (8).
int paqif_parts(int n_sys, int n, int beta, int requested) {
  Geom g;
  if (requested > 0) return geom_ok(n_sys, n, beta, requested, g) ? requested : -1;
  const int gpc = groups_per_cta(beta);
  if (gpc == 0 || n_sys < 1 || !geom_ok(n_sys, n, beta, 1, g)) return -1;
  const long long resident = (long long)kSmCount * resident_ctas(beta) * gpc;
  int best = 1;
  long long best_chain = g.sf;
  for (int r = 2; r <= gpc; ++r) {
    const long long groups = (long long)n_sys * r;
    if (groups > 2 * resident) break;
    if (!geom_ok(n_sys, n, beta, r, g)) continue;
    const long long chain = g.sf + 2LL * beta * r;
    if (chain < best_chain || (chain == best_chain && groups <= resident)) {
      best = r;
      best_chain = chain;
    }
  }
  return best;
}

static bool geom(int n_sys, int n, int beta, int parts, Geom& g) {
  const int r = paqif_parts(n_sys, n, beta, parts);
  return r > 0 && geom_ok(n_sys, n, beta, r, g);
}

size_t paqif_stack_bytes(int n_sys, int n, int beta, int parts) {
  Geom g;
  if (!geom(n_sys, n, beta, parts, g)) return 0;
  const size_t own = (size_t)g.grid * groups_per_cta(beta) * (size_t)g.sp * (size_t)(2 * beta + 1) * sizeof(float4);
  // the automatic choice may run the lane-pair kernel (modes 0 and 1): room for its stack too
  const int rp = parts == 0 ? paqif_pair_parts(n_sys, n, beta, 0, false, false) : 0;
  const size_t pair = rp > 0 ? paqif_pair_stack_bytes(n_sys, n, beta, rp) : 0;
  return own > pair ? own : pair;
}

static size_t reduced_store_bytes(const Geom& g, int beta) {
  return g.r > 1 ? (size_t)g.grid * g.spc * (size_t)(2 * g.r * 3 * beta * beta) * sizeof(float2) : 0;
}

size_t paqif_factor_store_bytes(int n_sys, int n, int beta, int parts) {
  Geom g;
  if (!geom(n_sys, n, beta, parts, g)) return 0;
  const size_t groups = (size_t)g.grid * groups_per_cta(beta) * (size_t)g.sp * (size_t)(2 * beta + 2) * sizeof(float4);
  return align_up(groups, kWorkspaceAlign) + reduced_store_bytes(g, beta);
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
  const cudaError_t e = paqif_pair_prepare(beta);
  if (e != cudaSuccess) return e;
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
  Geom g;
  if (!geom(L.n_sys, L.n, B, L.parts, g)) return cudaErrorInvalidValue;
  Paqif4Args a;
  a.n_sys = L.n_sys;
  a.n = L.n;
  a.mode = L.mode;
  a.r = g.r;
  a.np = g.np;
  a.sp = g.sp;
  a.sf = g.sf;
  a.spc = g.spc;
  a.band = L.band;
  a.rhs = L.rhs;
  a.act = L.act;
  a.stack = reinterpret_cast<float4*>(L.stack);
  a.fstore = reinterpret_cast<float4*>(fstore);
  a.rstore = nullptr;
  if (fstore && g.r > 1) {
    const size_t groups = (size_t)g.grid * C4<B>::GPC * (size_t)g.sp * C4<B>::FL * sizeof(float4);
    a.rstore = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(fstore) + align_up(groups, kWorkspaceAlign));
  }
  a.x = L.x;
  a.iters = L.iters;
  a.info = L.info;
  const size_t smem = p4_smem<B>();
  cudaError_t e = p4_attrs<B>();
  if (e != cudaSuccess) return e;
  const bool f32 = L.f32 && L.mode != 2;
  if (solve_only) {
    if (f32)
      paqif4_solve_kernel<B, true><<<g.grid, 32 * C4<B>::WARPS, smem, st>>>(a);
    else
      paqif4_solve_kernel<B, false><<<g.grid, 32 * C4<B>::WARPS, smem, st>>>(a);
  } else {
    if (f32)
      paqif4_kernel<B, true><<<g.grid, 32 * C4<B>::WARPS, smem, st>>>(a);
    else
      paqif4_kernel<B, false><<<g.grid, 32 * C4<B>::WARPS, smem, st>>>(a);
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
  if (blocks > kSmCount * 16) blocks = kSmCount * 16;
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

// The automatic choice (parts = 0) of a solve in modes 0 and 1 with float64 sweeps, b <= 4 and a
// band array on a 16-byte boundary runs the lane-pair kernel (paqif_pair.cu); everything else (a
// requested partition count, mode 2, float32 sweeps, a stored factorization, b > 4) this file's.
cudaError_t launch_paqif(const PaqifLaunch& L, cudaStream_t st) {
  if (L.parts == 0 && (reinterpret_cast<uintptr_t>(L.band) & 15u) == 0) {
    const int rp = paqif_pair_parts(L.n_sys, L.n, L.beta, L.mode, L.f32, false);
    if (rp > 0) return launch_paqif_pair(L, rp, st);
  }
  return dispatch4(L, st, nullptr, false);
}

cudaError_t launch_paqif_factor(const PaqifLaunch& L, void* fstore, cudaStream_t st) {
  if (L.mode == 2 || !fstore) return cudaErrorInvalidValue;
  return dispatch4(L, st, fstore, false);
}

cudaError_t launch_paqif_resolve(const PaqifLaunch& L, void* fstore, cudaStream_t st) {
  if (L.mode == 2 || !fstore) return cudaErrorInvalidValue;
  return dispatch4(L, st, fstore, true);
}

}  // namespace ehl
