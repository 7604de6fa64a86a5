// paqif.cu -- batched projected alternate quadrant interlocking factorization.
//
// Method (Sec. 2.2.1-2.2.3 of the paper; one partition per system, so the
// projection of Sec. 2.2.2 / Sec. 2.2.4 Steps 5 and 7 follows the solve):
// for an even order n = 2s, level k = 1..s takes the 2x2 pivot block on rows
// and columns (s-k+1, s+k) of the current Schur complement L0^(k): the rows
// of Z0 are that block's rows, the columns of W0 solve the 2x2 systems
//   z_pp w_ip + z_qp w_iq = l_ip,   z_pq w_ip + z_qq w_iq = l_iq,
// and L0^(k+1) = L0^(k) - w_p z_p^T - w_q z_q^T.  W0 Y = F is solved in the
// same middle-out sweep; Z0 U = Y is then solved from the two ends towards
// the middle with one 2x2 solve per level.
//
// GB300 mapping (this file's own design):
//  * one group of LS lanes per system, 32/LS systems per warp, all of a
//    warp's systems in lockstep (same n);
//  * for a band of half-width b only the (2b+2)^2 window of the Schur
//    complement on rows/columns {p-b..p} u {q..q+b} is ever non-trivial; it
//    lives in shared memory as a ring indexed by row mod (b+1), so moving
//    outwards one level overwrites the slots of the two eliminated pivots;
//  * band rows stream from HBM through cp.async into a 32-row ring per side,
//    two 8-row chunks ahead of use;
//  * every level pushes (Pi^-1 z_p, Pi^-1 z_q, Pi^-1 y) -- the Z0 rows
//    already multiplied by the inverse pivot -- onto a per-system stack in
//    the workspace; the ends-inwards Z0 solve reads it back in reverse with
//    16-byte cp.async.cg copies;
//  * arithmetic in double-float (df64.cuh), float64 only at the interface.
#include <cuda_runtime.h>
#include <stdint.h>

#include "df64.cuh"
#include "ehl_internal.h"

namespace ehl {

template <int B>
struct PaqifCfg {
  static constexpr int W = B + 1;        // window slots per side
  static constexpr int NS = 2 * W;       // window slots in all
  static constexpr int BW = 2 * B + 1;   // band row width
  static constexpr int NO = 2 * B;       // outer (non-pivot) indices per level
  static constexpr int LS = (B == 1) ? 4 : (B <= 3 ? 8 : (B <= 6 ? 16 : 32));
  static constexpr int G = 32 / LS;      // systems per warp
  static constexpr int RB = 32;          // staging ring rows per side
  static constexpr int CH = 8;           // rows per prefetch chunk
  static constexpr int STK = 4 * B + 2;  // stack entries per level
  static constexpr int NUPD = NO * NO;
  static constexpr int EPL = (NUPD + LS - 1) / LS;
  static constexpr int ACT_PER_LANE = (2 * CH + LS - 1) / LS;
};

template <int B>
struct __align__(16) SysSmem {
  using C = PaqifCfg<B>;
  df S[C::NS][C::NS];           // Schur-complement window
  df F[C::NS];                  // right-hand-side window (W0 Y = F sweep)
  df wb[C::NO][2];              // multipliers (w_ip, w_iq) of the outer rows
  union {
    double band[2][C::RB][C::BW];      // phase 1: band-row staging ring
    float2 stk[C::RB][C::STK];         // phase 2: Z-stack staging ring
  } u;
  double rhs[2][C::RB];
  int act[2][C::RB];
  df xr[2][C::W];               // phase 2: x of the last W levels per side
};
template <int B>
struct RingSizesMatch {
  static_assert(sizeof(double) * 2 * PaqifCfg<B>::BW == sizeof(float2) * PaqifCfg<B>::STK, "ring sizes");
  static constexpr bool ok = true;
};

struct PaqifArgs {
  int n_sys, n, s, mode;  // s = (n + 1) / 2 levels
  const double* band;
  const double* rhs;
  int* act;          // [n_sys][n] int32 active flags (workspace), or null
  float2* stack;     // [n_sys][s][STK]
  double* x;
  int* iters;
  int* info;
};

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16_cg(void* smem, const void* gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int B>
struct Paqif {
  using C = PaqifCfg<B>;

  // Stream index t >= 0 on side 0 (left) is row s-1-t, on side 1 (right) row s+t.
  static __device__ __forceinline__ int row_of(int side, int t, int s) { return side ? s + t : s - 1 - t; }

  // Issue the copies of prefetch chunk `c` (stream indices [8c, 8c+8)) of both sides.
  static __device__ __forceinline__ void issue_chunk(SysSmem<B>& sm, const PaqifArgs& a, int sys, int c, int u) {
    const int s = a.s, n = a.n;
    const double* bsys = a.band + (size_t)sys * n * C::BW;
    const double* rsys = a.rhs + (size_t)sys * n;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      // rows of this chunk, clipped to the real rows [0, n)
      int t0 = c * C::CH, t1 = t0 + C::CH - 1;
      int r_lo, r_hi;
      if (side == 0) {
        r_lo = s - 1 - t1;
        r_hi = s - 1 - t0;
      } else {
        r_lo = s + t0;
        r_hi = s + t1;
      }
      if (r_lo < 0) r_lo = 0;
      if (r_hi > n - 1) r_hi = n - 1;
      if (r_lo > r_hi) continue;
      int nel = (r_hi - r_lo + 1) * C::BW;
      for (int e = u; e < nel; e += C::LS) {
        int r = r_lo + e / C::BW, col = e % C::BW;
        int t = side ? r - s : s - 1 - r;
        cp_async8(&sm.u.band[side][t % C::RB][col], bsys + (size_t)r * C::BW + col);
      }
      for (int r = r_lo + u; r <= r_hi; r += C::LS) {
        int t = side ? r - s : s - 1 - r;
        cp_async8(&sm.rhs[side][t % C::RB], rsys + r);
      }
    }
  }

  // Active flags of chunk c: plain L2 loads into registers (the flags may
  // have been rewritten by this warp in the previous active-set step).
  static __device__ __forceinline__ void load_act_regs(int (&reg)[C::ACT_PER_LANE], const PaqifArgs& a, int sys,
                                                       int c, int u) {
#pragma unroll
    for (int m = 0; m < C::ACT_PER_LANE; ++m) {
      int e = u + m * C::LS;  // e in [0, 2*CH): side = e / CH, offset = e % CH
      reg[m] = 0;
      if (a.act != nullptr && e < 2 * C::CH) {
        int side = e / C::CH, t = c * C::CH + e % C::CH;
        int r = row_of(side, t, a.s);
        if (r >= 0 && r < a.n) reg[m] = __ldcg(a.act + (size_t)sys * a.n + r);
      }
    }
  }
  static __device__ __forceinline__ void store_act_regs(SysSmem<B>& sm, const int (&reg)[C::ACT_PER_LANE], int c,
                                                        int u) {
#pragma unroll
    for (int m = 0; m < C::ACT_PER_LANE; ++m) {
      int e = u + m * C::LS;
      if (e < 2 * C::CH) {
        int side = e / C::CH, t = c * C::CH + e % C::CH;
        sm.act[side][t % C::RB] = reg[m];
      }
    }
  }

  // Entry A[i][j] of the (padded, active-modified) matrix; rows i and j are
  // given by (side, stream index) pairs whose band rows sit in the ring.
  static __device__ __forceinline__ df entry(const SysSmem<B>& sm, int si, int ti, int sj, int tj, int s, int n) {
    int i = row_of(si, ti, s), j = row_of(sj, tj, s);
    int np = 2 * s;
    if (i < 0 || i >= np || j < 0 || j >= np) return df_zero();
    if (i >= n) return (i == j) ? make_df(1.f, 0.f) : df_zero();  // padding row
    if (j >= n) return df_zero();
    if (sm.act[si][ti % C::RB]) return (i == j) ? make_df(1.f, 0.f) : df_zero();
    int d = j - i;
    if (d < -B || d > B) return df_zero();
    return df_from_double(sm.u.band[si][ti % C::RB][B + d]);
  }
  static __device__ __forceinline__ df rhs_entry(const SysSmem<B>& sm, int side, int t, int s, int n) {
    int i = row_of(side, t, s);
    if (i < 0 || i >= n) return df_zero();
    if (sm.act[side][t % C::RB]) return df_zero();
    return df_from_double(sm.rhs[side][t % C::RB]);
  }

  // Window slot of stream index t on a side.
  static __device__ __forceinline__ int slot(int side, int t) { return side * C::W + t % C::W; }

  // Window slot and (side, t) of outer index o at level k.
  static __device__ __forceinline__ void outer(int o, int k, int& side, int& t) {
    if (o < B) {
      side = 0;
      t = k + 1 + o;
    } else {
      side = 1;
      t = k + 1 + (o - B);
    }
  }

  // Prefetch state of phase 1: chunks [0, issued) have been issued; the
  // registers hold the active flags of chunk issued-1, not yet in shared memory.
  struct Prefetch {
    int issued;
    int act_reg[C::ACT_PER_LANE];
  };

  static __device__ __forceinline__ void issue_next(SysSmem<B>& sm, const PaqifArgs& a, int dsys, int u, Prefetch& pf) {
    store_act_regs(sm, pf.act_reg, pf.issued - 1, u);
    load_act_regs(pf.act_reg, a, dsys, pf.issued, u);
    issue_chunk(sm, a, dsys, pf.issued, u);
    cp_async_commit();
    ++pf.issued;
  }

  // Middle-out sweep: the factorization of Sec. 2.2.3 fused with W0 Y = F.
  // `dsys` indexes the input data, `ssys` the stack slot (distinct for idle groups).
  static __device__ void factor_and_w_solve(SysSmem<B>& sm, const PaqifArgs& a, int dsys, int ssys, int u,
                                            int& flag) {
    const int s = a.s, n = a.n;
    float2* stk = a.stack + (size_t)ssys * s * C::STK;
    Prefetch pf;
    // prologue: chunks 0, 1 resident, chunk 2 in flight
    load_act_regs(pf.act_reg, a, dsys, 0, u);
    store_act_regs(sm, pf.act_reg, 0, u);
    load_act_regs(pf.act_reg, a, dsys, 1, u);
    issue_chunk(sm, a, dsys, 0, u);
    cp_async_commit();
    issue_chunk(sm, a, dsys, 1, u);
    cp_async_commit();
    pf.issued = 2;
    issue_next(sm, a, dsys, u, pf);  // stores chunk 1 flags, issues chunk 2
    cp_async_wait<1>();
    __syncwarp();

    // initial window: stream indices [0, B] on both sides
    for (int e = u; e < C::NS * C::NS; e += C::LS) {
      int r = e / C::NS, c = e % C::NS;
      int sr = r / C::W, tr = r % C::W, sc = c / C::W, tc = c % C::W;
      sm.S[r][c] = entry(sm, sr, tr, sc, tc, s, n);
    }
    for (int e = u; e < C::NS; e += C::LS) sm.F[e] = rhs_entry(sm, e / C::W, e % C::W, s, n);
    __syncwarp();

    for (int k = 0; k < s; ++k) {
      const int sp = slot(0, k), sq = slot(1, k);
      const df pa = sm.S[sp][sp], pb = sm.S[sp][sq], pc = sm.S[sq][sp], pd = sm.S[sq][sq];
      df det = df_det2(pa, pd, pb, pc);
      const float scale = fabsf(pa.hi * pd.hi) + fabsf(pb.hi * pc.hi);
      if (!(fabsf(det.hi) > 1e-13f * scale) || !(scale > 0.f)) {
        if (flag == 0) flag = EHL_INFO_SINGULAR;
        if (!(fabsf(det.hi) > 0.f)) det = make_df(1e-30f, 0.f);
      }
      const df inv = df_rcp(det);
      const df yp = sm.F[sp], yq = sm.F[sq];
      if (u < C::NO) {
        int side, t;
        outer(u, k, side, t);
        const int so = slot(side, t);
        const df sip = sm.S[so][sp], siq = sm.S[so][sq];
        // [w_ip, w_iq] = [l_ip, l_iq] Pi^{-1}
        const df wp = df_mul(df_det2(sip, pd, siq, pc), inv);
        const df wq = df_mul(df_det2(siq, pa, sip, pb), inv);
        sm.wb[u][0] = wp;
        sm.wb[u][1] = wq;
        sm.F[so] = df_sub_two_prods(sm.F[so], wp, yp, wq, yq);
        // folded Z0 rows: Pi^{-1} [z_p,o ; z_q,o]
        const df zpo = sm.S[sp][so], zqo = sm.S[sq][so];
        const df mp = df_mul(df_det2(pd, zpo, pb, zqo), inv);
        const df mq = df_mul(df_det2(pa, zqo, pc, zpo), inv);
        float2* dst = stk + (size_t)k * C::STK;
        dst[u] = make_float2(mp.hi, mp.lo);
        dst[C::NO + u] = make_float2(mq.hi, mq.lo);
      } else if (u == C::NO) {
        const df cp = df_mul(df_det2(pd, yp, pb, yq), inv);
        const df cq = df_mul(df_det2(pa, yq, pc, yp), inv);
        float2* dst = stk + (size_t)k * C::STK;
        dst[2 * C::NO] = make_float2(cp.hi, cp.lo);
        dst[2 * C::NO + 1] = make_float2(cq.hi, cq.lo);
      }
      __syncwarp();
      // rank-2 update of the outer block: L <- L - w_p z_p^T - w_q z_q^T
#pragma unroll
      for (int m = 0; m < C::EPL; ++m) {
        const int e = u + m * C::LS;
        if (e < C::NUPD) {
          const int o1 = e / C::NO, o2 = e % C::NO;
          int s1, t1, s2, t2;
          outer(o1, k, s1, t1);
          outer(o2, k, s2, t2);
          const int r = slot(s1, t1), c = slot(s2, t2);
          sm.S[r][c] = df_sub_two_prods(sm.S[r][c], sm.wb[o1][0], sm.S[sp][c], sm.wb[o1][1], sm.S[sq][c]);
        }
      }
      // the rows entering next have stream index tn on both sides; keep the
      // chunk holding tn resident and two more in flight
      const int tn = k + B + 1;
      if (pf.issued <= tn / C::CH + 2) {
        issue_next(sm, a, dsys, u, pf);
        cp_async_wait<2>();
      }
      __syncwarp();
      // new outer row/column on both sides, into the freed pivot slots
      for (int e = u; e < 4 * C::NS; e += C::LS) {
        const int side = e / (2 * C::NS);
        const int rem = e % (2 * C::NS);
        const int is_col = rem / C::NS;
        const int other = rem % C::NS;
        const int so = other / C::W;
        // stream index held by slot `other` in the window of level k+1
        const int to = k + 1 + (((other % C::W) - ((k + 1) % C::W)) % C::W + C::W) % C::W;
        const int sn = side ? sq : sp;
        if (!is_col) {
          sm.S[sn][other] = entry(sm, side, tn, so, to, s, n);
        } else if (other != sn) {
          sm.S[other][sn] = entry(sm, so, to, side, tn, s, n);
        }
      }
      if (u < 2) sm.F[u ? sq : sp] = rhs_entry(sm, u, tn, s, n);
      __syncwarp();
    }
    cp_async_wait<0>();
    __threadfence_block();
    __syncwarp();
  }

  // Z0 U = Y from both ends towards the middle, reading the stack in reverse.
  static __device__ void z_solve(SysSmem<B>& sm, const PaqifArgs& a, int dsys, int ssys, bool real, int u,
                                 int& flag) {
    const int s = a.s, n = a.n;
    const float2* stk = a.stack + (size_t)ssys * s * C::STK;
    double* xs = a.x + (size_t)dsys * n;
    for (int e = u; e < 2 * C::W; e += C::LS) sm.xr[e / C::W][e % C::W] = df_zero();
    // stream index v = s-1-k; chunk j holds v in [8j, 8j+8)
    auto issue = [&](int j) {
      const int v0 = j * C::CH;
      const int v1 = min(v0 + C::CH, s);
      if (v0 >= v1) return;
      // levels k in [s-v1, s-1-v0] are contiguous in memory
      const int k_lo = s - v1;
      const int nvec = (v1 - v0) * C::STK / 2;  // 16-byte vectors (STK is even)
      const float4* src = reinterpret_cast<const float4*>(stk + (size_t)k_lo * C::STK);
      for (int e = u; e < nvec; e += C::LS) {
        const int lvl = k_lo + (2 * e) / C::STK, off = (2 * e) % C::STK;
        const int v = s - 1 - lvl;
        cp_async16_cg(&sm.u.stk[v % C::RB][off], src + e);
      }
    };
    issue(0);
    cp_async_commit();
    issue(1);
    cp_async_commit();
    issue(2);
    cp_async_commit();
    cp_async_wait<2>();
    __syncwarp();
    for (int k = s - 1; k >= 0; --k) {
      const int v = s - 1 - k;
      if (v % C::CH == 0 && v > 0) {
        issue(v / C::CH + 2);
        cp_async_commit();
        cp_async_wait<2>();
        __syncwarp();
      }
      const float2* lv = sm.u.stk[v % C::RB];
      df sp_ = df_zero(), sq_ = df_zero();
      if (u < C::NO) {
        int side, t;
        outer(u, k, side, t);
        const df xo = sm.xr[side][t % C::W];
        const df mp = make_df(lv[u].x, lv[u].y), mq = make_df(lv[C::NO + u].x, lv[C::NO + u].y);
        sp_ = df_mul(mp, xo);
        sq_ = df_mul(mq, xo);
      }
#pragma unroll
      for (int off = C::LS / 2; off > 0; off >>= 1) {
        df op, oq;
        op.hi = __shfl_xor_sync(0xffffffffu, sp_.hi, off, C::LS);
        op.lo = __shfl_xor_sync(0xffffffffu, sp_.lo, off, C::LS);
        oq.hi = __shfl_xor_sync(0xffffffffu, sq_.hi, off, C::LS);
        oq.lo = __shfl_xor_sync(0xffffffffu, sq_.lo, off, C::LS);
        sp_ = df_add(sp_, op);
        sq_ = df_add(sq_, oq);
      }
      const df xp = df_sub(make_df(lv[2 * C::NO].x, lv[2 * C::NO].y), sp_);
      const df xq = df_sub(make_df(lv[2 * C::NO + 1].x, lv[2 * C::NO + 1].y), sq_);
      __syncwarp();
      if (u == 0) {
        sm.xr[0][k % C::W] = xp;
        sm.xr[1][k % C::W] = xq;
        const int p = s - 1 - k, q = s + k;
        double dp = df_to_double(xp), dq = df_to_double(xq);
        if ((!isfinite(dp) || !isfinite(dq)) && flag == 0) flag = EHL_INFO_NONFINITE;
        if (a.mode == 1) {
          dp = dp > 0.0 ? dp : 0.0;
          dq = dq > 0.0 ? dq : 0.0;
        }
        if (real) {
          xs[p] = dp;
          if (q < n) xs[q] = dq;
        }
      }
      __syncwarp();
    }
    cp_async_wait<0>();
    __threadfence_block();
    __syncwarp();
  }

  // One primal-dual active-set step for the LCP (mode 2): with w = A x - b,
  // a pinned row stays pinned while w_i > 0, a free row becomes pinned when
  // x_i < 0.  Returns, uniformly over the group, whether the set changed.
  static __device__ bool active_set_update(const PaqifArgs& a, int dsys, bool real, int u) {
    const int n = a.n;
    const double* bsys = a.band + (size_t)dsys * n * C::BW;
    const double* xs = a.x + (size_t)dsys * n;
    int* as = a.act + (size_t)dsys * n;
    int changed = 0;
    if (real) {
      for (int i = u; i < n; i += C::LS) {
        df w = df_neg(df_from_double(a.rhs[(size_t)dsys * n + i]));
#pragma unroll
        for (int j = 0; j < C::BW; ++j) {
          const int c = i - B + j;
          if (c >= 0 && c < n)
            w = df_fma(df_from_double(__ldg(bsys + (size_t)i * C::BW + j)), df_from_double(__ldcg(xs + c)), w);
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

// One group of LS lanes per system.  Groups past n_sys ("idle") replay a real
// system's loads with their own stack slot and no other global stores, so
// every __syncwarp / shuffle sees the full warp.  The active-set loop of mode
// 2 runs until no group of the warp changes its set (a converged group
// re-solves with the same set, which reproduces the same x).
template <int B>
__global__ void __launch_bounds__(128) paqif_kernel(PaqifArgs a) {
  using C = PaqifCfg<B>;
  static_assert(RingSizesMatch<B>::ok, "");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / C::LS, u = lane % C::LS;
  SysSmem<B>& sm = reinterpret_cast<SysSmem<B>*>(smem_raw)[warp * C::G + grp];
  const int ssys = (blockIdx.x * (blockDim.x >> 5) + warp) * C::G + grp;
  const bool real = ssys < a.n_sys;
  const int dsys = real ? ssys : a.n_sys - 1;
  if (__all_sync(0xffffffffu, !real)) return;

  int flag = 0;
  int solves = 0;
  bool more = real;
  const int max_solves = (a.mode == 2) ? kPaqifMaxActiveSetSteps : 1;
  for (int it = 0; it < max_solves; ++it) {
    Paqif<B>::factor_and_w_solve(sm, a, dsys, ssys, u, flag);
    Paqif<B>::z_solve(sm, a, dsys, ssys, real, u, flag);
    if (more) ++solves;
    if (a.mode != 2) {
      more = false;
      break;
    }
    const bool changed = Paqif<B>::active_set_update(a, dsys, real, u);
    if (!changed) more = false;
    if (!__any_sync(0xffffffffu, more)) break;
  }
  if (a.mode == 2 && more && flag == 0) flag = EHL_INFO_NOCONV;
  if (real && u == 0) {
    if (a.iters) a.iters[dsys] = solves;
    if (a.info) a.info[dsys] = flag;
  }
}

// int8 mask -> int32 flags in the workspace (mode 2 rewrites them in place).
__global__ void expand_active_kernel(const uint8_t* __restrict__ in, int* __restrict__ out, size_t total) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < total; i += stride) out[i] = in ? (in[i] ? 1 : 0) : 0;
}

template <int B>
static size_t paqif_smem_bytes() {
  return sizeof(SysSmem<B>) * (size_t)(kPaqifWarpsPerCta * PaqifCfg<B>::G);
}

template <int B>
static int paqif_systems_per_cta() {
  return kPaqifWarpsPerCta * PaqifCfg<B>::G;
}

size_t paqif_stack_bytes(int n_sys, int n, int beta) {
  const int s = (n + 1) / 2;
  int per_cta = 0;
  switch (beta) {
#define EHL_CASE(B) \
  case B:           \
    per_cta = paqif_systems_per_cta<B>(); \
    break;
    EHL_CASE(1) EHL_CASE(2) EHL_CASE(3) EHL_CASE(4) EHL_CASE(5) EHL_CASE(6) EHL_CASE(7) EHL_CASE(8)
#undef EHL_CASE
    default:
      return 0;
  }
  const size_t padded = (size_t)((n_sys + per_cta - 1) / per_cta) * per_cta;
  return padded * (size_t)s * (size_t)(4 * beta + 2) * sizeof(float2);
}

template <int B>
static cudaError_t launch_paqif_b(const PaqifLaunch& L, cudaStream_t st) {
  PaqifArgs a;
  a.n_sys = L.n_sys;
  a.n = L.n;
  a.s = (L.n + 1) / 2;
  a.mode = L.mode;
  a.band = L.band;
  a.rhs = L.rhs;
  a.act = L.act;
  a.stack = reinterpret_cast<float2*>(L.stack);
  a.x = L.x;
  a.iters = L.iters;
  a.info = L.info;
  const size_t smem = paqif_smem_bytes<B>();
  cudaError_t e = cudaFuncSetAttribute(paqif_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int per_cta = paqif_systems_per_cta<B>();
  const int grid = (L.n_sys + per_cta - 1) / per_cta;
  paqif_kernel<B><<<grid, 32 * kPaqifWarpsPerCta, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_expand_active(const uint8_t* in, int* out, size_t total, cudaStream_t st) {
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  expand_active_kernel<<<blocks, 256, 0, st>>>(in, out, total);
  return cudaGetLastError();
}

cudaError_t launch_paqif(const PaqifLaunch& L, cudaStream_t st) {
  switch (L.beta) {
    case 1: return launch_paqif_b<1>(L, st);
    case 2: return launch_paqif_b<2>(L, st);
    case 3: return launch_paqif_b<3>(L, st);
    case 4: return launch_paqif_b<4>(L, st);
    case 5: return launch_paqif_b<5>(L, st);
    case 6: return launch_paqif_b<6>(L, st);
    case 7: return launch_paqif_b<7>(L, st);
    case 8: return launch_paqif_b<8>(L, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ehl
