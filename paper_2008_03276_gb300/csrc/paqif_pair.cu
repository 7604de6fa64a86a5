// paqif_pair.cu -- batched PAQIF (Sec. 2.2.1-2.2.4) for half-bands b <= 4 with one lane per side
// of a block: the lane keeps its side's b + 1 rows of the elimination window in registers, so a
// level costs two warp shuffles of the pivot rows and otherwise only the lane's own arithmetic.
//
// Method (as in paqif4.cu): a block of order 2s is factored middle-out; level k pivots on the
// rows/columns at stream index k of the two sides (rows s-1-k and s+k of the block) with the 2x2
// block Pi = [[z_pp, z_pq], [z_qp, z_qq]]; an outer row i takes the multipliers
// w_i = [l_ip, l_iq] Pi^-1 and L0^(k+1) = L0^(k) - w_p z_p^T - w_q z_q^T; the rhs column rides
// along (W0 Y = F).  The pivot rows, folded as Pi^-1 [z_p; z_q] on the outer columns and the rhs,
// go to a stack that the Z0 sweep reads back from the block's ends towards its middle.  With r > 1
// blocks per system (Sec. 2.1, Eq. eqnn16; Sec. 2.2.4) the last b levels of a block are left out:
// the window then holds the Schur complement of the block on its first and last b unknowns, and
// these 2 b r unknowns of the system solve a block-tridiagonal reduced system (block elimination
// without pivoting, in shared memory, by the 2r lanes of the system).  The projection of mode 1
// is applied to the full solution, so the result does not depend on r.
//
// GB300 mapping:
//  * lane (block, side): 16 blocks per warp, the r blocks of a system in one warp (r | 16);
//  * the window is stored relative to the lane's side: column (own, d) is stream k + d of the
//    lane's side, (other, d) the same stream of the other side, d = 0..b, plus the rhs; the
//    columns move one slot towards the pivot each level (register renaming in a rolled loop);
//    the rank-2 update runs column by column, so each result lands on an entry already consumed;
//  * a band row enters the window through a two-row cp.async ring in shared memory, copied two
//    levels ahead; its entries beyond the window (up to b columns) wait in registers;
//  * the stack is interleaved by lane ([warp][level][word][lane]): a warp's stores and loads of
//    one level are coalesced;
//  * double-float arithmetic (df64.cuh); float64 only at the interface.
#include <cuda_runtime.h>
#include <stdint.h>

#include <math.h>

#include <atomic>

#include "df64.cuh"
#include "ehl_internal.h"
#include "paqif_pair.h"

namespace ehl {

namespace {

constexpr int kPairThreads = 128;  // 4 warps, 64 blocks per CTA
constexpr int kPairBlocksPerCta = kPairThreads / 2;
constexpr int kRingLane = 13 * 16;  // ring bytes per lane: 2 rows x (b + 2) x 16 used, the rest skews banks

template <int B>
struct PC {
  static constexpr int W = B + 1;          // window rows per side, column slots per side
  static constexpr int BW = 2 * B + 1;     // band row width
  static constexpr int NS = 2 * B + 1;     // stack entries per lane and level: own d = 1..b, other d = 1..b, rhs
  static constexpr int NQ = (NS + 1) / 2;  // float4 words per lane and level
  static constexpr int BB = B * B;
  static constexpr int SLOT = 16 * (B + 2);  // ring slot: the aligned words around a row, then its rhs
  // resident CTAs per SM the register budget is set for (65536 / (128 x registers))
  static constexpr int MINB = (B == 1) ? 6 : (B == 2 ? 4 : (B == 3 ? 3 : 2));
};

struct PairArgs {
  int n_sys, n, mode;
  int r, np, s, sf;  // blocks per system, block order 2s, levels s, levels swept (s - b if r > 1)
  const double* band;
  const double* rhs;
  const int* act;
  float4* stack;  // [warps][sf][NQ][32 lanes]
  double* x;
  int* iters;
  int* info;
};

// reduced-system storage of one warp: block row q of the warp (the lane that owns those rows):
// its sub-diagonal, diagonal and super-diagonal b x b blocks, the rhs and the solution
template <int B>
struct RedWarp {
  float2 T[32][3][PC<B>::BB];
  float2 f[32][B];
  float2 xs[32][B];
};

// shared memory of one warp: the row rings of its lanes and its reduced system during the
// factorization, then, in the same bytes, the Z0 sweep's stack rings of its lanes (DEPTH levels
// each, at most 8; lane stride skewed by 16 bytes against bank conflicts)
template <int B>
struct WarpSm {
  static constexpr int BYTES = 32 * kRingLane + (int)sizeof(RedWarp<B>);
  static constexpr int FIT = (BYTES / 32 - 16) / (PC<B>::NQ * 16);
  static constexpr int DEPTH = FIT < 8 ? FIT : 8;
  static constexpr int Z0LANE = DEPTH * PC<B>::NQ * 16 + 16;
  static_assert(DEPTH >= 2 && 32 * Z0LANE <= BYTES && BYTES % 16 == 0, "Z0 ring layout");
};

__device__ __forceinline__ df f2df(float2 v) { return make_df(v.x, v.y); }
__device__ __forceinline__ float2 df2f(df v) { return make_float2(v.hi, v.lo); }
__device__ __forceinline__ df shfl_x1(df v) {
  return make_df(__shfl_xor_sync(0xffffffffu, v.hi, 1), __shfl_xor_sync(0xffffffffu, v.lo, 1));
}
__device__ __forceinline__ df sel(bool c, df a, df b) { return c ? a : b; }

// local row of stream t on a side of a block of order 2s
__device__ __forceinline__ int row_of(int side, int t, int s) { return side ? s + t : s - 1 - t; }

struct PairBlk {
  const double* band;  // row 0 of the block
  const double* rhs;
  const int* act;
  double* x;
  const double* band_end;  // one past the last row of the whole band array (which starts 16-byte aligned)
  float4* stk;             // this lane's word 0 of level 0 (stride 32 between words)
  int s, nb;               // levels; real rows of the block (rows nb..2s-1 are identity rows)
  int side;
};

// A[i][c] of the block (local indices): 0 outside the block's real rows and the band;
// identity rows (padding, active) have their 1 on the diagonal
__device__ __forceinline__ df block_entry(const PairBlk& p, int B, int i, int c) {
  if (i < 0 || i >= 2 * p.s || c < 0 || c >= 2 * p.s) return df_zero();
  if (i >= p.nb || (p.act && __ldg(p.act + i))) return (i == c) ? make_df(1.f, 0.f) : df_zero();
  if (c >= p.nb || c - i > B || i - c > B) return df_zero();
  return df_from_double(__ldg(p.band + (size_t)i * (2 * B + 1) + (B + c - i)));
}

template <int B>
struct RowMeta {
  int i;  // local row
  bool odd, real, ident;
};

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) { return (uint32_t)__cvta_generic_to_shared(ptr); }
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Start the copy of the row of stream t on this lane's side into ring slot `slot` (one commit
// group): the 16-byte aligned words around the row (the array starts on a 16-byte boundary, so
// the word before an odd row is inside it; past the array's end nothing is read, cp.async fills
// zeros), then the rhs.  Rows that are not read copy nothing.  The copies go through L1
// (.ca): consecutive rows of a lane share 128-byte lines (4 % faster than .cg).
template <int B>
__device__ __forceinline__ RowMeta<B> fetch_row(const PairBlk& p, int t, unsigned char* slot) {
  using C = PC<B>;
  RowMeta<B> o;
  const int i = row_of(p.side, t, p.s);
  const bool exists = t < p.s;
  o.i = i;
  o.ident = exists && (i >= p.nb || (p.act && __ldg(p.act + i)));
  o.real = exists && !o.ident;
  const double* a = p.band + (size_t)(o.real ? i : 0) * C::BW;
  o.odd = (reinterpret_cast<uintptr_t>(a) & 15u) != 0;
  const double2* a2 = reinterpret_cast<const double2*>(a - (o.odd ? 1 : 0));
  const int full = o.real ? 16 : 0;
#pragma unroll
  for (int q = 0; q < B; ++q) cp_async16(slot + 16 * q, a2 + q, full);
  const bool last_whole = reinterpret_cast<const double*>(a2 + B) + 2 <= p.band_end;
  cp_async16(slot + 16 * B, a2 + B, o.real ? (last_whole ? 16 : 8) : 0);
  cp_async8(slot + 16 * (B + 1), p.rhs + (o.real ? i : 0), o.real ? 8 : 0);
  cp_commit();
  return o;
}

// Place a fetched row (its copy complete) at window slot b: its own-side window columns are the
// streams t - b .. t at distances b - d (other-side columns are zero), its next b own-side
// columns wait in fut.
template <int B>
__device__ __forceinline__ void place_row(const PairBlk& p, const RowMeta<B>& o, const unsigned char* slot,
                                          df (&own)[PC<B>::W], df& rhs, double (&fut)[B]) {
  const double r = *reinterpret_cast<const double*>(slot + 16 * (B + 1));
  const int sd = p.side, i = o.i;
  // away from the block's ends (every lane of the warp): no range checks, and each entry read at
  // the lane's own offset instead of selected among the staged words
  if (__all_sync(0xffffffffu, o.real && i >= B && i < p.nb - B)) {
    const double* row = reinterpret_cast<const double*>(slot) + (o.odd ? 1 : 0);
#pragma unroll
    for (int d = 0; d <= B; ++d) own[d] = df_from_double_sel(row[sd ? d : 2 * B - d]);
#pragma unroll
    for (int q = 0; q < B; ++q) fut[q] = row[sd ? B + 1 + q : B - 1 - q];
    rhs = df_from_double_sel(r);
    return;
  }
  double v[2 * B + 2];
#pragma unroll
  for (int q = 0; q <= B; ++q) {
    const double2 w = *reinterpret_cast<const double2*>(slot + 16 * q);
    v[2 * q] = w.x;
    v[2 * q + 1] = w.y;
  }
  auto bq = [&](int q) { return o.odd ? v[q + 1] : v[q]; };
#pragma unroll
  for (int d = 0; d <= B; ++d) {
    // left: column i + b - d (band 2b - d); right: i - b + d (band d)
    const int col = sd ? i - B + d : i + B - d;
    const double e = (o.real && col < p.nb) ? (sd ? bq(d) : bq(2 * B - d)) : 0.0;
    own[d] = o.ident ? (d == B ? make_df(1.f, 0.f) : df_zero()) : df_from_double_sel(e);
  }
#pragma unroll
  for (int q = 0; q < B; ++q) {
    // column stream t + 1 + q: left i - 1 - q (band b - 1 - q), right i + 1 + q (band b + 1 + q)
    const int col = sd ? i + 1 + q : i - 1 - q;
    fut[q] = (o.real && col >= 0 && col < p.nb) ? (sd ? bq(B + 1 + q) : bq(B - 1 - q)) : 0.0;
  }
  rhs = o.real ? df_from_double_sel(r) : df_zero();
}

// ------------------------------------------------------------------ reduced system
// Block tridiagonal, 2r block rows of b unknowns per system (row 2m: the first b rows of block m,
// row 2m+1: its last b rows), in the warp's shared storage at index (lane of the owner):
//   L_q = T_q,q-1 D_{q-1}^-1,  D_q = T_q,q - L_q T_q-1,q,  y_q = f_q - L_q y_{q-1},
//   x_q = D_q^-1 (y_q - T_q,q+1 x_{q+1});  D_q^-1 by Gauss-Jordan elimination without pivoting.
// The 2r lanes of a system share the b x b entries; every system of the warp runs the same steps.
template <int B>
struct Red {
  using C = PC<B>;
  static constexpr int NT = (C::BB + 3) / 4;  // entries per lane, at least 4 lanes per system
  // C = A X (sub = false) or C = C - A X; entries e = u, u + nl, ... of the b x b result
  static __device__ __forceinline__ void matmul(const float2* Am, const float2* Xm, float2* Cm, bool sub, int u,
                                                int nl) {
    df tmp[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int e = u + t * nl;
      df a = df_zero();
      if (e < C::BB) {
        const int i = e / B, jj = e % B;
        a = sub ? f2df(Cm[e]) : df_zero();
#pragma unroll
        for (int q = 0; q < B; q += 2) {
          const df a0 = f2df(Am[i * B + q]), x0 = f2df(Xm[q * B + jj]);
          const df a1 = (q + 1 < B) ? f2df(Am[i * B + q + 1]) : df_zero();
          const df x1 = (q + 1 < B) ? f2df(Xm[(q + 1) * B + jj]) : df_zero();
          a = sub ? df_sub_two_prods(a, a0, x0, a1, x1) : df_sub_two_prods(a, df_neg(a0), x0, df_neg(a1), x1);
        }
      }
      tmp[t] = a;
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int e = u + t * nl;
      if (e < C::BB) Cm[e] = df2f(tmp[t]);
    }
    __syncwarp();
  }
  static __device__ void invert(float2* M, int u, int nl, int& flag) {
    for (int q = 0; q < B; ++q) {
      const df piv = f2df(M[q * B + q]);
      if (!(fabsf(piv.hi) > 0.f) && flag == 0) flag = EHL_INFO_SINGULAR;
      const df ip = df_rcp((fabsf(piv.hi) > 0.f) ? piv : make_df(1e-30f, 0.f));
      df tmp[NT];
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int e = u + t * nl;
        df v = df_zero();
        if (e < C::BB) {
          const int i = e / B, jj = e % B;
          const df mij = f2df(M[e]), miq = f2df(M[i * B + q]), mqj = f2df(M[q * B + jj]);
          if (i == q && jj == q)
            v = ip;
          else if (i == q)
            v = df_mul(mqj, ip);
          else if (jj == q)
            v = df_neg(df_mul(miq, ip));
          else
            v = df_sub_two_prods(mij, df_mul(miq, ip), mqj, df_zero(), df_zero());
        }
        tmp[t] = v;
      }
      __syncwarp();
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int e = u + t * nl;
        if (e < C::BB) M[e] = df2f(tmp[t]);
      }
      __syncwarp();
    }
  }
  // y = f - A x (sub) or y = A x, entry u (< b) by one lane
  static __device__ __forceinline__ void matvec(const float2* Am, const float2* xv, const float2* fv, float2* y,
                                                bool sub, int u) {
    df a = df_zero();
    if (u < B) {
      a = sub ? f2df(fv[u]) : df_zero();
#pragma unroll
      for (int q = 0; q < B; q += 2) {
        const df a0 = f2df(Am[u * B + q]), x0 = f2df(xv[q]);
        const df a1 = (q + 1 < B) ? f2df(Am[u * B + q + 1]) : df_zero();
        const df x1 = (q + 1 < B) ? f2df(xv[q + 1]) : df_zero();
        a = sub ? df_sub_two_prods(a, a0, x0, a1, x1) : df_sub_two_prods(a, df_neg(a0), x0, df_neg(a1), x1);
      }
    }
    __syncwarp();
    if (u < B) y[u] = df2f(a);
    __syncwarp();
  }
  // the system whose block rows are base .. base + 2r - 1 of the warp; u = lane - base
  static __device__ void solve(RedWarp<B>& R, int base, int r, int u, int& flag) {
    const int nb = 2 * r, nl = 2 * r;
    for (int q = 0; q < nb; ++q) {
      const int w = base + q;
      if (q > 0) {
        matmul(R.T[w][0], R.T[w - 1][1], R.T[w][0], false, u, nl);  // L_q = T_q,q-1 D_{q-1}^-1
        matmul(R.T[w][0], R.T[w - 1][2], R.T[w][1], true, u, nl);   // D_q -= L_q T_q-1,q
      }
      invert(R.T[w][1], u, nl, flag);
    }
    // y_0 = f_0, y_q = f_q - L_q y_{q-1} (into xs)
    if (u < B) R.xs[base][u] = R.f[base][u];
    __syncwarp();
    for (int q = 1; q < nb; ++q) matvec(R.T[base + q][0], R.xs[base + q - 1], R.f[base + q], R.xs[base + q], true, u);
    // x_q = D_q^-1 (y_q - T_q,q+1 x_{q+1}), the bracket staged in f
    for (int q = nb - 1; q >= 0; --q) {
      const int w = base + q;
      if (q < nb - 1) {
        matvec(R.T[w][2], R.xs[w + 1], R.xs[w], R.f[w], true, u);
      } else {
        if (u < B) R.f[w][u] = R.xs[w][u];
        __syncwarp();
      }
      matvec(R.T[w][1], R.f[w], nullptr, R.xs[w], false, u);
    }
  }
};

// ------------------------------------------------------------------ the kernel
template <int B>
__global__ void __launch_bounds__(kPairThreads, PC<B>::MINB) paqif_pair_kernel(PairArgs a) {
  using C = PC<B>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sd = lane & 1;
  const int gblk = blockIdx.x * kPairBlocksPerCta + (threadIdx.x >> 1);
  const int sys = gblk / a.r, m = gblk - sys * a.r;
  const bool real = sys < a.n_sys;
  const int dsys = real ? sys : a.n_sys - 1;
  if (a.r == 1 && __all_sync(0xffffffffu, !real)) return;  // no shared steps with one block per system

  PairBlk p;
  const int row0 = m * a.np;
  p.nb = min(max(a.n - row0, 0), a.np);
  p.s = a.s;
  p.side = sd;
  p.band = a.band + ((size_t)dsys * a.n + row0) * C::BW;
  p.rhs = a.rhs + (size_t)dsys * a.n + row0;
  p.act = a.act ? a.act + (size_t)dsys * a.n + row0 : nullptr;
  p.x = a.x + (size_t)dsys * a.n + row0;
  p.band_end = a.band + (size_t)a.n_sys * a.n * C::BW;
  p.stk = a.stack + (size_t)((blockIdx.x * kPairThreads + threadIdx.x) >> 5) * a.sf * C::NQ * 32 + lane;
  const int s = a.s, sf = a.sf;
  int flag = 0;

  // ---- the window of level 0: rows and columns at streams 0..b of both sides
  df Ro[C::W][C::W], Rx[C::W][C::W], Rr[C::W];
  double Fu[C::W][B];
#pragma unroll
  for (int j = 0; j < C::W; ++j) {
    const int i = row_of(sd, j, s);
    const bool exists = j < s;
#pragma unroll
    for (int d = 0; d < C::W; ++d) {
      Ro[j][d] = exists ? block_entry(p, B, i, row_of(sd, d, s)) : df_zero();
      Rx[j][d] = exists ? block_entry(p, B, i, row_of(1 - sd, d, s)) : df_zero();
    }
    const bool rr = exists && i < p.nb && !(p.act && __ldg(p.act + i));
    Rr[j] = rr ? df_from_double(__ldg(p.rhs + i)) : df_zero();
#pragma unroll
    for (int q = 0; q < B; ++q) {
      // future own-side column stream b + 1 + q (only q < j is within the band of the row)
      double v = 0.0;
      if (q < j && exists) {
        const int c = row_of(sd, B + 1 + q, s);
        if (i >= 0 && i < p.nb && !(p.act && __ldg(p.act + i)) && c >= 0 && c < p.nb)
          v = __ldg(p.band + (size_t)i * C::BW + (B + c - i));
      }
      Fu[j][q] = v;
    }
  }

  // the rows entering at levels 0 and 1 (streams b+1, b+2) are copied ahead; at the end of level k
  // the row of stream k+1+b is placed and the copy of stream k+3+b takes its slot
  unsigned char* wsm = smem_raw + (size_t)warp * WarpSm<B>::BYTES;
  unsigned char* ring = wsm + (size_t)lane * kRingLane;
  RowMeta<B> meta0 = fetch_row<B>(p, B + 1, ring);
  RowMeta<B> meta1 = fetch_row<B>(p, B + 2, ring + C::SLOT);

  // ---- factorization: levels 0 .. sf-1
  for (int k = 0; k < sf; ++k) {
    // the partner's pivot row in this lane's orientation: its (other, d) is our (own, d)
    df Zo[C::W], Zx[C::W];
#pragma unroll
    for (int d = 0; d < C::W; ++d) {
      Zo[d] = shfl_x1(Rx[0][d]);
      Zx[d] = shfl_x1(Ro[0][d]);
    }
    const df Zr = shfl_x1(Rr[0]);
    // Pi in (left, right) orientation, identical on both lanes
    const df pa = sel(sd, Zx[0], Ro[0][0]);  // left row, left column
    const df pb = sel(sd, Zo[0], Rx[0][0]);  // left row, right column
    const df pc = sel(sd, Rx[0][0], Zo[0]);  // right row, left column
    const df pd = sel(sd, Ro[0][0], Zx[0]);  // right row, right column
    df det = df_det2(pa, pd, pb, pc);
    const float scale = fabsf(pa.hi * pd.hi) + fabsf(pb.hi * pc.hi);
    const bool weak = !(fabsf(det.hi) > 1e-13f * scale) || !(scale > 0.f);
    flag = (weak && flag == 0) ? EHL_INFO_SINGULAR : flag;
    det = (fabsf(det.hi) > 0.f) ? det : make_df(1e-30f, 0.f);
    const df inv = df_rcp(det);
    const df I00 = df_mul(pd, inv), I01 = df_neg(df_mul(pb, inv));
    const df I10 = df_neg(df_mul(pc, inv)), I11 = df_mul(pa, inv);
    // Pi^-1 in this lane's (own row / own column first) orientation
    const df ioo = sel(sd, I11, I00), iox = sel(sd, I10, I01);
    const df ixo = sel(sd, I01, I10), ixx = sel(sd, I00, I11);
    // the folded pivot row of this side: row "own" of Pi^-1 [z_own; z_other] on the outer columns
    {
      float4* st = p.stk + (size_t)k * C::NQ * 32;
      const df nio = df_neg(ioo), nix = df_neg(iox);
      df M[C::NS + 1];
#pragma unroll
      for (int d = 1; d <= B; ++d) {
        M[d - 1] = df_sub_two_prods(df_zero(), nio, Ro[0][d], nix, Zo[d]);
        M[B + d - 1] = df_sub_two_prods(df_zero(), nio, Rx[0][d], nix, Zx[d]);
      }
      M[2 * B] = df_sub_two_prods(df_zero(), nio, Rr[0], nix, Zr);
      M[C::NS] = df_zero();
#pragma unroll
      for (int q = 0; q < C::NQ; ++q)
        st[q * 32] = make_float4(M[2 * q].hi, M[2 * q].lo, M[2 * q + 1].hi, M[2 * q + 1].lo);
    }
    // outer rows: multipliers, then the rank-2 update column by column; the result moves one slot
    // up and left, onto entries whose column was consumed before (the pivot row included)
    df wo[C::W], wx[C::W];
#pragma unroll
    for (int j = 1; j < C::W; ++j) {
      const df lo = Ro[j][0], lx = Rx[j][0];
      wo[j] = df_sub_two_prods(df_zero(), df_neg(lo), ioo, df_neg(lx), ixo);
      wx[j] = df_sub_two_prods(df_zero(), df_neg(lo), iox, df_neg(lx), ixx);
    }
#pragma unroll
    for (int d = 1; d < C::W; ++d) {
#pragma unroll
      for (int j = 1; j < C::W; ++j) Ro[j - 1][d - 1] = df_sub_two_prods(Ro[j][d], wo[j], Ro[0][d], wx[j], Zo[d]);
#pragma unroll
      for (int j = 1; j < C::W; ++j) Rx[j - 1][d - 1] = df_sub_two_prods(Rx[j][d], wo[j], Rx[0][d], wx[j], Zx[d]);
    }
    const df Pr = Rr[0];
#pragma unroll
    for (int j = 1; j < C::W; ++j) {
      Rr[j - 1] = df_sub_two_prods(Rr[j], wo[j], Pr, wx[j], Zr);
      // the column entering at slot b: own side from the row's next band entry, other side 0
      Ro[j - 1][B] = df_from_double_sel(Fu[j][0]);
      Rx[j - 1][B] = df_zero();
#pragma unroll
      for (int q = 0; q + 1 < B; ++q) Fu[j - 1][q] = Fu[j][q + 1];
      Fu[j - 1][B - 1] = 0.0;
    }
    // the row entering at slot b: stream k + 1 + b, in ring slot k & 1
    cp_wait1();
    unsigned char* slot = ring + ((k & 1) ? C::SLOT : 0);
    place_row<B>(p, (k & 1) ? meta1 : meta0, slot, Ro[B], Rr[B], Fu[B]);
#pragma unroll
    for (int d = 0; d < C::W; ++d) Rx[B][d] = df_zero();
    if (k & 1)
      meta1 = fetch_row<B>(p, k + 3 + B, slot);
    else
      meta0 = fetch_row<B>(p, k + 3 + B, slot);
  }
  cp_wait0();  // the copies issued past the last level (zero-size reads) are retired

  // ---- the reduced system (r > 1): the window holds streams s-b .. s (slot b is past the block)
  df xo[B], xx[B];  // solved unknowns of streams k+1 .. k+b of this side / the other side
#pragma unroll
  for (int d = 0; d < B; ++d) {
    xo[d] = df_zero();
    xx[d] = df_zero();
  }
  if (a.r > 1) {
    RedWarp<B>& R = *reinterpret_cast<RedWarp<B>*>(wsm + 32 * kRingLane);
    const int q = lane;  // block row of the warp: 2m (left lane) or 2m + 1 (right lane)
    // rows j = 0..b-1 of the window: left: local row b-1-j (index b-1-j of row 2m), right: local
    // row 2s-b+j (index j of row 2m+1); own column slot d: left index b-1-d of column block 2m,
    // right index d of 2m+1; other-side slots map the other way
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const int ri = sd ? j : B - 1 - j;
#pragma unroll
      for (int d = 0; d < B; ++d) {
        const int co = sd ? d : B - 1 - d;  // own-side column index
        const int cx = sd ? B - 1 - d : d;  // other-side column index
        R.T[q][1][ri * B + co] = df2f(Ro[j][d]);
        R.T[q][sd ? 0 : 2][ri * B + cx] = df2f(Rx[j][d]);
      }
      R.f[q][ri] = df2f(Rr[j]);
    }
    // band entries coupling the block to its neighbours: left lane, its first b rows to the last
    // b columns of block m-1 (sub-diagonal block of row 2m); right lane, its last b rows to the
    // first b columns of block m+1 (super-diagonal block of row 2m+1)
#pragma unroll
    for (int e = 0; e < C::BB; ++e) {
      const int i = e / B, jj = e % B;
      df v = df_zero();
      if (sd == 0) {
        const int lr = i;  // local row i, column row0 - b + jj: band offset jj - i
        if (m > 0 && jj >= i && lr < p.nb && !(p.act && __ldg(p.act + lr)))
          v = df_from_double(__ldg(p.band + (size_t)lr * C::BW + (jj - i)));
      } else {
        const int lr = 2 * s - B + i;  // column row0 + 2s + jj: band offset 2b - i + jj
        if (m < a.r - 1 && jj <= i && lr < p.nb && row0 + 2 * s + jj < a.n && !(p.act && __ldg(p.act + lr)))
          v = df_from_double(__ldg(p.band + (size_t)lr * C::BW + (2 * B - i + jj)));
      }
      R.T[q][sd ? 2 : 0][e] = df2f(v);
    }
    __syncwarp();
    const int u = lane % (2 * a.r), base = lane - u;
    Red<B>::solve(R, base, a.r, u, flag);
    // the solved outer unknowns; the Z0 sweep starts at level sf-1 = s-b-1 with streams s-b..s-1
    // (slot d-1 of xo: stream s-b-1+d; left: local row b-d = index b-d of row 2m; right: local
    // row 2s-b-1+d = index d-1 of row 2m+1)
#pragma unroll
    for (int d = 1; d <= B; ++d) {
      xo[d - 1] = f2df(R.xs[q][sd ? d - 1 : B - d]);
      xx[d - 1] = f2df(R.xs[q ^ 1][sd ? B - d : d - 1]);
    }
    // this lane writes its own outer unknowns
#pragma unroll
    for (int d = 1; d <= B; ++d) {
      const int lr = sd ? 2 * s - B - 1 + d : B - d;
      const df xv = xo[d - 1];
      if (!isfinite(xv.hi) && flag == 0) flag = EHL_INFO_NONFINITE;
      const double dv = (a.mode == 1 && !(xv.hi > 0.f)) ? 0.0 : df_to_double(xv);
      if (real && lr < p.nb) p.x[lr] = dv;
    }
    __syncwarp();
  }

  // ---- Z0 sweep: levels sf-1 .. 0, from the block's ends towards its middle.  The stack levels
  // are copied DEPTH - 1 levels ahead with cp.async into this lane's ring in the warp's
  // shared memory (free now: the rows are placed and the reduced system is solved); a slot is
  // refilled one level after it was read
  __syncwarp();
  {
    float4* zr = reinterpret_cast<float4*>(wsm + (size_t)lane * WarpSm<B>::Z0LANE);
    const float4* st = p.stk;
    auto issue = [&](int k, int slot) {
      if (k >= 0) {
#pragma unroll
        for (int q = 0; q < C::NQ; ++q) cp_async16(zr + slot * C::NQ + q, st + ((size_t)k * C::NQ + q) * 32, 16);
      }
      cp_commit();
    };
#pragma unroll
    for (int u = 0; u < WarpSm<B>::DEPTH - 1; ++u) issue(sf - 1 - u, u);
    for (int k = sf - 1; k >= 0; --k) {
      const int v = sf - 1 - k, slot = v % WarpSm<B>::DEPTH;
      // level k is group v; groups up to v + WarpSm<B>::DEPTH - 2 are committed
      asm volatile("cp.async.wait_group %0;\n" ::"n"(WarpSm<B>::DEPTH - 2) : "memory");
      df M[2 * C::NQ];
#pragma unroll
      for (int q = 0; q < C::NQ; ++q) {
        const float4 w = zr[slot * C::NQ + q];
        M[2 * q] = make_df(w.x, w.y);
        M[2 * q + 1] = make_df(w.z, w.w);
      }
      // the slot read at the previous level takes level k - (WarpSm<B>::DEPTH - 1)
      issue(k - (WarpSm<B>::DEPTH - 1), (v + WarpSm<B>::DEPTH - 1) % WarpSm<B>::DEPTH);
      // the terms of the farther unknowns first: only the last one waits for the level before
      df acc = M[2 * B];
#pragma unroll
      for (int d = B; d >= 1; --d) acc = df_sub_two_prods(acc, M[d - 1], xo[d - 1], M[B + d - 1], xx[d - 1]);
      const df xp = shfl_x1(acc);
#pragma unroll
      for (int d = B - 1; d >= 1; --d) {
        xo[d] = xo[d - 1];
        xx[d] = xx[d - 1];
      }
      xo[0] = acc;
      xx[0] = xp;
      const int lr = row_of(sd, k, s);
      if (!isfinite(acc.hi) && flag == 0) flag = EHL_INFO_NONFINITE;
      const double dv = (a.mode == 1 && !(acc.hi > 0.f)) ? 0.0 : df_to_double(acc);
      if (real && lr < p.nb) p.x[lr] = dv;
    }
    cp_wait0();
  }

  // ---- status: the first nonzero flag among the system's lanes
  const int u = lane % (2 * a.r), base = lane - u;
  int f = 0;
  for (int i = 0; i < 2 * a.r; ++i) {
    const int o = __shfl_sync(0xffffffffu, flag, base + i);
    if (f == 0) f = o;
  }
  if (real && u == 0) {
    if (a.iters) a.iters[dsys] = 1;
    if (a.info) a.info[dsys] = f;
  }
}

template <int B>
size_t pair_smem_bytes(int) {
  return (size_t)WarpSm<B>::BYTES * (kPairThreads / 32);
}

template <int B>
cudaError_t pair_attrs() {
  static std::atomic<unsigned long long> set{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (set.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(paqif_pair_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)pair_smem_bytes<B>(2));
  if (e == cudaSuccess && bit) set.fetch_or(bit, std::memory_order_release);
  return e;
}

}  // namespace

// Geometry of r blocks per system: blocks of even order 2 ceil(n / 2r); with r > 1 each block
// has an interior level (2s >= 2b + 2) and at least one real row, and r divides the 16 blocks
// of a warp (the reduced system stays inside one warp).
static bool pair_geom(int n, int beta, int r, int& s, int& sf) {
  if (r != 1 && r != 2 && r != 4 && r != 8 && r != 16) return false;
  s = (n + 2 * r - 1) / (2 * r);
  if (r > 1 && (2 * s < 2 * beta + 2 || (r - 1) * 2 * s >= n)) return false;
  sf = (r > 1) ? s - beta : s;
  return true;
}

static int pair_min_ctas(int beta) {
  switch (beta) {
    case 1:
      return PC<1>::MINB;
    case 2:
      return PC<2>::MINB;
    case 3:
      return PC<3>::MINB;
    case 4:
      return PC<4>::MINB;
    default:
      return 0;
  }
}

// The block count: among the r whose blocks fit in one round of the resident lane pairs (a
// second, partial round would double the time of the chain; r = 1 always qualifies), the one
// with the shortest chain: its sf elimination levels plus the 2r block steps of the reduced
// system, about b levels each (the system's lanes eliminate it one block row after another).
// Measured for 4096 systems of n = 1024, b = 4 (CUDA events): 2.53, 1.25, 0.55, 0.72 ms for
// r = 1, 2, 4, 8 (the rule takes 4); one system of n = 127, b = 2: 42 us at r = 16, 39 us at the
// rule's r = 4 (ncu launch times): a lone system's time is the latency of each step, not the
// choice of r.
int paqif_pair_parts(int n_sys, int n, int beta, int mode, bool f32, bool factor_store) {
  if (beta < 1 || beta > 4 || mode == 2 || f32 || factor_store || n_sys < 1 || n < 1) return 0;
  const long long resident = (long long)kSmCount * pair_min_ctas(beta) * kPairBlocksPerCta;
  int best = 0;
  long long best_cost = 0;
  for (int r = 1; r <= 16; r *= 2) {
    int s, sf;
    if (!pair_geom(n, beta, r, s, sf)) continue;
    if (r > 1 && (long long)n_sys * r > resident) continue;
    const long long cost = sf + (r > 1 ? 2LL * r * beta : 0);
    if (best == 0 || cost < best_cost) {
      best = r;
      best_cost = cost;
    }
  }
  return best;
}

size_t paqif_pair_stack_bytes(int n_sys, int n, int beta, int r) {
  int s, sf;
  if (beta < 1 || beta > 4 || !pair_geom(n, beta, r, s, sf)) return 0;
  const size_t grid = ((size_t)n_sys * r + kPairBlocksPerCta - 1) / kPairBlocksPerCta;
  const size_t nq = (size_t)(2 * beta + 2) / 2;
  return grid * kPairBlocksPerCta * (size_t)sf * 2 * nq * sizeof(float4);
}

template <int B>
static cudaError_t launch_pair(const PaqifLaunch& L, int r, cudaStream_t st) {
  int s, sf;
  if (!pair_geom(L.n, B, r, s, sf)) return cudaErrorInvalidValue;
  PairArgs a;
  a.n_sys = L.n_sys;
  a.n = L.n;
  a.mode = L.mode;
  a.r = r;
  a.np = 2 * s;
  a.s = s;
  a.sf = sf;
  a.band = L.band;
  a.rhs = L.rhs;
  a.act = L.act;
  a.stack = reinterpret_cast<float4*>(L.stack);
  a.x = L.x;
  a.iters = L.iters;
  a.info = L.info;
  cudaError_t e = pair_attrs<B>();
  if (e != cudaSuccess) return e;
  const int grid = (int)(((long long)L.n_sys * r + kPairBlocksPerCta - 1) / kPairBlocksPerCta);
  paqif_pair_kernel<B><<<grid, kPairThreads, pair_smem_bytes<B>(r), st>>>(a);
  note_launch();
  return cudaGetLastError();
}

cudaError_t paqif_pair_prepare(int beta) {
  switch (beta) {
    case 1:
      return pair_attrs<1>();
    case 2:
      return pair_attrs<2>();
    case 3:
      return pair_attrs<3>();
    case 4:
      return pair_attrs<4>();
    default:
      return cudaSuccess;
  }
}

cudaError_t launch_paqif_pair(const PaqifLaunch& L, int r, cudaStream_t st) {
  if (L.mode == 2 || L.f32 || (reinterpret_cast<uintptr_t>(L.band) & 15u) != 0) return cudaErrorInvalidValue;
  switch (L.beta) {
    case 1:
      return launch_pair<1>(L, r, st);
    case 2:
      return launch_pair<2>(L, r, st);
    case 3:
      return launch_pair<3>(L, r, st);
    case 4:
      return launch_pair<4>(L, r, st);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace ehl
