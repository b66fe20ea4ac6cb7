// nb_sym.cu -- symmetric (half-pair) force kernel: each unordered pair of ions
// is evaluated once and its force is applied to both ions with opposite
// signs (Newton's third law), halving the pair arithmetic of the FP64-pipe
// bound precisions (fp64, df64).
//
// The split and literal mixed precisions use it too (FP32 pair arithmetic
// with per-step FP32 partials added into FP64, or into double-float sums on
// the FP32 pipe for split).  In the split path's large blocks (G >= 16) a
// lane holds four P-ions, whose arithmetic runs as two packed pairs of FP32
// (.f32x2) instructions: sym_offdiag_split4.
//
// Ions are grouped in blocks of BI = 32 G ions (G tiles of one warp).  One
// CTA handles one work item, a block pair (P, Q) with P <= Q, drawn from the
// round-robin schedule of nb_symsched.cuh:
//  - P < Q: both blocks' positions are staged in shared memory together with
//    accumulators for P and Q.  Each warp takes Q-tiles; for a Q-tile it
//    visits the P-tiles in the staggered order pt = (qs + k) mod G, one
//    per __syncthreads-separated step k, so at any step the warps hold
//    distinct P-tiles.  Within a step lane l holds P-ion l; the Q-tile's
//    positions and its force accumulators rotate one lane per iteration
//    (warp shuffles), so after 32 iterations every (P-ion, Q-ion) pair of
//    the two tiles has been evaluated once and the Q data is back home.
//  - P == Q: the block's internal pairs, one-sided (each ion against all
//    others of the block).
// Output: the item adds its sums into acc[c * n + i] in round order
// (nb_symsched.cuh), so the result is bitwise reproducible with no partial
// buffer and no atomics on the data.
//
// With per-ion charges the two sides carry different weights: ion i gets
// q_j d/r^3 and ion j gets -q_i d/r^3 (the sums exclude the ion's own
// charge, as in the one-sided kernel).  The ragged last block is padded with
// weight-0 ions far away; only items that touch it apply the weights when
// the charge is uniform.
#include <algorithm>
#include <mutex>

#include "nb_common.cuh"
#include "nb_symsched.cuh"

namespace nb {

// Threads per item: one warp per 32-ion tile for 32- and 64-ion blocks
// (G <= 2, the small n where items are few); 128 (4 warps) for 128-ion
// blocks (G = 4); 256 (8 warps) above, and 512 for the split kernel's
// 1024-ion blocks.  The staggered schedule needs at least as many P-tiles
// as warps.
constexpr int SYM_THREADS = 256;
constexpr int SYM_THREADS_SMALL = 128;
constexpr double SYM_FAR = 1e18;

struct __align__(16) SD4 {
  double x, y, z, w;
};

__device__ __forceinline__ double shfl_next(double v, int lane) {
  return __shfl_sync(0xffffffffu, v, (lane + 1) & 31);
}
__device__ __forceinline__ float shfl_next(float v, int lane) {
  return __shfl_sync(0xffffffffu, v, (lane + 1) & 31);
}

// One 32x32 tile step for the FP64 pair arithmetic.  pp: this lane's P-ion;
// qd: the Q-ion currently held (rotating); b: its accumulators
// (rotating); a: the P-ion's accumulators.
template <bool W, int CNT = 32>
__device__ __forceinline__ void sym_step_fp64(const SD4 &pp, SD4 qd, double soft2, int lane,
                                              double a[3], double b[3]) {
#pragma unroll 2
  for (int r = 0; r < CNT; ++r) {
    const double dx = pp.x - qd.x, dy = pp.y - qd.y, dz = pp.z - qd.z;
    const double s = rinv3_fp64(dx, dy, dz, soft2);
    const double sp = W ? s * qd.w : s;
    const double sq = W ? s * pp.w : s;
    a[0] = fma(dx, sp, a[0]);
    a[1] = fma(dy, sp, a[1]);
    a[2] = fma(dz, sp, a[2]);
    b[0] = fma(-dx, sq, b[0]);
    b[1] = fma(-dy, sq, b[1]);
    b[2] = fma(-dz, sq, b[2]);
    qd.x = shfl_next(qd.x, lane);
    qd.y = shfl_next(qd.y, lane);
    qd.z = shfl_next(qd.z, lane);
    if (W) qd.w = shfl_next(qd.w, lane);
    b[0] = shfl_next(b[0], lane);
    b[1] = shfl_next(b[1], lane);
    b[2] = shfl_next(b[2], lane);
  }
}

// The same step with double-float pair arithmetic (see pair_df64).  The
// weights w (charge, or 1 / 0 for real / padding ions) are FP64; a, b are
// double-float (h, l) accumulators for this step.
template <bool W, int CNT = 32>
__device__ __forceinline__ void sym_step_df64(const SD4 &pp, SD4 qd, float s2h, float s2l, int lane,
                                              float ah[3], float al[3], float bh[3], float bl[3]) {
  float wph = 1.0f, wpl = 0.0f;
  if (W) split_f64(pp.w, wph, wpl);
#pragma unroll 1
  for (int r = 0; r < CNT; ++r) {
    float dh[3], dl[3];
    split_f64(pp.x - qd.x, dh[0], dl[0]);
    split_f64(pp.y - qd.y, dh[1], dl[1]);
    split_f64(pp.z - qd.z, dh[2], dl[2]);
    float sh, sl;
    df_rinv3(dh, dl, s2h, s2l, sh, sl);
    // weights: P-side times w_q, Q-side times w_p (double-float products)
    float sph = sh, spl = sl, sqh = sh, sql = sl;
    if (W) {
      float wqh, wql;
      split_f64(qd.w, wqh, wql);
      sph = sh * wqh;
      spl = fmaf(sh, wql, fmaf(sl, wqh, fmaf(sh, wqh, -sph)));
      sqh = sh * wph;
      sql = fmaf(sh, wpl, fmaf(sl, wph, fmaf(sh, wph, -sqh)));
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float ph = dh[k] * sph;
      float pl = fmaf(dh[k], spl, fmaf(dl[k], sph, fmaf(dh[k], sph, -ph)));
      float s, t;
      two_sum_f(ah[k], ph, s, t);
      ah[k] = s;
      al[k] += t + pl;
      if (W) {
        ph = dh[k] * sqh;
        pl = fmaf(dh[k], sql, fmaf(dl[k], sqh, fmaf(dh[k], sqh, -ph)));
      }
      two_sum_f(bh[k], -ph, s, t);
      bh[k] = s;
      bl[k] += t - pl;
    }
    qd.x = shfl_next(qd.x, lane);
    qd.y = shfl_next(qd.y, lane);
    qd.z = shfl_next(qd.z, lane);
    if (W) qd.w = shfl_next(qd.w, lane);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      bh[k] = shfl_next(bh[k], lane);
      bl[k] = shfl_next(bl[k], lane);
    }
  }
}

// FP32 weight kept in the low word of a staged entry's w (mixed modes).
__device__ __forceinline__ float wf32(double w) { return __int_as_float(__double2loint(w)); }
__device__ __forceinline__ double wpack(float w) { return __hiloint2double(0, __float_as_int(w)); }

// Literal mixed step: FP64 displacement, FP32 bulk, FP32 partials for this
// step (a: the P-ion, b: the rotating Q-ion).
template <bool W, int CNT = 32>
__device__ __forceinline__ void sym_step_mixed(const SD4 &pp, SD4 qd, float soft2f, int lane,
                                               float a[3], float b[3]) {
  const float wp = wf32(pp.w);
  float wq = wf32(qd.w);
#pragma unroll 2
  for (int r = 0; r < CNT; ++r) {
    const float fx = f64_to_f32_rn(pp.x - qd.x);
    const float fy = f64_to_f32_rn(pp.y - qd.y);
    const float fz = f64_to_f32_rn(pp.z - qd.z);
    const float s = f32_rinv3(fx, fy, fz, soft2f);
    const float sp = W ? s * wq : s, sq = W ? s * wp : s;
    a[0] = fmaf(fx, sp, a[0]);
    a[1] = fmaf(fy, sp, a[1]);
    a[2] = fmaf(fz, sp, a[2]);
    b[0] = fmaf(-fx, sq, b[0]);
    b[1] = fmaf(-fy, sq, b[1]);
    b[2] = fmaf(-fz, sq, b[2]);
    qd.x = shfl_next(qd.x, lane);
    qd.y = shfl_next(qd.y, lane);
    qd.z = shfl_next(qd.z, lane);
    if (W) wq = shfl_next(wq, lane);
    b[0] = shfl_next(b[0], lane);
    b[1] = shfl_next(b[1], lane);
    b[2] = shfl_next(b[2], lane);
  }
}

// One split-precision pair evaluation: P-ion (ph, pl) against Q-ion (qh, ql),
// positions as FP32 (hi, lo) pairs with the weight in hi.w; the force goes
// into a (P side) and, with the opposite sign, into b (Q side).
template <bool W, bool SEED>
__device__ __forceinline__ void split_eval(const float4 &ph, const float4 &pl, const float4 &qh,
                                           const float4 &ql, float soft2f, float a[3], float b[3]) {
  const float fx = (ph.x - qh.x) + (pl.x - ql.x);
  const float fy = (ph.y - qh.y) + (pl.y - ql.y);
  const float fz = (ph.z - qh.z) + (pl.z - ql.z);
  const float s = f32_rinv3<SEED>(fx, fy, fz, soft2f);
  const float sp = W ? s * qh.w : s, sq = W ? s * ph.w : s;
  a[0] = fmaf(fx, sp, a[0]);
  a[1] = fmaf(fy, sp, a[1]);
  a[2] = fmaf(fz, sp, a[2]);
  b[0] = fmaf(-fx, sq, b[0]);
  b[1] = fmaf(-fy, sq, b[1]);
  b[2] = fmaf(-fz, sq, b[2]);
}

// Split mixed step: the Q-tile's positions are read from shared memory at
// the rotated index (lane + r) mod 32 (two conflict-free 128-bit loads per
// pair); only the Q accumulators rotate through shuffles.  qhi, qlo point at
// this lane's entry of the duplicated tile, so entry r of the rotation is
// qhi[r] (a compile-time offset once the loop is unrolled).
template <bool W, bool SEED, int CNT = 32>
__device__ __forceinline__ void sym_step_split(const float4 &ph, const float4 &pl, const float4 *qhi,
                                               const float4 *qlo, float soft2f, int lane, float a[3],
                                               float b[3]) {
#pragma unroll
  for (int r = 0; r < CNT; ++r) {
    split_eval<W, SEED>(ph, pl, qhi[r], qlo[r], soft2f, a, b);
    b[0] = shfl_next(b[0], lane);
    b[1] = shfl_next(b[1], lane);
    b[2] = shfl_next(b[2], lane);
  }
}

// Where an item keeps the finished sums of its Q block (and a diagonal item
// its block's sums): in the Q-tile's own 1 KB of staged positions, which only
// the warp that owns that Q-tile reads, so it is free once that warp is done
// with the tile.  Sum c of ion i of the block: [i / 32][c][i mod 32].
__device__ __forceinline__ double &qsum(SD4 *posQ, int c, int i) {
  return reinterpret_cast<double *>(posQ)[(i >> 5) * 128 + c * 32 + (i & 31)];
}

// Double-float accumulation on the FP32 pipe: (h, l) += v (TwoSum), for the
// split path's per-step FP32 partials, so that its pair loop and tile
// flushes issue no FP64 instruction.
__device__ __forceinline__ void df_add(float &h, float &l, float v) {
  float s, e;
  two_sum_f(h, v, s, e);
  h = s;
  l += e;
}

// Packed FP32 pairs (.f32x2): one instruction applies the same IEEE
// operation, rounded to nearest, to both halves.  It takes one issue slot and
// two cycles of the FMA pipe, so an issue-bound loop gains where its FMA pipe
// has room; a pair {x, x} built from one register feeds it without an
// instruction of its own.
typedef unsigned long long f2;
__device__ __forceinline__ f2 f2_pack(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_split(f2 v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// The four P-ions of a lane as two packed pairs (ions 0-1 and 2-3), staged
// in shared memory already paired: for P-tile t, pair v and lane, four
// float4 at ((t 2 + v) 4 + k) 32 + lane, k = 0..3, holding (hx, hy), (hz, lx),
// (ly, lz) and (w, 0) with each coordinate as the pair (ion 2v, ion 2v+1).
// Loading a pair from one 128-bit entry gives it an aligned register pair;
// pairs assembled from separate loads were re-assembled inside the pair loop
// by the compiler (about 20 register moves per 128 evaluations).
__device__ __forceinline__ void sym_stage_p4(float4 *f, int t, int BI, int64_t p0, int64_t n, const double *q,
                                             const PosF32 &pf, bool qarr) {
  const int pt = t >> 6, v = (t >> 5) & 1, lane = t & 31;
  const int64_t ga = p0 + pt * 128 + 64 * v + lane, gb = ga + 32;  // ions 2v and 2v + 1 of the lane
  const bool ra = ga < n, rb = gb < n;
  const float far = (float)SYM_FAR;
  float4 *e = f + (pt * 2 + v) * 128 + lane;
  e[0] = make_float4(ra ? pf.xh[ga] : far, rb ? pf.xh[gb] : far, ra ? pf.yh[ga] : far, rb ? pf.yh[gb] : far);
  e[32] = make_float4(ra ? pf.zh[ga] : far, rb ? pf.zh[gb] : far, ra ? pf.xl[ga] : 0.0f, rb ? pf.xl[gb] : 0.0f);
  e[64] = make_float4(ra ? pf.yl[ga] : 0.0f, rb ? pf.yl[gb] : 0.0f, ra ? pf.zl[ga] : 0.0f, rb ? pf.zl[gb] : 0.0f);
  e[96] = make_float4(ra ? (qarr ? (float)q[ga] : 1.0f) : 0.0f, rb ? (qarr ? (float)q[gb] : 1.0f) : 0.0f, 0.0f, 0.0f);
}

// sym_step_split4 with the four P-ions' arithmetic in two packed pairs
// (ions 0-1 and 2-3): two independent chains per lane; per ion the same
// operations in the same order as split_eval, and the Q sum takes the ions'
// terms in the order 0, 1, 2, 3.  pe: this lane's first staged entry of the
// P-tile (sym_stage_p4's layout).
template <bool W, bool SEED>
__device__ __forceinline__ void sym_step_split4_packed(const float4 *pe, const float4 *qhi, const float4 *qlo,
                                                       float soft2f, int lane, float a[4][3], float b[3]) {
  f2 phx[2], phy[2], phz[2], plx[2], ply[2], plz[2], pw[2], ax[2], ay[2], az[2];
#pragma unroll
  for (int v = 0; v < 2; ++v) {
    const float4 e0 = pe[v * 128], e1 = pe[v * 128 + 32], e2 = pe[v * 128 + 64];
    phx[v] = f2_pack(e0.x, e0.y);
    phy[v] = f2_pack(e0.z, e0.w);
    phz[v] = f2_pack(e1.x, e1.y);
    plx[v] = f2_pack(e1.z, e1.w);
    ply[v] = f2_pack(e2.x, e2.y);
    plz[v] = f2_pack(e2.z, e2.w);
    if (W) {
      const float4 e3 = pe[v * 128 + 96];
      pw[v] = f2_pack(e3.x, e3.y);
    }
    ax[v] = f2_pack(a[2 * v][0], a[2 * v + 1][0]);
    ay[v] = f2_pack(a[2 * v][1], a[2 * v + 1][1]);
    az[v] = f2_pack(a[2 * v][2], a[2 * v + 1][2]);
  }
  const f2 s2 = f2_pack(soft2f, soft2f), m15 = f2_pack(-1.5f, -1.5f), p15 = f2_pack(1.5f, 1.5f);
#pragma unroll(SEED ? 32 : 16)
  for (int r = 0; r < 32; ++r) {
    const float4 qh = qhi[r], ql = qlo[r];
    const f2 qhx = f2_pack(qh.x, qh.x), qhy = f2_pack(qh.y, qh.y), qhz = f2_pack(qh.z, qh.z);
    const f2 qlx = f2_pack(ql.x, ql.x), qly = f2_pack(ql.y, ql.y), qlz = f2_pack(ql.z, ql.z);
    float dxs[4], dys[4], dzs[4], sqs[4];
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const f2 dx = f2_add(f2_sub(phx[v], qhx), f2_sub(plx[v], qlx));
      const f2 dy = f2_add(f2_sub(phy[v], qhy), f2_sub(ply[v], qly));
      const f2 dz = f2_add(f2_sub(phz[v], qhz), f2_sub(plz[v], qlz));
      const f2 r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_fma(dz, dz, s2)));
      float r2a, r2b, ya, yb;
      f2_split(r2, r2a, r2b);
      asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(ya) : "f"(r2a));
      asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yb) : "f"(r2b));
      const f2 y = f2_pack(fminf(ya, F32_YMAX), fminf(yb, F32_YMAX));
      const f2 y2 = f2_mul(y, y);
      const f2 y3 = f2_mul(y2, y);
      const f2 sv = SEED ? y3 : f2_fma(y3, f2_fma(f2_mul(m15, r2), y2, p15), y3);
      const f2 sp = W ? f2_mul(sv, f2_pack(qh.w, qh.w)) : sv;
      const f2 sq = W ? f2_mul(sv, pw[v]) : sv;
      ax[v] = f2_fma(dx, sp, ax[v]);
      ay[v] = f2_fma(dy, sp, ay[v]);
      az[v] = f2_fma(dz, sp, az[v]);
      f2_split(dx, dxs[2 * v], dxs[2 * v + 1]);
      f2_split(dy, dys[2 * v], dys[2 * v + 1]);
      f2_split(dz, dzs[2 * v], dzs[2 * v + 1]);
      f2_split(sq, sqs[2 * v], sqs[2 * v + 1]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      b[0] = fmaf(-dxs[u], sqs[u], b[0]);
      b[1] = fmaf(-dys[u], sqs[u], b[1]);
      b[2] = fmaf(-dzs[u], sqs[u], b[2]);
    }
    b[0] = shfl_next(b[0], lane);
    b[1] = shfl_next(b[1], lane);
    b[2] = shfl_next(b[2], lane);
  }
#pragma unroll
  for (int v = 0; v < 2; ++v) {
    f2_split(ax[v], a[2 * v][0], a[2 * v + 1][0]);
    f2_split(ay[v], a[2 * v][1], a[2 * v + 1][1]);
    f2_split(az[v], a[2 * v][2], a[2 * v + 1][2]);
  }
}

// Off-diagonal item, split precision with 128-ion P-tiles: GP = G/4 P-tiles
// and NW = 2 GP warps (8 warps for 512-ion blocks, 16 for 1024); posP holds
// the P block in sym_stage_p4's paired layout.  At step k
// warp w holds P-tile (qs + k) mod GP, which it shares with warp w +- GP; the
// two keep their P sums in separate double-float copies (accPf: [2][2][3][BI]
// floats, copy w / GP), added in copy order at the end, so no two warps ever
// update one word.
template <bool W, int NW, bool SEED>
__device__ __forceinline__ void sym_offdiag_split4(const SD4 *posP, SD4 *posQ, float *accPf, int G, int BI,
                                                   double soft2) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int GP = G >> 2;
  float *acc = accPf + (warp / GP) * 6 * BI;
  const float4 *fP = reinterpret_cast<const float4 *>(posP);
  const float4 *fQ = reinterpret_cast<const float4 *>(posQ);
  for (int qs = warp; qs < G; qs += NW) {
    float qh[3] = {0.0f, 0.0f, 0.0f}, ql[3] = {0.0f, 0.0f, 0.0f};
    const float4 *qhi = fQ + qs * 64 + lane, *qlo = fQ + 2 * BI + qs * 64 + lane;
    for (int k = 0; k < GP; ++k) {
      const int pt = (qs + k) % GP;
      __syncthreads();  // all warps are at step k
      float a[4][3], b[3] = {0, 0, 0};
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u][0] = a[u][1] = a[u][2] = 0.0f;
      sym_step_split4_packed<W, SEED>(fP + pt * 256 + lane, qhi, qlo, (float)soft2, lane, a, b);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = pt * 128 + 32 * u + lane;
#pragma unroll
        for (int c = 0; c < 3; ++c) df_add(acc[c * BI + i], acc[(3 + c) * BI + i], a[u][c]);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) df_add(qh[c], ql[c], b[c]);
    }
    __syncwarp();  // every lane is done reading the tile
#pragma unroll
    for (int c = 0; c < 3; ++c) qsum(posQ, c, qs * 32 + lane) = f32_to_f64(qh[c]) + f32_to_f64(ql[c]);
  }
}

// Off-diagonal item in the other layouts.  The P sums go to accP in shared
// memory (FP64, or double-float accPf for split), the Q sums (FP64) to qsum
// once the warp is done with its Q-tile.
template <int MODE, bool W, int NW>
__device__ __forceinline__ void sym_offdiag(const SD4 *posP, SD4 *posQ, double *accP, int G, int BI,
                                            double soft2, float s2h, float s2l) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float *accPf = reinterpret_cast<float *>(accP);
  for (int qs = warp; qs < G; qs += NW) {
    const SD4 qh = posQ[qs * 32 + lane];
    double aq[3] = {0.0, 0.0, 0.0};
    float qfh[3] = {0.0f, 0.0f, 0.0f}, qfl[3] = {0.0f, 0.0f, 0.0f};
    for (int k = 0; k < G; ++k) {
      const int pt = (qs + k) % G;
      __syncthreads();  // all warps are at step k: their P-tiles are distinct
      const SD4 pp = posP[pt * 32 + lane];
      const int ip = pt * 32 + lane;
      if (MODE == MODE_MIXED || split_like(MODE)) {
        float a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
        if (MODE == MODE_MIXED) {
          sym_step_mixed<W>(pp, qh, (float)soft2, lane, a, b);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            accP[c * BI + ip] += f32_to_f64(a[c]);
            aq[c] += f32_to_f64(b[c]);
          }
        } else {
          const float4 *fP = reinterpret_cast<const float4 *>(posP);
          const float4 *fQ = reinterpret_cast<const float4 *>(posQ);
          sym_step_split<W, MODE == MODE_SPLIT_RSQ>(fP[ip], fP[BI + ip], fQ + qs * 64 + lane,
                                                    fQ + 2 * BI + qs * 64 + lane, (float)soft2, lane, a, b);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            df_add(accPf[c * BI + ip], accPf[(3 + c) * BI + ip], a[c]);
            df_add(qfh[c], qfl[c], b[c]);
          }
        }
      } else if (MODE == MODE_DF64) {
        float ah[3] = {0, 0, 0}, al[3] = {0, 0, 0}, bh[3] = {0, 0, 0}, bl[3] = {0, 0, 0};
        sym_step_df64<W>(pp, qh, s2h, s2l, lane, ah, al, bh, bl);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          accP[c * BI + ip] += f32_to_f64(ah[c]) + f32_to_f64(al[c]);
          aq[c] += f32_to_f64(bh[c]) + f32_to_f64(bl[c]);
        }
      } else {
        double a[3] = {0.0, 0.0, 0.0}, b[3] = {0.0, 0.0, 0.0};
        sym_step_fp64<W>(pp, qh, soft2, lane, a, b);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          accP[c * BI + ip] += a[c];
          aq[c] += b[c];
        }
      }
    }
    __syncwarp();  // every lane is done reading the tile
#pragma unroll
    for (int c = 0; c < 3; ++c)
      qsum(posQ, c, qs * 32 + lane) = split_like(MODE) ? f32_to_f64(qfh[c]) + f32_to_f64(qfl[c]) : aq[c];
  }
}

// Staged entry of ion g (or a padding entry when g >= n): FP64 position and
// weight for fp64/df64; FP64 position and FP32 weight (low word of w) for
// mixed; two float4 (hi x, y, z, weight; lo x, y, z) for split.
template <int MODE, bool QARR>
__device__ __forceinline__ void sym_stage(SD4 *dst, int i, int BI, int64_t g, int64_t n, const double *x,
                                          const double *y, const double *z, const double *q,
                                          const PosF32 &pf, bool dup) {
  const bool real = g < n;
  const double w = real ? (QARR ? q[g] : 1.0) : 0.0;
  if (split_like(MODE)) {
    // P side: [BI hi entries][BI lo entries].  Q side (dup): every 32-ion
    // tile stored twice back to back, [2 BI hi][2 BI lo], so that the entry
    // (lane + r) of a rotation is at a fixed offset r from the lane's base.
    float4 *f = reinterpret_cast<float4 *>(dst);
    const float4 hi = real ? make_float4(pf.xh[g], pf.yh[g], pf.zh[g], (float)w)
                           : make_float4((float)SYM_FAR, (float)SYM_FAR, (float)SYM_FAR, 0.0f);
    const float4 lo = real ? make_float4(pf.xl[g], pf.yl[g], pf.zl[g], 0.0f) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (dup) {
      const int k = (i >> 5) * 64 + (i & 31);
      f[k] = hi;
      f[k + 32] = hi;
      f[2 * BI + k] = lo;
      f[2 * BI + k + 32] = lo;
    } else {
      f[i] = hi;
      f[BI + i] = lo;
    }
    return;
  }
  SD4 e;
  if (real) {
    e.x = x[g]; e.y = y[g]; e.z = z[g];
  } else {
    e.x = SYM_FAR; e.y = SYM_FAR; e.z = SYM_FAR;
  }
  e.w = (MODE == MODE_MIXED) ? wpack((float)w) : w;
  dst[i] = e;
}

// Register budgets: fp64 two 256-thread blocks per SM; the split path's
// packed four-ion step with 256 threads three blocks per SM, the number its
// 72 KB of shared memory allows (80 registers, a few bytes of spills outside
// the pair loop: 2.6 % faster at n = 1e5 than two blocks of 102 registers,
// 0.5-1 % slower at n = 16384-40000).
template <int MODE, bool QARR, bool P2, int NT, bool INPLACE>
__global__ void __launch_bounds__(NT, MODE == MODE_FP64 ? 512 / NT : (P2 && NT == 256) ? 3 : 0) k_pair_sym(int64_t n, int nbk, int G,
                                                         const double *__restrict__ x,
                                                         const double *__restrict__ y,
                                                         const double *__restrict__ z,
                                                         const double *__restrict__ q, PosF32 pf,
                                                         double soft2, double *__restrict__ acc,
                                                         int *__restrict__ sync, unsigned *err) {
  constexpr bool inplace = INPLACE;  // the output mode, fixed at compile time
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int BI = 32 * G;
  SD4 *posP = reinterpret_cast<SD4 *>(smem_raw);
  SD4 *posQ = posP + BI;
  double *accP = reinterpret_cast<double *>(posQ + (split_like(MODE) ? 2 * BI : BI));  // [3][BI]
  const SymItem it = sym_block_item(inplace, sync, nbk);
  const int P = it.P, Q = it.Q;
  const int64_t p0 = (int64_t)P * BI, q0 = (int64_t)Q * BI;
  const int np = (int)min((int64_t)BI, n - p0), nq = (int)min((int64_t)BI, n - q0);
  const int tid = threadIdx.x;
  const bool paired = P2 && P != Q;  // off-diagonal four-ion items: P block staged in pairs
  if (paired)
    for (int t = tid; t < BI / 2; t += NT) sym_stage_p4(reinterpret_cast<float4 *>(posP), t, BI, p0, n, q, pf, QARR);
  for (int i = tid; i < BI; i += NT) {
    if (!paired) sym_stage<MODE, QARR>(posP, i, BI, p0 + i, n, x, y, z, q, pf, false);
    if (P != Q) sym_stage<MODE, QARR>(posQ, i, BI, q0 + i, n, x, y, z, q, pf, true);
    accP[i] = 0.0;
    accP[BI + i] = 0.0;
    accP[2 * BI + i] = 0.0;
    if (P2) {  // the second copy of the P sums
      accP[3 * BI + i] = 0.0;
      accP[4 * BI + i] = 0.0;
      accP[5 * BI + i] = 0.0;
    }
  }
  float s2h = 0.0f, s2l = 0.0f;
  if (MODE == MODE_DF64) split_f64(soft2, s2h, s2l);
  __syncthreads();

  if (P == Q) {  // the block's own pairs, one-sided; sums into qsum (posQ is not staged)
    for (int i = tid; i < np; i += NT) {
      const SD4 pi = posP[i];
      double a[3] = {0.0, 0.0, 0.0};
      if (MODE == MODE_MIXED || split_like(MODE)) {
        float af[3] = {0, 0, 0};
        const float4 *f = reinterpret_cast<const float4 *>(posP);
        for (int j = 0; j < np; ++j) {
          float fx, fy, fz, wj;
          if (MODE == MODE_MIXED) {
            const SD4 pj = posP[j];
            fx = f64_to_f32_rn(pi.x - pj.x);
            fy = f64_to_f32_rn(pi.y - pj.y);
            fz = f64_to_f32_rn(pi.z - pj.z);
            wj = wf32(pj.w);
          } else {
            const float4 ih = f[i], il = f[BI + i], jh = f[j], jl = f[BI + j];
            fx = (ih.x - jh.x) + (il.x - jl.x);
            fy = (ih.y - jh.y) + (il.y - jl.y);
            fz = (ih.z - jh.z) + (il.z - jl.z);
            wj = jh.w;
          }
          float sj = f32_rinv3<MODE == MODE_SPLIT_RSQ>(fx, fy, fz, (float)soft2);
          if (QARR) sj *= wj;
          af[0] = fmaf(fx, sj, af[0]);
          af[1] = fmaf(fy, sj, af[1]);
          af[2] = fmaf(fz, sj, af[2]);
          if ((j & 31) == 31) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              a[k] += f32_to_f64(af[k]);
              af[k] = 0.0f;
            }
          }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) a[k] += f32_to_f64(af[k]);
      } else if (MODE == MODE_DF64) {
        float ah[3] = {0, 0, 0}, al[3] = {0, 0, 0};
        for (int j = 0; j < np; ++j) {
          const SD4 pj = posP[j];
          float dh[3], dl[3];
          split_f64(pi.x - pj.x, dh[0], dl[0]);
          split_f64(pi.y - pj.y, dh[1], dl[1]);
          split_f64(pi.z - pj.z, dh[2], dl[2]);
          float sh, sl;
          df_rinv3(dh, dl, s2h, s2l, sh, sl);
          if (QARR) {
            float wh, wl;
            split_f64(pj.w, wh, wl);
            const float ph = sh * wh;
            sl = fmaf(sh, wl, fmaf(sl, wh, fmaf(sh, wh, -ph)));
            sh = ph;
          }
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const float ph = dh[k] * sh;
            const float pl = fmaf(dh[k], sl, fmaf(dl[k], sh, fmaf(dh[k], sh, -ph)));
            float s, tt;
            two_sum_f(ah[k], ph, s, tt);
            ah[k] = s;
            al[k] += tt + pl;
          }
          if ((j & 255) == 255) {  // flush the double-float sum every 256 pairs
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              a[k] += f32_to_f64(ah[k]) + f32_to_f64(al[k]);
              ah[k] = al[k] = 0.0f;
            }
          }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) a[k] += f32_to_f64(ah[k]) + f32_to_f64(al[k]);
      } else {
        for (int j = 0; j < np; ++j) {
          const SD4 pj = posP[j];
          const double dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
          double s = rinv3_fp64(dx, dy, dz, soft2);
          if (QARR) s *= pj.w;
          a[0] = fma(dx, s, a[0]);
          a[1] = fma(dy, s, a[1]);
          a[2] = fma(dz, s, a[2]);
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) qsum(posQ, c, i) = a[c];
    }
    __syncthreads();
    sym_output<NT>(inplace, it, n, p0, np, q0, nq, acc, sync, err, [&](int c, int i) { return qsum(posQ, c, i); },
                   [&](int c, int i) { return 0.0; });
    return;
  }

  const bool weighted = QARR || np < BI || nq < BI;
  float *accPf = reinterpret_cast<float *>(accP);
  if (P2) {
    if (weighted)
      sym_offdiag_split4<true, NT / 32, MODE == MODE_SPLIT_RSQ>(posP, posQ, accPf, G, BI, soft2);
    else
      sym_offdiag_split4<false, NT / 32, MODE == MODE_SPLIT_RSQ>(posP, posQ, accPf, G, BI, soft2);
  } else if (weighted) {
    sym_offdiag<MODE, true, NT / 32>(posP, posQ, accP, G, BI, soft2, s2h, s2l);
  } else {
    sym_offdiag<MODE, false, NT / 32>(posP, posQ, accP, G, BI, soft2, s2h, s2l);
  }
  __syncthreads();
  if (P2)  // two copies of the P sums, added in copy order
    sym_output<NT>(inplace, it, n, p0, np, q0, nq, acc, sync, err,
                   [&](int c, int i) {
                     return ((f32_to_f64(accPf[c * BI + i]) + f32_to_f64(accPf[(3 + c) * BI + i])) +
                             f32_to_f64(accPf[(6 + c) * BI + i])) +
                            f32_to_f64(accPf[(9 + c) * BI + i]);
                   },
                   [&](int c, int i) { return qsum(posQ, c, i); });
  else if (split_like(MODE))
    sym_output<NT>(inplace, it, n, p0, np, q0, nq, acc, sync, err,
                   [&](int c, int i) { return f32_to_f64(accPf[c * BI + i]) + f32_to_f64(accPf[(3 + c) * BI + i]); },
                   [&](int c, int i) { return qsum(posQ, c, i); });
  else
    sym_output<NT>(inplace, it, n, p0, np, q0, nq, acc, sync, err, [&](int c, int i) { return accP[c * BI + i]; },
                   [&](int c, int i) { return qsum(posQ, c, i); });
}

// 32-ion blocks (the mid-range n, where the items are too few to fill the
// GPU with one warp each): RW warps share an item's 32 rotations, warp w
// taking rotations [w C, (w + 1) C), C = 32 / RW, starting from the Q-tile
// turned by w C.  Each warp's P and Q sums go to shared memory (pb, qb:
// [RW][3][32] doubles each) and are added in warp order, so the result is
// deterministic.  A diagonal item gives warp w the partners [w C, (w+1) C)
// of every ion of the block.
template <int MODE, bool QARR, int RW, bool INPLACE>
__global__ void __launch_bounds__(32 * RW) k_pair_sym_rot(int64_t n, int nbk, const double *__restrict__ x,
                                                           const double *__restrict__ y,
                                                           const double *__restrict__ z,
                                                           const double *__restrict__ q, PosF32 pf, double soft2,
                                                           double *__restrict__ acc, int *__restrict__ sync,
                                                           unsigned *err) {
  constexpr int BI = 32, C = 32 / RW, NT = 32 * RW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SD4 *posP = reinterpret_cast<SD4 *>(smem_raw);
  SD4 *posQ = posP + BI;
  double *pb = reinterpret_cast<double *>(posQ + (split_like(MODE) ? 2 * BI : BI));  // [RW][3][32]
  double *qb = pb + RW * 3 * 32;                                                      // [RW][3][32]
  const SymItem it = sym_block_item(INPLACE, sync, nbk);
  const int P = it.P, Q = it.Q;
  const int64_t p0 = (int64_t)P * BI, q0 = (int64_t)Q * BI;
  const int np = (int)min((int64_t)BI, n - p0), nq = (int)min((int64_t)BI, n - q0);
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31, r0 = w * C;
  if (tid < BI) {
    sym_stage<MODE, QARR>(posP, tid, BI, p0 + tid, n, x, y, z, q, pf, false);
    if (P != Q) sym_stage<MODE, QARR>(posQ, tid, BI, q0 + tid, n, x, y, z, q, pf, true);
  }
  float s2h = 0.0f, s2l = 0.0f;
  if (MODE == MODE_DF64) split_f64(soft2, s2h, s2l);
  __syncthreads();
  const float4 *fP = reinterpret_cast<const float4 *>(posP);
  const float4 *fQ = reinterpret_cast<const float4 *>(posQ);
  constexpr bool SEED = MODE == MODE_SPLIT_RSQ;
  double a[3] = {0.0, 0.0, 0.0};
  if (P == Q) {  // ion `lane` against the partners [r0, r0 + C) of the block
    const int i = lane;
    const SD4 pi = posP[i];
    float af[3] = {0, 0, 0}, al[3] = {0, 0, 0};
    for (int j = r0; j < min(r0 + C, np); ++j) {
      if (MODE == MODE_FP64) {
        const SD4 pj = posP[j];
        const double dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
        double sv = rinv3_fp64(dx, dy, dz, soft2);
        if (QARR) sv *= pj.w;
        a[0] = fma(dx, sv, a[0]);
        a[1] = fma(dy, sv, a[1]);
        a[2] = fma(dz, sv, a[2]);
      } else if (MODE == MODE_DF64) {
        const SD4 pj = posP[j];
        float dh[3], dl[3];
        split_f64(pi.x - pj.x, dh[0], dl[0]);
        split_f64(pi.y - pj.y, dh[1], dl[1]);
        split_f64(pi.z - pj.z, dh[2], dl[2]);
        float sh, sl;
        df_rinv3(dh, dl, s2h, s2l, sh, sl);
        if (QARR) {
          float wh, wl;
          split_f64(pj.w, wh, wl);
          const float ph = sh * wh;
          sl = fmaf(sh, wl, fmaf(sl, wh, fmaf(sh, wh, -ph)));
          sh = ph;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float ph = dh[k] * sh;
          const float pl = fmaf(dh[k], sl, fmaf(dl[k], sh, fmaf(dh[k], sh, -ph)));
          float sv, tt;
          two_sum_f(af[k], ph, sv, tt);
          af[k] = sv;
          al[k] += tt + pl;
        }
      } else {
        float fx, fy, fz, wj;
        if (MODE == MODE_MIXED) {
          const SD4 pj = posP[j];
          fx = f64_to_f32_rn(pi.x - pj.x);
          fy = f64_to_f32_rn(pi.y - pj.y);
          fz = f64_to_f32_rn(pi.z - pj.z);
          wj = wf32(pj.w);
        } else {
          const float4 ih = fP[i], il = fP[BI + i], jh = fP[j], jl = fP[BI + j];
          fx = (ih.x - jh.x) + (il.x - jl.x);
          fy = (ih.y - jh.y) + (il.y - jl.y);
          fz = (ih.z - jh.z) + (il.z - jl.z);
          wj = jh.w;
        }
        float sj = f32_rinv3<SEED>(fx, fy, fz, (float)soft2);
        if (QARR) sj *= wj;
        af[0] = fmaf(fx, sj, af[0]);
        af[1] = fmaf(fy, sj, af[1]);
        af[2] = fmaf(fz, sj, af[2]);
      }
    }
    if (MODE != MODE_FP64)
#pragma unroll
      for (int k = 0; k < 3; ++k) a[k] = f32_to_f64(af[k]) + f32_to_f64(al[k]);
#pragma unroll
    for (int c = 0; c < 3; ++c) pb[(w * 3 + c) * 32 + lane] = a[c];
    __syncthreads();
    sym_output<NT>(INPLACE, it, n, p0, np, q0, nq, acc, sync, err,
                   [&](int c, int i) {
                     double v = 0.0;
#pragma unroll
                     for (int u = 0; u < RW; ++u) v += pb[(u * 3 + c) * 32 + i];
                     return v;
                   },
                   [&](int c, int i) { return 0.0; });
    return;
  }
  const bool weighted = QARR || np < BI || nq < BI;
  double b[3] = {0.0, 0.0, 0.0};
  if (MODE == MODE_FP64) {
    const SD4 pp = posP[lane], qd = posQ[(lane + r0) & 31];
    if (weighted)
      sym_step_fp64<true, C>(pp, qd, soft2, lane, a, b);
    else
      sym_step_fp64<false, C>(pp, qd, soft2, lane, a, b);
  } else if (MODE == MODE_DF64) {
    const SD4 pp = posP[lane], qd = posQ[(lane + r0) & 31];
    float ah[3] = {0, 0, 0}, al[3] = {0, 0, 0}, bh[3] = {0, 0, 0}, bl[3] = {0, 0, 0};
    if (weighted)
      sym_step_df64<true, C>(pp, qd, s2h, s2l, lane, ah, al, bh, bl);
    else
      sym_step_df64<false, C>(pp, qd, s2h, s2l, lane, ah, al, bh, bl);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      a[c] = f32_to_f64(ah[c]) + f32_to_f64(al[c]);
      b[c] = f32_to_f64(bh[c]) + f32_to_f64(bl[c]);
    }
  } else {
    float af[3] = {0, 0, 0}, bf[3] = {0, 0, 0};
    if (MODE == MODE_MIXED) {
      const SD4 pp = posP[lane], qd = posQ[(lane + r0) & 31];
      if (weighted)
        sym_step_mixed<true, C>(pp, qd, (float)soft2, lane, af, bf);
      else
        sym_step_mixed<false, C>(pp, qd, (float)soft2, lane, af, bf);
    } else {
      // the doubled Q-tile: entry (lane + r0 + r) at a fixed offset for every r < C
      if (weighted)
        sym_step_split<true, SEED, C>(fP[lane], fP[BI + lane], fQ + lane + r0, fQ + 2 * BI + lane + r0,
                                      (float)soft2, lane, af, bf);
      else
        sym_step_split<false, SEED, C>(fP[lane], fP[BI + lane], fQ + lane + r0, fQ + 2 * BI + lane + r0,
                                       (float)soft2, lane, af, bf);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      a[c] = f32_to_f64(af[c]);
      b[c] = f32_to_f64(bf[c]);
    }
  }
  // after C rotations lane l holds the sums of Q-ion (l + r0 + C) mod 32
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    pb[(w * 3 + c) * 32 + lane] = a[c];
    qb[(w * 3 + c) * 32 + ((lane + r0 + C) & 31)] = b[c];
  }
  __syncthreads();
  sym_output<NT>(INPLACE, it, n, p0, np, q0, nq, acc, sync, err,
                 [&](int c, int i) {
                   double v = 0.0;
#pragma unroll
                   for (int u = 0; u < RW; ++u) v += pb[(u * 3 + c) * 32 + i];
                   return v;
                 },
                 [&](int c, int i) {
                   double v = 0.0;
#pragma unroll
                   for (int u = 0; u < RW; ++u) v += qb[(u * 3 + c) * 32 + i];
                   return v;
                 });
}

// Warps per 32-ion item (rotation split), the fastest measured on GB300 for
// n = 1000-2000 step by step: against one warp per item two were 10 % faster
// for mixed at n = 1000, 4.5 % for fp64 at n = 1500 and 7 % for df64 at
// n = 2000 (2 % slower for mixed at n = 1500); four were slower than two
// everywhere.
constexpr int SYM_ROT_WARPS = 2;

static size_t sym_rot_smem_bytes(int mode) {
  return (size_t)32 * ((split_like(mode) ? 3 : 2) * sizeof(SD4)) + 2 * (size_t)SYM_ROT_WARPS * 3 * 32 * sizeof(double);
}

template <int MODE>
static cudaError_t launch_sym_rot(int64_t n, int nbk, const double *x, const double *y, const double *z,
                                  const double *q, const PosF32 &pf, double soft2, double *part, int *sync,
                                  unsigned *err, bool inplace, cudaStream_t st) {
  constexpr int RW = SYM_ROT_WARPS;
  if (inplace) {
    cudaError_t e = cudaMemsetAsync(sync, 0, sizeof(int) * sym_sync_ints(nbk), st);
    if (e != cudaSuccess) return e;
  }
  const int items = nbk * (nbk + 1) / 2;
  const size_t smem = sym_rot_smem_bytes(MODE);
  if (q && inplace)
    k_pair_sym_rot<MODE, true, RW, true><<<items, 32 * RW, smem, st>>>(n, nbk, x, y, z, q, pf, soft2, part, sync, err);
  else if (q)
    k_pair_sym_rot<MODE, true, RW, false><<<items, 32 * RW, smem, st>>>(n, nbk, x, y, z, q, pf, soft2, part, sync,
                                                                        err);
  else if (inplace)
    k_pair_sym_rot<MODE, false, RW, true><<<items, 32 * RW, smem, st>>>(n, nbk, x, y, z, q, pf, soft2, part, sync,
                                                                        err);
  else
    k_pair_sym_rot<MODE, false, RW, false><<<items, 32 * RW, smem, st>>>(n, nbk, x, y, z, q, pf, soft2, part, sync,
                                                                         err);
  return cudaGetLastError();
}

size_t sym_smem_bytes(int G, int mode) {
  // the split path with four P-ions per lane (G >= 16) keeps two copies of the P sums
  const int acc = (split_like(mode) && G >= 16) ? 6 : 3;
  return (size_t)32 * G * ((split_like(mode) ? 3 : 2) * sizeof(SD4) + acc * sizeof(double));
}

template <int MODE, bool P2, int NT>
static cudaError_t launch_sym_m(int64_t n, int nbk, int G, const double *x, const double *y,
                                const double *z, const double *q, const PosF32 &pf, double soft2,
                                double *part, int *sync, unsigned *err, bool inplace, cudaStream_t st) {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!done[dev]) {
      const int lim = (int)sym_smem_bytes(32, MODE);
      e = cudaFuncSetAttribute(k_pair_sym<MODE, true, P2, NT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pair_sym<MODE, false, P2, NT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 lim);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pair_sym<MODE, true, P2, NT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 lim);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pair_sym<MODE, false, P2, NT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 lim);
      if (e != cudaSuccess) return e;
      done[dev] = true;
    }
  }
  if (inplace) {
    e = cudaMemsetAsync(sync, 0, sizeof(int) * sym_sync_ints(nbk), st);
    if (e != cudaSuccess) return e;
  }
  const int items = nbk * (nbk + 1) / 2;
  const size_t smem = sym_smem_bytes(G, MODE);
  if (q && inplace)
    k_pair_sym<MODE, true, P2, NT, true><<<items, NT, smem, st>>>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err);
  else if (q)
    k_pair_sym<MODE, true, P2, NT, false><<<items, NT, smem, st>>>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err);
  else if (inplace)
    k_pair_sym<MODE, false, P2, NT, true><<<items, NT, smem, st>>>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err);
  else
    k_pair_sym<MODE, false, P2, NT, false><<<items, NT, smem, st>>>(n, nbk, G, x, y, z, q, pf, soft2, part, sync,
                                                                     err);
  return cudaGetLastError();
}

cudaError_t launch_pair_sym(int mode, int64_t n, int nbk, int G, const double *x, const double *y,
                            const double *z, const double *q, const PosF32 &pf, double soft2,
                            double *part, int *sync, unsigned *err, bool inplace, cudaStream_t st) {
  if (G != 1 && G != 2 && G != 4 && G != 8 && G != 16 && G != 32) return cudaErrorInvalidValue;
  constexpr int S = SYM_THREADS_SMALL, L = SYM_THREADS;
  if (G == 1) {  // 32-ion blocks: several warps share an item's rotations
    switch (mode) {
      case MODE_FP64: return launch_sym_rot<MODE_FP64>(n, nbk, x, y, z, q, pf, soft2, part, sync, err, inplace, st);
      case MODE_DF64: return launch_sym_rot<MODE_DF64>(n, nbk, x, y, z, q, pf, soft2, part, sync, err, inplace, st);
      case MODE_MIXED: return launch_sym_rot<MODE_MIXED>(n, nbk, x, y, z, q, pf, soft2, part, sync, err, inplace, st);
      case MODE_SPLIT: return launch_sym_rot<MODE_SPLIT>(n, nbk, x, y, z, q, pf, soft2, part, sync, err, inplace, st);
      case MODE_SPLIT_RSQ:
        return launch_sym_rot<MODE_SPLIT_RSQ>(n, nbk, x, y, z, q, pf, soft2, part, sync, err, inplace, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (G <= 2) {  // 64-ion blocks at small n: one warp per 32-ion tile
    switch (mode) {
      case MODE_FP64:
        return G == 1 ? launch_sym_m<MODE_FP64, false, 32>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st)
                      : launch_sym_m<MODE_FP64, false, 64>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st);
      case MODE_DF64:
        return G == 1 ? launch_sym_m<MODE_DF64, false, 32>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st)
                      : launch_sym_m<MODE_DF64, false, 64>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st);
      case MODE_MIXED:
        return G == 1 ? launch_sym_m<MODE_MIXED, false, 32>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st)
                      : launch_sym_m<MODE_MIXED, false, 64>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st);
      case MODE_SPLIT:
        return G == 1 ? launch_sym_m<MODE_SPLIT, false, 32>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st)
                      : launch_sym_m<MODE_SPLIT, false, 64>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st);
      case MODE_SPLIT_RSQ:
        return G == 1 ? launch_sym_m<MODE_SPLIT_RSQ, false, 32>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err,
                                                                inplace, st)
                      : launch_sym_m<MODE_SPLIT_RSQ, false, 64>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err,
                                                                inplace, st);
      default: return cudaErrorInvalidValue;
    }
  }
  const bool small = G == 4;  // 4 warps for 128-ion blocks
  switch (mode) {
    case MODE_FP64:
      return small ? launch_sym_m<MODE_FP64, false, S>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st)
                   : launch_sym_m<MODE_FP64, false, L>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st);
    case MODE_DF64:
      return small ? launch_sym_m<MODE_DF64, false, S>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st)
                   : launch_sym_m<MODE_DF64, false, L>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st);
    case MODE_MIXED:
      return small ? launch_sym_m<MODE_MIXED, false, S>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st)
                   : launch_sym_m<MODE_MIXED, false, L>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st);
    case MODE_SPLIT:  // four P-ions per lane (128-ion P-tiles) from 512-ion blocks
      if (small) return launch_sym_m<MODE_SPLIT, false, S>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st);
      if (G == 32)  // 1024-ion blocks: 16 warps, two on each of the 8 P-tiles of 128 ions
        return launch_sym_m<MODE_SPLIT, true, 512>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st);
      return G >= 16 ? launch_sym_m<MODE_SPLIT, true, L>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st)
                     : launch_sym_m<MODE_SPLIT, false, L>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st);
    case MODE_SPLIT_RSQ:
      if (small) return launch_sym_m<MODE_SPLIT_RSQ, false, S>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st);
      if (G == 32)  // 1024-ion blocks: 16 warps, two on each of the 8 P-tiles of 128 ions
        return launch_sym_m<MODE_SPLIT_RSQ, true, 512>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st);
      return G >= 16 ? launch_sym_m<MODE_SPLIT_RSQ, true, L>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st)
                     : launch_sym_m<MODE_SPLIT_RSQ, false, L>(n, nbk, G, x, y, z, q, pf, soft2, part, sync, err, inplace, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace nb
