// nb_vjpterm.cuh -- the pair term of the force VJP (the Jacobian-vector
// product of the Sec. III pair sum) and the block-floating double-float sums
// it is accumulated in, shared by the one-sided and the half-pair VJP
// kernels (nb_vjp.cu).
#pragma once

#include "nb_common.cuh"

namespace nb {

// Double-float helpers: exact-product multiply, TwoSum-based add of (hi, lo)
// pairs (relative error about 2^-44) and accumulation of a double-float term
// into a double-float sum.
__device__ __forceinline__ void dfmul(float ah, float al, float bh, float bl, float &h, float &l) {
  h = ah * bh;
  l = fmaf(ah, bl, fmaf(al, bh, fmaf(ah, bh, -h)));
}
__device__ __forceinline__ void dfadd(float ah, float al, float bh, float bl, float &h, float &l) {
  float e;
  two_sum_f(ah, bh, h, e);
  l = e + (al + bl);
}
__device__ __forceinline__ void df_acc(float &ah, float &al, float bh, float bl) {
  float s, e;
  two_sum_f(ah, bh, s, e);
  ah = s;
  al += e + bl;
}

// Unit of a vanishing VJP term (far below any FP64 exponent).
constexpr int VJP_DEAD = -(1 << 24);

// The pair-force VJP term for one pair, T = dl r^-3 - 3 (d . dl) r^-5 d, with
// d the FP64 displacement and dl the FP64 difference of the cotangents.  All
// of it runs in double-float on the FP32 pipe: d is split into FP32 (hi, lo)
// with the scale 2^-sc that puts its largest component (or sqrt(soft2)) in
// [1, 2), dl with its own scale 2^-se; r^2, the seed 1/r with a compensated
// residual, r^-3 and 3 r^-5 with the third-order corrections, the dot product
// and T are formed in those scaled units.  Returns the pair's unit se - 3 sc, with
// T = (th + tl) 2^unit per component; relative error about 2^-44 of the larger
// of the two terms.  When dl = 0, or d = 0 without softening, T = 0: the unit
// is VJP_DEAD and th = tl = 0.
__device__ __forceinline__ int vjp_term(double dx, double dy, double dz, double lx, double ly,
                                                double lz, double soft2, float th[3], float tl[3]) {
  const int ex = (__double2hiint(dx) >> 20) & 0x7ff;
  const int ey = (__double2hiint(dy) >> 20) & 0x7ff;
  const int ez = (__double2hiint(dz) >> 20) & 0x7ff;
  const int e2 = (__double2hiint(soft2) >> 20) & 0x7ff;
  const int es2 = e2 ? ((e2 - 1023) >> 1) + 1023 : 0;
  const int em = max(max(ex, ey), max(ez, es2));
  const int sc = em - 1023;
  const int fx = (__double2hiint(lx) >> 20) & 0x7ff;
  const int fy = (__double2hiint(ly) >> 20) & 0x7ff;
  const int fz = (__double2hiint(lz) >> 20) & 0x7ff;
  const int fm = max(max(fx, fy), fz);
  const int se = fm - 1023;
  float dh[3], dl[3], eh[3], el[3], s2h = 0.0f, s2l = 0.0f;
  split_f64_scaled(dx, sc, dh[0], dl[0]);
  split_f64_scaled(dy, sc, dh[1], dl[1]);
  split_f64_scaled(dz, sc, dh[2], dl[2]);
  split_f64_scaled(lx, se, eh[0], el[0]);
  split_f64_scaled(ly, se, eh[1], el[1]);
  split_f64_scaled(lz, se, eh[2], el[2]);
  if (e2) split_f64_scaled(soft2, 2 * sc, s2h, s2l);
  // double-float r^2, seed, compensated residual (as in df_rinv3)
  const float p0 = dh[0] * dh[0], p1 = dh[1] * dh[1], p2 = dh[2] * dh[2];
  const float q0 = fmaf(dh[0], dh[0], -p0), q1 = fmaf(dh[1], dh[1], -p1), q2 = fmaf(dh[2], dh[2], -p2);
  float h, t1, t2;
  two_sum_f(p0, p1, h, t1);
  two_sum_f(h, p2, h, t2);
  float l = (t1 + t2) + (q0 + q1 + q2);
  l = fmaf(dh[0] + dh[0], dl[0], l);
  l = fmaf(dh[1] + dh[1], dl[1], l);
  l = fmaf(dh[2] + dh[2], dl[2], l);
  if (e2) {
    float t3;
    two_sum_f(h, s2h, h, t3);
    l += t3 + s2l;
  }
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(h));
  const float y2 = y * y;
  const float y2e = fmaf(y, y, -y2);
  float r = fmaf(-h, y2, 1.0f);
  r = fmaf(-h, y2e, r);
  r = fmaf(-l, y2, r);
  const float c3 = r * fmaf(r, 1.875f, 1.5f);
  const float c5 = r * fmaf(r, 4.375f, 2.5f);
  const float y3h = y2 * y;
  float y3e = fmaf(y2, y, -y3h);
  y3e = fmaf(y2e, y, y3e);
  const float y5h = y3h * y2;
  float y5e = fmaf(y3h, y2, -y5h);
  y5e = fmaf(y3h, y2e, fmaf(y3e, y2, y5e));
  const float s3h = y3h, s3l = fmaf(y3h, c3, y3e);
  const float s5h = y5h, s5l = fmaf(y5h, c5, y5e);
  // dot = d . dl (scaled units)
  float dth, dtl, ph, pl;
  dfmul(dh[0], dl[0], eh[0], el[0], dth, dtl);
  dfmul(dh[1], dl[1], eh[1], el[1], ph, pl);
  dfadd(dth, dtl, ph, pl, dth, dtl);
  dfmul(dh[2], dl[2], eh[2], el[2], ph, pl);
  dfadd(dth, dtl, ph, pl, dth, dtl);
  // w = 3 r^-5 dot
  float wh, wl;
  dfmul(dth, dtl, s5h, s5l, wh, wl);
  const float w3h = 3.0f * wh;
  const float w3l = fmaf(3.0f, wh, -w3h) + 3.0f * wl;
  const bool live = em && fm;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float uh, ul, vh, vl, h, l;
    dfmul(eh[k], el[k], s3h, s3l, uh, ul);
    dfmul(dh[k], dl[k], w3h, w3l, vh, vl);
    dfadd(uh, ul, -vh, -vl, h, l);
    th[k] = live ? h : 0.0f;
    tl[k] = live ? l : 0.0f;
  }
  return live ? se - 3 * sc : VJP_DEAD;
}

// Block-floating double-float sums.  Each term comes in its pair's own unit
// (vjp_term); an accumulator holds three (hi, lo) FP32 pairs in one unit 2^e,
// the largest unit it has met.  A term of a larger unit first scales the
// sums down to it; a term of a smaller unit is scaled down to the sums' unit.
// Both scalings are by powers of two, exact down to FP32's normal range
// (below it the part lost is under 2^-126 of the sums' unit).  A kernel
// widens the sums to FP64 once per 32 partners, so the pair loop's only FP64
// work is the six differences.
constexpr int VJP_BF_EMPTY = -(1 << 28);  // the unit of an empty accumulator

// 2^k for k <= 0, 0 below FP32's normal range.
__device__ __forceinline__ float pow2_down(int k) { return k >= -126 ? __int_as_float((127 + k) << 23) : 0.0f; }

__device__ __forceinline__ void bf_acc(float h[3], float l[3], int &e, const float th[3], const float tl[3],
                                       int u) {
  if (u > e) {
    const float f = pow2_down(e - u);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      h[c] *= f;
      l[c] *= f;
    }
    e = u;
  }
  const float f = pow2_down(u - e);
#pragma unroll
  for (int c = 0; c < 3; ++c) df_acc(h[c], l[c], th[c] * f, tl[c] * f);
}

// (h + l) 2^e per component, widened to FP64 (one FP64 add each).
__device__ __forceinline__ void bf_widen(const float h[3], const float l[3], int e, double out[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) out[c] = f32_to_f64_scaled(h[c], e) + f32_to_f64_scaled(l[c], e);
}

// A weight w as an FP32 (hi, lo) pair scaled by its own exponent:
// w = (wh + wl) 2^ew with wh in [1, 2); a zero or subnormal weight gives
// (0, 0) with ew = VJP_DEAD.
__device__ __forceinline__ void vjp_weight(double w, float &wh, float &wl, int &ew) {
  const int eb = (__double2hiint(w) >> 20) & 0x7ff;
  ew = eb ? eb - 1023 : VJP_DEAD;
  wh = wl = 0.0f;
  if (eb) split_f64_scaled(w, ew, wh, wl);
}

}  // namespace nb
