// nb_pairterm.cuh -- the pair terms of the force sum (Eq. 1; the Sec. III pair
// loop) in each precision, shared by the multi-kernel force kernel
// (nb_pair.cu) and the single-block step kernel (nb_small.cu), so that both
// evaluate an ion's partners with the same instructions.
#pragma once

#include "nb_common.cuh"

namespace nb {

// One staged j-particle: position and weight (or lambda), 16-byte aligned so
// a tile entry is read with two 128-bit shared-memory loads.
struct __align__(16) D4 {
  double x, y, z, w;
};
__device__ __forceinline__ D4 make_d4(double x, double y, double z, double w) {
  D4 r;
  r.x = x; r.y = y; r.z = z; r.w = w;
  return r;
}

// ---------------------------------------------------------------------------
// Pair terms.

// FP64: acc += w_j (r_i - r_j) / (|r_i - r_j|^2 + soft2)^(3/2)
template <bool QARR>
__device__ __forceinline__ void pair_f64(double xi, double yi, double zi, const D4 &pj,
                                         double soft2, double &ax, double &ay, double &az) {
  const double dx = xi - pj.x;
  const double dy = yi - pj.y;
  const double dz = zi - pj.z;
  double s = rinv3_fp64(dx, dy, dz, soft2);
  if (QARR) s *= pj.w;
  ax = fma(dx, s, ax);
  ay = fma(dy, s, ay);
  az = fma(dz, s, az);
}

// FP64 pair term with the 1/sqrt method of the ladder (Sec. IV): SQRT+DIV,
// the bare seed, or the seed refined by y <- y (3 - r^2 y^2) / 2 once or
// twice (the recurrence of Sec. IV); then r^-3 = y^3.
template <int MODE, bool QARR>
__device__ __forceinline__ void pair_ladder(double xi, double yi, double zi, const D4 &pj,
                                            double soft2, double &ax, double &ay, double &az) {
  const double dx = xi - pj.x;
  const double dy = yi - pj.y;
  const double dz = zi - pj.z;
  const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, soft2)));
  double s = ladder_rinv3<MODE>(r2);
  if (QARR) s *= pj.w;
  ax = fma(dx, s, ax);
  ay = fma(dy, s, ay);
  az = fma(dz, s, az);
}

// ---------------------------------------------------------------------------
// FP64-class pair term on the FP32 pipe ("double-float", MODE_DF64).
// The displacement is an FP64 subtraction (exact for close pairs), split into
// FP32 (hi, lo) parts.  r^2 is summed as a double-float from exact products
// (FMA) and TwoSums; r^-3 takes the FP32 seed of its high part and the
// Newton residual formed in compensated FP32, with y^3 kept as a double-float; the
// three force products are exact-product double-floats accumulated with
// TwoSum into a per-tile double-float, flushed into FP64 once per tile.
// Relative error per pair about 2^-44 (the residual's FP32 roundings).

template <bool QARR>
__device__ __forceinline__ void pair_df64(double xi, double yi, double zi, const D4 &pj,
                                          float s2h, float s2l, float ah[3], float al[3]) {
  float dh[3], dl[3];
  split_f64(xi - pj.x, dh[0], dl[0]);
  split_f64(yi - pj.y, dh[1], dl[1]);
  split_f64(zi - pj.z, dh[2], dl[2]);
  float sh, sl;
  df_rinv3(dh, dl, s2h, s2l, sh, sl);
  if (QARR) {  // times q_j, carried as an FP32 pair in the staged entry's w
    const float2 q = *reinterpret_cast<const float2 *>(&pj.w);
    const float ph = sh * q.x;
    const float pe = fmaf(sh, q.x, -ph);
    sl = fmaf(sh, q.y, fmaf(sl, q.x, pe));
    sh = ph;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float ph = dh[k] * sh;
    const float pe = fmaf(dh[k], sh, -ph);
    const float pl = fmaf(dh[k], sl, fmaf(dl[k], sh, pe));
    float s, t;
    two_sum_f(ah[k], ph, s, t);
    ah[k] = s;
    al[k] += t + pl;
  }
}

// Adds a tile's FP32 partial to an FP64 accumulator with TwoSum
// compensation (the error term is kept in c and added at the end).
__device__ __forceinline__ void flush_tile(float &af, double &ad, double &c) {
  double s, e;
  two_sum(ad, f32_to_f64(af), s, e);
  ad = s;
  c += e;
  af = 0.0f;
}

}  // namespace nb
