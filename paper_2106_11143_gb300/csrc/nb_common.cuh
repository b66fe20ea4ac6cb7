// nb_common.cuh -- device helpers and internal launch interface of libnb.so.
//
// Internal to the library: the public ABI is include/nb.h.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/nb.h"

namespace nb {

// ---------------------------------------------------------------------------
// Device error word bits (reported by nb_sync_status).
enum : unsigned { ERR_NONFINITE = 1u, ERR_TIMEOUT = 2u };

// CODATA 2018 exact Boltzmann constant (J/K), for the Langevin kick.
constexpr double KB = 1.380649e-23;

// Pair-arithmetic modes (nb_precision).
enum Mode : int {
  MODE_FP64 = 0,
  MODE_MIXED = 1,
  MODE_SPLIT = 2,
  MODE_DF64 = 3,
  // the 1/sqrt ladder of Sec. IV-VI, all FP64 pair arithmetic:
  MODE_SQRTDIV = 4,  // 1.0 / sqrt(r^2)
  MODE_RSQ = 5,      // hardware seed only (relative error ~2^-22)
  MODE_RSQ_NR1 = 6,  // seed + one FP64 Newton-Raphson step
  MODE_RSQ_NR2 = 7,  // seed + two FP64 Newton-Raphson steps
  // the split positions with the bare FP32 seed for r^-3 (no correction)
  MODE_SPLIT_RSQ = 8
};
// the ladder modes: FP64 pair arithmetic with one of the 1/sqrt methods
__host__ __device__ constexpr bool ladder_mode(int m) { return m >= MODE_SQRTDIV && m <= MODE_RSQ_NR2; }
__host__ __device__ constexpr bool fp64_like(int m) { return m == MODE_FP64 || ladder_mode(m); }
// FP32 (hi, lo) position pairs and FP32 pair arithmetic
__host__ __device__ constexpr bool split_like(int m) { return m == MODE_SPLIT || m == MODE_SPLIT_RSQ; }

// ---------------------------------------------------------------------------
// Integer-only conversions between FP64 and FP32 bit patterns.  On this GPU
// the FP64<->FP32 convert instructions issue on the narrow FP64 pipe (about
// 1.7 lanes/clk/SM), so the pair loop builds the FP32 operand and the FP64
// seed with integer shifts and adds instead (64 lanes/clk/SM).

// 1/sqrt(r2) for an FP64 r2 >= 0, from the FP32 hardware approximation
// (MUFU.RSQ, relative error about 2^-22), returned as an FP64 value.
// r2 = 1.m * 2^E is scaled by 2^-2k (k = floor(E/2)) into [1, 4) while
// building the FP32 bit pattern, so every normal FP64 r2 is accepted; the
// FP32 result is rescaled by 2^-k while building the FP64 bit pattern.
// The mantissa is truncated to 23 bits (relative error < 2^-23 on r2).
// r2 == 0 or subnormal returns 0, which makes the pair contribute nothing.
__device__ __forceinline__ double rsqrt_seed_f64(double r2) {
  const int hi = __double2hiint(r2);
  const unsigned lo = (unsigned)__double2loint(r2);
  const int e = hi >> 20;                     // biased exponent (r2 >= 0)
  const int k = (e - 1023) >> 1;              // floor((e - 1023) / 2)
  const unsigned fs = __funnelshift_l(lo, (unsigned)hi, 3);
  // exponent 127 ([1,2)) when e - 1023 is even, 128 ([2,4)) when odd
  const unsigned fexp = (e & 1) ? 0x3f800000u : 0x40000000u;
  const float r2s = __uint_as_float((fs & 0x007fffffu) | fexp);
  float ys;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(ys) : "f"(r2s));
  const unsigned yb = __float_as_uint(ys);
  const int yhi = (int)(yb >> 3) + ((896 - k) << 20);
  const int ylo = (int)(yb << 29);
  return (e == 0) ? 0.0 : __hiloint2double(yhi, ylo);
}

// r2^(-3/2) by the precision-ladder methods of Sec. IV: SQRT+DIV (1/sqrt in
// FP64), the bare FP32 seed, or the seed refined by one or two Newton steps
// y <- y (3/2 - (r2/2) y^2); then the cube y^3.  r2 == 0 gives 0.
template <int MODE>
__device__ __forceinline__ double ladder_rinv3(double r2) {
  double y;
  if (MODE == MODE_SQRTDIV) {
    y = (r2 > 0.0) ? 1.0 / sqrt(r2) : 0.0;
  } else {
    y = rsqrt_seed_f64(r2);
    if (MODE == MODE_RSQ_NR1 || MODE == MODE_RSQ_NR2) {
      const double h = 0.5 * r2;
      y = y * fma(-h * y, y, 1.5);
      if (MODE == MODE_RSQ_NR2) y = y * fma(-h * y, y, 1.5);
    }
  }
  return (y * y) * y;
}

// FP64 -> FP32 rounded to nearest (ties away from zero) with 32-bit integer
// ops only: 64-bit integer adds and masks would issue on the FP64 pipe.  The
// rounding increment at mantissa bit 29 is a carry-chained 32-bit add.
// |d| < 2^-126 yields an FP32 zero or subnormal of the same sign (such
// displacements only occur as exact zeros); |d| must be below 2^128.
__device__ __forceinline__ float f64_to_f32_rn(double d) {
  const unsigned lo = (unsigned)__double2loint(d);
  const unsigned hi = (unsigned)__double2hiint(d);
  unsigned lo2, ahi2;
  asm("add.cc.u32 %0, %2, 0x10000000;\n\taddc.u32 %1, %3, 0;"
      : "=r"(lo2), "=r"(ahi2)
      : "r"(lo), "r"(hi & 0x7fffffffu));
  const int t = max((int)ahi2 - (896 << 20), 0);  // FP32 exponent field in bits 20..27
  const unsigned mag = __funnelshift_l(lo2, (unsigned)t, 3);
  return __uint_as_float(mag | (hi & 0x80000000u));
}

// Splits an FP64 value into FP32 parts d ~ h + l: h = RN32(d) (integer
// ops), l = RN32(d - h) rebuilt from the 29 mantissa bits below h's rounding
// point (a signed 29-bit integer, converted by I2F and scaled by 2^(E-52)).
// |h + l - d| <= 2^-48 |d| for |d| >= 2^-74; below that l is 0.
__device__ __forceinline__ void split_f64(double d, float &h, float &l) {
  const unsigned lo = (unsigned)__double2loint(d);
  const unsigned hi = (unsigned)__double2hiint(d);
  unsigned lo2, ahi2;
  asm("add.cc.u32 %0, %2, 0x10000000;\n\taddc.u32 %1, %3, 0;"
      : "=r"(lo2), "=r"(ahi2)
      : "r"(lo), "r"(hi & 0x7fffffffu));
  const int t = max((int)ahi2 - (896 << 20), 0);
  const unsigned sign = hi & 0x80000000u;
  h = __uint_as_float(__funnelshift_l(lo2, (unsigned)t, 3) | sign);
  // remainder below the rounding point: the low 29 bits as a signed value
  const int r = ((int)(lo << 3)) >> 3;
  const int e64 = (int)((hi >> 20) & 0x7ffu);
  const int se = max(e64 - 948, 0);  // FP32 exponent field of 2^(E - 52)
  const float scale = __uint_as_float(((unsigned)se << 23) | sign);
  l = __int2float_rn(r) * scale;
}

// Error-free FP32 sum: s + e == a + b exactly (Knuth TwoSum).
__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Double-float pair term: y larger than 2^42 would overflow y^3 (1 + c) in
// FP32; real pairs need |r_i - r_j| >= 2.3e-13 (caller's length unit).
constexpr float DF_YMAX = 4.398046511104e12f;  // 2^42

// Double-float r^-3 (sh + sl) of the FP64 displacement split into FP32
// (hi, lo) parts dh, dl (see pair_df64): double-float r^2 from exact
// products and TwoSums, FP32 seed, compensated Newton residual, y^3 as a
// double-float.  Relative error about 2^-44.
__device__ __forceinline__ void df_rinv3(const float dh[3], const float dl[3], float s2h, float s2l,
                                         float &sh, float &sl) {
  const float p0 = dh[0] * dh[0], p1 = dh[1] * dh[1], p2 = dh[2] * dh[2];
  const float e0 = fmaf(dh[0], dh[0], -p0), e1 = fmaf(dh[1], dh[1], -p1), e2 = fmaf(dh[2], dh[2], -p2);
  float h, t1, t2;
  two_sum_f(p0, p1, h, t1);
  two_sum_f(h, p2, h, t2);
  float l = (t1 + t2) + (e0 + e1 + e2);
  l = fmaf(dh[0] + dh[0], dl[0], l);
  l = fmaf(dh[1] + dh[1], dl[1], l);
  l = fmaf(dh[2] + dh[2], dl[2], l);
  if (s2h != 0.0f) {
    float t3;
    two_sum_f(h, s2h, h, t3);
    l += t3 + s2l;
  }
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(h));
  y = fminf(y, DF_YMAX);
  const float y2 = y * y;
  const float y2e = fmaf(y, y, -y2);
  float r = fmaf(-h, y2, 1.0f);
  r = fmaf(-h, y2e, r);
  r = fmaf(-l, y2, r);
  const float c = r * fmaf(r, 1.875f, 1.5f);
  const float y3h = y2 * y;
  float y3e = fmaf(y2, y, -y3h);
  y3e = fmaf(y2e, y, y3e);
  sh = y3h;
  sl = fmaf(y3h, c, y3e);
}

// Mixed-mode clamp of the FP32 seed: a zero displacement (the self pair, r2 =
// soft2 = 0) gives s = 2.5 * 2^120, finite even times a weight |w_j| < 100, so
// the term is d * s = 0.  Real pairs with |r_i - r_j| >= 2^-40 (9.1e-13 in the
// caller's length unit) never reach the clamp.
constexpr float F32_YMAX = 1.099511627776e12f;  // 2^40

// FP32 (hi, lo) split of d * 2^-sc, sc an integer: split_f64 with the scale
// applied to the exponent fields.  A value that the scale takes below the FP32
// normal range becomes a zero or subnormal (only components negligible next to
// a scaled largest component in [1, 2) do).
__device__ __forceinline__ void split_f64_scaled(double d, int sc, float &h, float &l) {
  const unsigned lo = (unsigned)__double2loint(d);
  const unsigned hi = (unsigned)__double2hiint(d);
  unsigned lo2, ahi2;
  asm("add.cc.u32 %0, %2, 0x10000000;\n\taddc.u32 %1, %3, 0;"
      : "=r"(lo2), "=r"(ahi2)
      : "r"(lo), "r"(hi & 0x7fffffffu));
  const int t = max((int)ahi2 - (896 + sc) * (1 << 20), 0);
  const unsigned sign = hi & 0x80000000u;
  h = __uint_as_float(__funnelshift_l(lo2, (unsigned)t, 3) | sign);
  const int r = ((int)(lo << 3)) >> 3;
  const int e64 = (int)((hi >> 20) & 0x7ffu);
  const int se = max(e64 - 948 - sc, 0);
  l = __int2float_rn(r) * __uint_as_float(((unsigned)se << 23) | sign);
}

// Exact FP32 -> FP64 widening of f * 2^sc by integer ops: a zero or
// subnormal f gives a signed zero, and a result outside the FP64 normal range
// gives a signed zero or infinity.
__device__ __forceinline__ double f32_to_f64_scaled(float f, int sc) {
  const unsigned b = __float_as_uint(f);
  const unsigned a = b & 0x7fffffffu;
  const unsigned sign = b & 0x80000000u;
  const int e = (int)(a >> 23) + 896 + sc;
  const int hi = (int)(sign | ((unsigned)e << 20) | ((a >> 3) & 0xfffffu));
  const int lo = (int)(b << 29);
  if (a < 0x00800000u || e <= 0) return __hiloint2double((int)sign, 0);
  if (e >= 2047) return __hiloint2double((int)(sign | 0x7ff00000u), 0);
  return __hiloint2double(hi, lo);
}

// (|d|^2 + soft2)^(-3/2) for an FP64 displacement d, with the r^2, 1/sqrt and
// cube arithmetic on the FP32 pipe and one FP64 add.  d (and soft2) are scaled
// by 2^-sc so that the largest of |d_k| and sqrt(soft2) lies in [1, 2): the
// double-float r^2, residual and y^3 of df_rinv3 then stay far from FP32
// overflow and underflow for any FP64 input, and the double-float result is
// widened to FP64 with the scale 2^(-3 sc) put back in the exponent.
// Relative error about 2^-44 (the double-float residual).  A zero
// displacement without softening (the self pair) gives 0.
__device__ __forceinline__ double rinv3_fp64(double dx, double dy, double dz, double soft2) {
  const int ex = (__double2hiint(dx) >> 20) & 0x7ff;
  const int ey = (__double2hiint(dy) >> 20) & 0x7ff;
  const int ez = (__double2hiint(dz) >> 20) & 0x7ff;
  const int e2 = (__double2hiint(soft2) >> 20) & 0x7ff;
  const int es = e2 ? ((e2 - 1023) >> 1) + 1023 : 0;  // biased exponent of sqrt(soft2)
  const int em = max(max(ex, ey), max(ez, es));
  const int sc = em - 1023;
  float dh[3], dl[3], s2h = 0.0f, s2l = 0.0f;
  split_f64_scaled(dx, sc, dh[0], dl[0]);
  split_f64_scaled(dy, sc, dh[1], dl[1]);
  split_f64_scaled(dz, sc, dh[2], dl[2]);
  if (e2) split_f64_scaled(soft2, 2 * sc, s2h, s2l);
  float sh, sl;
  df_rinv3(dh, dl, s2h, s2l, sh, sl);
  const double s = f32_to_f64_scaled(sh, -3 * sc) + f32_to_f64_scaled(sl, -3 * sc);
  return em ? s : 0.0;
}

// (|d|^2 + soft2)^(-1/2) for the potential, as rinv3_fp64 does r^-3: the
// double-float r^2 and compensated residual e of df_rinv3, then
// r^-1 = y (1 + 1/2 e + 3/8 e^2) as the double-float (y, y c) widened with one
// FP64 add.  0 for a zero displacement without softening.
__device__ __forceinline__ double rinv1_fp64(double dx, double dy, double dz, double soft2) {
  const int ex = (__double2hiint(dx) >> 20) & 0x7ff;
  const int ey = (__double2hiint(dy) >> 20) & 0x7ff;
  const int ez = (__double2hiint(dz) >> 20) & 0x7ff;
  const int e2 = (__double2hiint(soft2) >> 20) & 0x7ff;
  const int es = e2 ? ((e2 - 1023) >> 1) + 1023 : 0;
  const int em = max(max(ex, ey), max(ez, es));
  const int sc = em - 1023;
  float dh[3], dl[3], s2h = 0.0f, s2l = 0.0f;
  split_f64_scaled(dx, sc, dh[0], dl[0]);
  split_f64_scaled(dy, sc, dh[1], dl[1]);
  split_f64_scaled(dz, sc, dh[2], dl[2]);
  if (e2) split_f64_scaled(soft2, 2 * sc, s2h, s2l);
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
  const float c = r * fmaf(r, 0.375f, 0.5f);
  const double a = f32_to_f64_scaled(y, -sc) + f32_to_f64_scaled(y * c, -sc);
  return em ? a : 0.0;
}

// FP32 r^-3 of an FP32 displacement (the mixed modes' bulk without the
// accumulation): y = MUFU.RSQ(r^2) clamped against FP32 overflow, corrected
// once: s = y^3 (1 + 3/2 e), e = 1 - r^2 y^2.  SEED: the bare seed's cube
// y^3 (Sec. IV's approximate 1/sqrt without a Newton step; the seed's
// relative error 2^-22.9 gives at most 3.9e-7 on r^-3).
template <bool SEED = false>
__device__ __forceinline__ float f32_rinv3(float fx, float fy, float fz, float soft2f) {
  const float r2 = fmaf(fx, fx, fmaf(fy, fy, fmaf(fz, fz, soft2f)));
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r2));
  y = fminf(y, F32_YMAX);
  const float y2 = y * y;
  const float y3 = y2 * y;
  if (SEED) return y3;
  const float e15 = fmaf(-1.5f * r2, y2, 1.5f);
  return fmaf(y3, e15, y3);
}

// FP32 bulk shared by the mixed modes: given the FP32 displacement,
// acc += w_j d / s^3 with s^-3 from f32_rinv3.
template <bool QARR, bool SEED = false>
__device__ __forceinline__ void pair_f32_bulk(float fx, float fy, float fz, float qj,
                                              float soft2f, float &ax, float &ay, float &az) {
  float s = f32_rinv3<SEED>(fx, fy, fz, soft2f);
  if (QARR) s *= qj;
  ax = fmaf(fx, s, ax);
  ay = fmaf(fy, s, ay);
  az = fmaf(fz, s, az);
}

// Exact FP32 -> FP64 widening by integer ops, for normal or zero inputs
// (subnormal FP32 inputs flush to zero).
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned a = b & 0x7fffffffu;
  const int hi = (int)((b & 0x80000000u) | ((a >> 3) + (896u << 20)));
  const int lo = (int)(b << 29);
  return (a < 0x00800000u) ? __hiloint2double((int)(b & 0x80000000u), 0)
                           : __hiloint2double(hi, lo);
}

// Non-finite test on the FP64 bit pattern (exponent all ones).
__device__ __forceinline__ bool not_finite(double v) {
  return (__double2hiint(v) & 0x7ff00000) == 0x7ff00000;
}

// Error-free sum: s + e == a + b exactly (Knuth TwoSum).
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
  s = a + b;
  const double bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

// ---------------------------------------------------------------------------
// Physics parameters as the kernels see them (copied by value).
struct Phys {
  double k_coulomb, mass, charge, soft2;
  int trap, precision;
  double omega[3], omega_rate[3];
  double q_mathieu, omega_rf, rf_phase, gamma, dt, t0, noise_T;
  unsigned long long seed;
  unsigned instance;
};

// Trap acceleration at time t (Eq. 1).
__device__ __forceinline__ void trap_accel(const Phys &p, double t, double x, double y,
                                           double z, double &tx, double &ty, double &tz) {
  if (p.trap == NB_TRAP_RF) {
    const double c = 0.5 * p.q_mathieu * p.omega_rf * p.omega_rf * cos(p.omega_rf * t + p.rf_phase);
    const double wz = p.omega[2] + p.omega_rate[2] * t;
    tx = -c * x;
    ty = c * y;
    tz = -wz * wz * z;
  } else {
    const double wx = p.omega[0] + p.omega_rate[0] * t;
    const double wy = p.omega[1] + p.omega_rate[1] * t;
    const double wz = p.omega[2] + p.omega_rate[2] * t;
    tx = -wx * wx * x;
    ty = -wy * wy * y;
    tz = -wz * wz * z;
  }
}

// ---------------------------------------------------------------------------
// Pair-sum launch plan: blocks of `block` threads, each thread owns R
// i-particles (i-tile = block * R), j split into chunks of `jchunk`
// (a multiple of block) so that n_it * n_jc blocks fill the GPU.  Each
// (i-tile, j-chunk) block writes its partial sums to its own slot; a later
// kernel adds the slots in chunk order, so the result is deterministic.
struct Plan {
  int block = 128;
  int R = 1;
  int64_t jchunk = 0;
  int n_it = 0;
  int n_jc = 0;
  // symmetric (half-pair) kernels: nbk blocks of 32 G ions.  They either
  // add into one output slot in a fixed round order (nb_symsched.cuh,
  // n_jc = 1) or write one partial slot per partner block (n_jc = nbk).
  int sym = 0;
  int G = 0;
  int nbk = 0;
  int pad_ = 0;
};

// kind: 0 force, 1 phi, 2 vjp.  allow_sym = false gives the one-sided plan;
// ni >= 0 (one-sided only) sizes the i-tiles for ni target ions of an
// i-range, keeping the chunks of the full plan.
Plan make_plan(int64_t n, int mode, int kind, bool allow_sym = true, int64_t ni = -1);

// The pair kernel's output buffer: the partial sums [n_jc][ncomp][n]
// doubles, followed for the symmetric kernels by their schedule counters
// (nbk + 1 ints, rounded up to whole doubles).
inline size_t part_doubles(const Plan &pl, int64_t n, int ncomp) {
  return (size_t)pl.n_jc * ncomp * (size_t)n + (pl.sym ? (size_t)(pl.nbk + 2) / 2 : 0);
}
inline int *part_sync(const Plan &pl, double *part, int64_t n, int ncomp) {
  return pl.sym ? reinterpret_cast<int *>(part + (size_t)pl.n_jc * ncomp * (size_t)n) : nullptr;
}
int device_sm_count();

// Host-side argument checks shared by every entry point (nb_api.cu): they
// record a message for nb_last_error() and return NB_EINVAL before any CUDA
// call.  fail() records a printf-style message and returns `s`.
nb_status fail(nb_status s, const char *fmt, ...);
nb_status check_params(const nb_params *p);
nb_status check_system(const nb_system *s, bool need_v, bool need_a);
#define NB_TRY(expr)            \
  do {                          \
    nb_status s_ = (expr);      \
    if (s_ != NB_OK) return s_; \
  } while (0)

// Launch accounting and optional event timing of pair kernels (nb_api.cu).
void count_launches(uint64_t k);
void record_error(const char *msg);  // message returned by nb_last_error()
void timing_begin(cudaStream_t st);
void timing_end(cudaStream_t st);

// Pair kernels (nb_pair.cu).  Partial outputs are [n_jc][3][n] (force, vjp)
// or [n_jc][n] (phi), un-scaled sums over j of the pair terms.
struct PosF32 {  // split FP32 positions for the split modes: hi and lo parts
  const float *xh, *yh, *zh, *xl, *yl, *zl;
};
// part: part_doubles(pl, n, 3) doubles; err: the stream's device error word
// (the symmetric kernels set ERR_TIMEOUT there if a bounded wait gives up).
cudaError_t launch_pair_force(const Plan &pl, int mode, int64_t n, const double *x,
                              const double *y, const double *z, const double *q,
                              const PosF32 &pf, double soft2, double *part, unsigned *err,
                              cudaStream_t st);
// The one-sided force kernel for target ions [i0, i0 + ni) against all n:
// part[(jc * 3 + c) * ni + i - i0]; pl from make_plan(n, mode, 0, false, ni).
cudaError_t launch_pair_force_range(const Plan &pl, int mode, int64_t n, int64_t i0, int64_t ni,
                                    const double *x, const double *y, const double *z, const double *q,
                                    const PosF32 &pf, double soft2, double *part, cudaStream_t st);
cudaError_t launch_pair_phi(const Plan &pl, int64_t n, const double *x, const double *y,
                            const double *z, const double *q, double charge, double soft2,
                            double *part, cudaStream_t st);
// VJP pair kernels (nb_vjp.cu): the one-sided kernel into the plan's chunk
// partials, or the half-pair kernel when pl.sym.
cudaError_t launch_pair_vjp(const Plan &pl, int64_t n, const double *x, const double *y,
                            const double *z, const double *q, const double *lx,
                            const double *ly, const double *lz, double soft2, double *part,
                            unsigned *err, cudaStream_t st);
cudaError_t launch_split_positions(int64_t n, const double *x, const double *y,
                                   const double *z, float *out6, cudaStream_t st);
cudaError_t launch_pair_sym(int mode, int64_t n, int nbk, int G, const double *x, const double *y,
                            const double *z, const double *q, const PosF32 &pf, double soft2,
                            double *part, int *sync, unsigned *err, bool inplace, cudaStream_t st);
cudaError_t launch_vjp_sym(int64_t n, int nbk, int G, const double *x, const double *y,
                           const double *z, const double *q, const double *lx, const double *ly,
                           const double *lz, double soft2, double *part, int *sync, unsigned *err,
                           bool inplace, cudaStream_t st);

// Epilogue kernels (nb_integrate.cu).
struct StateView {
  int64_t n;
  double *x, *y, *z, *vx, *vy, *vz, *ax, *ay, *az;
  const double *q;
  const double *m = nullptr;  // per-ion mass (two species) or nullptr
  int64_t ion0 = 0;           // global index of ion 0 of the view (an i-range's start)
};

// Mass of ion i, and the scale of its trap acceleration relative to the
// reference species of the trap parameters: (q_i/m_i) / (charge/mass).
__device__ __forceinline__ double ion_mass(const Phys &p, const StateView &s, int64_t i) {
  return s.m ? s.m[i] : p.mass;
}
__device__ __forceinline__ double trap_scale(const Phys &p, const StateView &s, int64_t i) {
  if (!s.m && !s.q) return 1.0;
  const double qi = s.q ? s.q[i] : p.charge;
  return (qi / ion_mass(p, s, i)) / (p.charge / p.mass);
}
// The kernels' view of the ABI structs (nb_api.cu).
Phys to_phys(const nb_params *p);
StateView to_view(const nb_system *s);
cudaError_t launch_epi_forces(const Phys &p, const StateView &s, const double *part, int n_jc,
                              int flags, double t, unsigned *err, cudaStream_t st);
cudaError_t launch_epi_vjp(const Phys &p, const StateView &s, const double *part, int n_jc,
                           const double *lx, const double *ly, const double *lz, double *gx,
                           double *gy, double *gz, int flags, double t, cudaStream_t st);
cudaError_t launch_drift(const Phys &p, const StateView &s, double *px, double *py, double *pz,
                         cudaStream_t st);
// One Verlet epilogue: forces at positions (cx,cy,cz) = r+ (time index snew)
// -> kick v and a in s; then drift into (nx,ny,nz) if nx != nullptr, else
// copy r+ into s.x/y/z.
cudaError_t launch_epi_step(const Phys &p, const StateView &s, const double *cx,
                            const double *cy, const double *cz, const double *part, int n_jc,
                            int64_t snew, double *nx, double *ny, double *nz, unsigned *err,
                            cudaStream_t st, const int64_t *cin = nullptr,
                            int64_t *cout = nullptr, int64_t cout_off = 0);
// Ensemble kernel (nb_batched.cu).
int batched_plan(int n_inst, const int64_t *offsets, int n_bins, unsigned short *order,
                 unsigned short *bin_start, double *max_load, double *mean_load);
cudaError_t launch_batched(const Phys &p, const Phys *ptab, const StateView &s, int n_inst, const int64_t *offsets,
                           int n_bins, int threads, bool allow_sym, int64_t step0, int64_t nsteps,
                           unsigned *err, cudaStream_t st);
constexpr int BATCH_LIMIT_INST = 1024;
constexpr int BATCH_LIMIT_N = 6144;
// Single-block step kernel for small systems (nb_small.cu): one thread per
// ion in the kick, so at most SMALL_THREADS ions; positions and the chunk
// partials of the one-sided plan `pl` in at most SMALL_SMEM_MAX bytes of
// shared memory (small_smem_bytes).
constexpr int SMALL_THREADS = 512;
constexpr int SMALL_MAX_N = SMALL_THREADS;
constexpr int SMALL_SMEM_MAX = 227 * 1024;
size_t small_smem_bytes(const Plan &pl, int mode, int64_t n);
cudaError_t launch_small_steps(const Plan &pl, int mode, const Phys &p, const StateView &s,
                               int64_t step0, int64_t nsteps, unsigned *err, cudaStream_t st);

// An NVTX range over an ABI call, so that timeline tools (nsys, ncu --nvtx)
// can attribute kernels to the call that launched them.  Header-only NVTX 3:
// without an attached tool a push or pop is a branch on a null pointer.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// Launch-shape overrides set by nb_set_tuning (nb_pair.cu); kind 3 is the
// ensemble kernel (block = threads per CTA).
bool tuning_lookup(int kind, int mode, int64_t n, int *block, int *R, int *blocks_per_sm);
uint64_t tuning_generation();  // changes whenever the override table does
void tuning_set(int kind, int mode, int64_t n_lo, int64_t n_hi, int block, int R, int blocks_per_sm);
void tuning_clear();

// Adjoint kernels (nb_adjoint.cu).
cudaError_t launch_adj_init(const Phys &p, int64_t n, const double *const xT[3],
                            const double *const aT[3], const double *const tgt[3], double *const xb[3],
                            double *const vb[3], double *const ab[3], double *const wacc[3],
                            cudaStream_t st);
cudaError_t launch_adj_epi(const Phys &p, int64_t n, const double *q, const double *const x[3],
                           const double *part, int n_jc, double *const xb[3], double *const vb[3],
                           double *const ab[3], double *const wacc[3], int last, int more,
                           cudaStream_t st);
cudaError_t launch_adj_out(int64_t n, double *const xb[3], double *const vb[3], double *const wacc[3],
                           const double *gscale, double *gx0, double *gv0, double *gw, double *bpart,
                           cudaStream_t st);
cudaError_t launch_loss(const Phys &p, int64_t n, const double *q, const double *const x[3],
                        const double *const tgt[3], const double *phi_part, int n_jc, double *bpart,
                        double *loss, cudaStream_t st);
constexpr int ADJ_PART_BLOCKS = 128;

// Energies: block partials then one final block; out4 is device memory.
constexpr int ENERGY_BLOCKS = 128;
constexpr int ENERGY_THREADS = 256;
cudaError_t launch_energy(const Phys &p, const StateView &s, const double *phi_part, int n_jc,
                          double t, double *block_part, double *out4, cudaStream_t st);

}  // namespace nb
