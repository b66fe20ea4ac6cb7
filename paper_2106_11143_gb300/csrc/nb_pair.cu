// nb_pair.cu -- the O(N^2) pair kernels of libnb.so (sm_103a).
//
// Each kernel evaluates the sum over j of a pair term for the i-particles
// of one i-tile and the j-particles of one j-chunk (Eq. 1 of the paper;
// the Sec. III double loop).  Grid: x = i-tile, y = j-chunk.  The j-chunk
// is streamed through shared memory one block-sized tile at a time; every
// thread reads the same j entry (a broadcast load) and applies it to the R
// i-particles it keeps in registers, the GPU analogue of the paper's packed
// i x j register tile (Sec. VI.A).  The partial sums of each (i-tile,
// j-chunk) block go to their own slot of `part`; the epilogue kernels add
// the slots in chunk order, so no atomics are used and the result does not
// depend on scheduling.
//
// 1/sqrt: the paper replaces SQRT+DIV by an approximate reciprocal square
// root refined by Newton-Raphson (Sec. IV).  Here the seed is the FP32
// MUFU.RSQ of an FP32 copy of r^2 built with integer ops, and a single
// third-order refinement is applied directly to r^-3:
//   Y ~ r2^(-1/2),  e = 1 - r2 Y^2,  r^-3 = Y^3 (1 - e)^(-3/2)
//                                        ~ Y^3 (1 + 3/2 e + 15/8 e^2),
// whose truncation error (35/16)|e|^3 < 2^-61 is below FP64 rounding for
// the |e| < 2^-20.7 the seed guarantees.
#include <algorithm>
#include <mutex>
#include <vector>

#include "nb_pairterm.cuh"

namespace nb {

// ---------------------------------------------------------------------------
// Force kernel: part[(jc*3 + c)*ni + i - i0] = sum_{j in chunk jc} w_j d_ij^c / s_ij^3
// for the target ions i in [i0, i0 + ni) (all n ions: i0 = 0, ni = n) and the
// source ions j of chunk jc of [0, n).
template <int MODE, int R, bool QARR>
__global__ void __launch_bounds__(256) k_pair_force(int64_t n, int64_t jchunk, int64_t i0, int64_t ni,
                                                    const double *__restrict__ x,
                                                    const double *__restrict__ y,
                                                    const double *__restrict__ z,
                                                    const double *__restrict__ q, PosF32 pf,
                                                    double soft2, double *__restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int B = blockDim.x;
  const int tid = threadIdx.x;
  const int64_t ibase = i0 + (int64_t)blockIdx.x * B * R + tid;
  const int64_t iend = i0 + ni;
  const int64_t jb = (int64_t)blockIdx.y * jchunk;
  const int64_t je = min(jb + jchunk, n);

  double xi[R], yi[R], zi[R];
  float xh[R], yh[R], zh[R], xl[R], yl[R], zl[R];
  double ad[R][3], cd[R][3];
  float af[R][3];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t i = min(ibase + (int64_t)r * B, iend - 1);
    if (split_like(MODE)) {
      xh[r] = pf.xh[i]; yh[r] = pf.yh[i]; zh[r] = pf.zh[i];
      xl[r] = pf.xl[i]; yl[r] = pf.yl[i]; zl[r] = pf.zl[i];
    } else {
      xi[r] = x[i]; yi[r] = y[i]; zi[r] = z[i];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) { ad[r][c] = 0.0; cd[r][c] = 0.0; af[r][c] = 0.0f; }
  }
  const float soft2f = (float)soft2;
  float s2h = 0.0f, s2l = 0.0f;
  if (MODE == MODE_DF64) split_f64(soft2, s2h, s2l);

  for (int64_t j0 = jb; j0 < je; j0 += B) {
    __syncthreads();
    const int64_t j = j0 + tid;
    if (j < je) {
      if (split_like(MODE)) {
        float4 *s4 = reinterpret_cast<float4 *>(smem_raw);
        const float qf = QARR ? (float)q[j] : 0.0f;
        s4[2 * tid] = make_float4(pf.xh[j], pf.yh[j], pf.zh[j], qf);
        s4[2 * tid + 1] = make_float4(pf.xl[j], pf.yl[j], pf.zl[j], 0.0f);
      } else if (MODE == MODE_DF64) {
        D4 *s4 = reinterpret_cast<D4 *>(smem_raw);
        D4 e = make_d4(x[j], y[j], z[j], 0.0);
        if (QARR) {
          float qh, ql;
          split_f64(q[j], qh, ql);
          *reinterpret_cast<float2 *>(&e.w) = make_float2(qh, ql);
        }
        s4[tid] = e;
      } else {
        D4 *s4 = reinterpret_cast<D4 *>(smem_raw);
        s4[tid] = make_d4(x[j], y[j], z[j], QARR ? q[j] : 0.0);
      }
    }
    __syncthreads();
    const int cnt = (int)min((int64_t)B, je - j0);
    if (MODE == MODE_FP64) {
      const D4 *s4 = reinterpret_cast<const D4 *>(smem_raw);
#pragma unroll 2
      for (int k = 0; k < cnt; ++k) {
        const D4 pj = s4[k];
#pragma unroll
        for (int r = 0; r < R; ++r)
          pair_f64<QARR>(xi[r], yi[r], zi[r], pj, soft2, ad[r][0], ad[r][1], ad[r][2]);
      }
    } else if (ladder_mode(MODE)) {
      const D4 *s4 = reinterpret_cast<const D4 *>(smem_raw);
#pragma unroll 2
      for (int k = 0; k < cnt; ++k) {
        const D4 pj = s4[k];
#pragma unroll
        for (int r = 0; r < R; ++r)
          pair_ladder<MODE, QARR>(xi[r], yi[r], zi[r], pj, soft2, ad[r][0], ad[r][1], ad[r][2]);
      }
    } else if (MODE == MODE_DF64) {
      const D4 *s4 = reinterpret_cast<const D4 *>(smem_raw);
      float al[R][3];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) al[r][c] = 0.0f;
#pragma unroll 2
      for (int k = 0; k < cnt; ++k) {
        const D4 pj = s4[k];
#pragma unroll
        for (int r = 0; r < R; ++r) pair_df64<QARR>(xi[r], yi[r], zi[r], pj, s2h, s2l, af[r], al[r]);
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          ad[r][c] += f32_to_f64(af[r][c]) + f32_to_f64(al[r][c]);
          af[r][c] = 0.0f;
        }
    } else if (MODE == MODE_MIXED) {
      const D4 *s4 = reinterpret_cast<const D4 *>(smem_raw);
#pragma unroll 2
      for (int k = 0; k < cnt; ++k) {
        const D4 pj = s4[k];
        const float qf = QARR ? (float)pj.w : 0.0f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float fx = f64_to_f32_rn(xi[r] - pj.x);
          const float fy = f64_to_f32_rn(yi[r] - pj.y);
          const float fz = f64_to_f32_rn(zi[r] - pj.z);
          pair_f32_bulk<QARR>(fx, fy, fz, qf, soft2f, af[r][0], af[r][1], af[r][2]);
        }
      }
    } else {
      const float4 *s4 = reinterpret_cast<const float4 *>(smem_raw);
#pragma unroll 4
      for (int k = 0; k < cnt; ++k) {
        const float4 ph = s4[2 * k];
        const float4 pl = s4[2 * k + 1];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float fx = (xh[r] - ph.x) + (xl[r] - pl.x);
          const float fy = (yh[r] - ph.y) + (yl[r] - pl.y);
          const float fz = (zh[r] - ph.z) + (zl[r] - pl.z);
          pair_f32_bulk<QARR, MODE == MODE_SPLIT_RSQ>(fx, fy, fz, ph.w, soft2f, af[r][0], af[r][1], af[r][2]);
        }
      }
    }
    if (MODE == MODE_MIXED || split_like(MODE)) {
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) flush_tile(af[r][c], ad[r][c], cd[r][c]);
    }
  }

#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t i = ibase + (int64_t)r * B;
    if (i < iend) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
        part[((int64_t)blockIdx.y * 3 + c) * ni + (i - i0)] =
            (fp64_like(MODE) || MODE == MODE_DF64) ? ad[r][c] : ad[r][c] + cd[r][c];
    }
  }
}

// ---------------------------------------------------------------------------
// Potential kernel (FP64): part[jc*n + i] = sum_{j in chunk, j != i} w_j / s_ij,
// 1/s = Y (1 - e)^(-1/2) ~ Y (1 + e/2 + 3/8 e^2).
template <bool QARR>
__global__ void __launch_bounds__(256) k_pair_phi(int64_t n, int64_t jchunk,
                                                  const double *__restrict__ x,
                                                  const double *__restrict__ y,
                                                  const double *__restrict__ z,
                                                  const double *__restrict__ q, double soft2,
                                                  double *__restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  D4 *s4 = reinterpret_cast<D4 *>(smem_raw);
  const int B = blockDim.x;
  const int tid = threadIdx.x;
  const int64_t i = (int64_t)blockIdx.x * B + tid;
  const int64_t ic = min(i, n - 1);
  const int64_t jb = (int64_t)blockIdx.y * jchunk;
  const int64_t je = min(jb + jchunk, n);
  const double xi = x[ic], yi = y[ic], zi = z[ic];
  double acc = 0.0;
  for (int64_t j0 = jb; j0 < je; j0 += B) {
    __syncthreads();
    const int64_t j = j0 + tid;
    if (j < je) s4[tid] = make_d4(x[j], y[j], z[j], QARR ? q[j] : 1.0);
    __syncthreads();
    const int cnt = (int)min((int64_t)B, je - j0);
    for (int k = 0; k < cnt; ++k) {
      const D4 pj = s4[k];
      const double dx = xi - pj.x, dy = yi - pj.y, dz = zi - pj.z;
      double inv = rinv1_fp64(dx, dy, dz, soft2);
      inv = (j0 + k == ic) ? 0.0 : inv;  // self pair (matters when soft2 > 0)
      acc = QARR ? fma(pj.w, inv, acc) : acc + inv;
    }
  }
  if (i < n) part[(int64_t)blockIdx.y * n + i] = acc;
}

// ---------------------------------------------------------------------------
// Split FP64 positions into FP32 (hi, lo): hi = fl32(x), lo = fl32(x - hi).
// out6 = [xh | yh | zh | xl | yl | zl], n floats each.
__global__ void k_split_positions(int64_t n, const double *__restrict__ x,
                                  const double *__restrict__ y, const double *__restrict__ z,
                                  float *__restrict__ out6) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v[3] = {x[i], y[i], z[i]};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float h = __double2float_rn(v[c]);
    out6[c * n + i] = h;
    out6[(3 + c) * n + i] = __double2float_rn(v[c] - (double)h);
  }
}

// ---------------------------------------------------------------------------
// Launchers.

static int round_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

template <int MODE, int R>
static cudaError_t launch_force_mr(const Plan &pl, int64_t n, int64_t i0, int64_t ni, const double *x,
                                   const double *y, const double *z, const double *q, const PosF32 &pf,
                                   double soft2, double *part, cudaStream_t st) {
  const dim3 grid(pl.n_it, pl.n_jc);
  const size_t smem = (split_like(MODE) ? 2 * sizeof(float4) : sizeof(D4)) * pl.block;
  if (q)
    k_pair_force<MODE, R, true><<<grid, pl.block, smem, st>>>(n, pl.jchunk, i0, ni, x, y, z, q, pf, soft2, part);
  else
    k_pair_force<MODE, R, false><<<grid, pl.block, smem, st>>>(n, pl.jchunk, i0, ni, x, y, z, q, pf, soft2, part);
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_force_m(const Plan &pl, int64_t n, int64_t i0, int64_t ni, const double *x,
                                  const double *y, const double *z, const double *q, const PosF32 &pf,
                                  double soft2, double *part, cudaStream_t st) {
  switch (pl.R) {
    case 1: return launch_force_mr<MODE, 1>(pl, n, i0, ni, x, y, z, q, pf, soft2, part, st);
    case 2: return launch_force_mr<MODE, 2>(pl, n, i0, ni, x, y, z, q, pf, soft2, part, st);
    case 4: return launch_force_mr<MODE, 4>(pl, n, i0, ni, x, y, z, q, pf, soft2, part, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pair_force_range(const Plan &pl, int mode, int64_t n, int64_t i0, int64_t ni,
                                    const double *x, const double *y, const double *z, const double *q,
                                    const PosF32 &pf, double soft2, double *part, cudaStream_t st) {
  if (pl.sym || i0 < 0 || ni < 1 || i0 + ni > n) return cudaErrorInvalidValue;
  switch (mode) {
    case MODE_FP64: return launch_force_m<MODE_FP64>(pl, n, i0, ni, x, y, z, q, pf, soft2, part, st);
    case MODE_MIXED: return launch_force_m<MODE_MIXED>(pl, n, i0, ni, x, y, z, q, pf, soft2, part, st);
    case MODE_SPLIT: return launch_force_m<MODE_SPLIT>(pl, n, i0, ni, x, y, z, q, pf, soft2, part, st);
    case MODE_DF64: return launch_force_m<MODE_DF64>(pl, n, i0, ni, x, y, z, q, pf, soft2, part, st);
    case MODE_SQRTDIV: return launch_force_m<MODE_SQRTDIV>(pl, n, i0, ni, x, y, z, q, pf, soft2, part, st);
    case MODE_RSQ: return launch_force_m<MODE_RSQ>(pl, n, i0, ni, x, y, z, q, pf, soft2, part, st);
    case MODE_RSQ_NR1: return launch_force_m<MODE_RSQ_NR1>(pl, n, i0, ni, x, y, z, q, pf, soft2, part, st);
    case MODE_RSQ_NR2: return launch_force_m<MODE_RSQ_NR2>(pl, n, i0, ni, x, y, z, q, pf, soft2, part, st);
    case MODE_SPLIT_RSQ: return launch_force_m<MODE_SPLIT_RSQ>(pl, n, i0, ni, x, y, z, q, pf, soft2, part, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pair_force(const Plan &pl, int mode, int64_t n, const double *x,
                              const double *y, const double *z, const double *q,
                              const PosF32 &pf, double soft2, double *part, unsigned *err,
                              cudaStream_t st) {
  if (pl.sym)
    return launch_pair_sym(mode, n, pl.nbk, pl.G, x, y, z, q, pf, soft2, part, part_sync(pl, part, n, 3), err,
                           pl.n_jc == 1, st);
  return launch_pair_force_range(pl, mode, n, 0, n, x, y, z, q, pf, soft2, part, st);
}

cudaError_t launch_pair_phi(const Plan &pl, int64_t n, const double *x, const double *y,
                            const double *z, const double *q, double charge, double soft2,
                            double *part, cudaStream_t st) {
  (void)charge;
  const dim3 grid(pl.n_it, pl.n_jc);
  const size_t smem = sizeof(D4) * pl.block;
  if (q)
    k_pair_phi<true><<<grid, pl.block, smem, st>>>(n, pl.jchunk, x, y, z, q, soft2, part);
  else
    k_pair_phi<false><<<grid, pl.block, smem, st>>>(n, pl.jchunk, x, y, z, q, soft2, part);
  return cudaGetLastError();
}

cudaError_t launch_split_positions(int64_t n, const double *x, const double *y, const double *z,
                                   float *out6, cudaStream_t st) {
  const int T = 256;
  k_split_positions<<<round_up(n, T), T, 0, st>>>(n, x, y, z, out6);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Plan: i-tile and j-chunk sizes.  Blocks of one to four warps; enough
// (i-tile, j-chunk) blocks for about 16 per SM so the last wave is short;
// j-chunks of at least 4 tiles so the partial-sum traffic stays small.
// SMs of the current device; without a usable device (host-only planning),
// the GB300's 152.
int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 152;
  }
  return sms;
}

// ---------------------------------------------------------------------------
// Launch-shape overrides (set by the autotuner through nb_set_tuning).
struct TuneEntry {
  int kind, mode;
  int64_t n_lo, n_hi;
  int block, R, bps;
};
static std::mutex g_tune_mu;
static std::vector<TuneEntry> g_tune;
static uint64_t g_tune_gen = 0;

void tuning_set(int kind, int mode, int64_t n_lo, int64_t n_hi, int block, int R, int bps) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.push_back(TuneEntry{kind, mode, n_lo, n_hi, block, R, bps});
  ++g_tune_gen;
}

void tuning_clear() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
  ++g_tune_gen;
}

uint64_t tuning_generation() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return g_tune_gen;
}

bool tuning_lookup(int kind, int mode, int64_t n, int *block, int *R, int *bps) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (auto it = g_tune.rbegin(); it != g_tune.rend(); ++it)  // latest entry wins
    if (it->kind == kind && it->mode == mode && n >= it->n_lo && n <= it->n_hi) {
      *block = it->block;
      *R = it->R;
      *bps = it->bps;
      return true;
    }
  return false;
}

// The symmetric kernels number their work items with an int: at most
// SYM_MAX_BLOCKS blocks (nbk (nbk + 1) / 2 items).
constexpr int64_t SYM_MAX_BLOCKS = 60000;
// Output mode of the symmetric kernels (nb_symsched.cuh): the round-ordered
// in-place adds from SYM_INPLACE_BLOCKS blocks on (at least about 4600
// items, ten waves of three items per SM on 152 SMs, so the chain of nbk
// commits overlaps later rounds' arithmetic), or earlier when the
// per-partner-block partials (nbk * 3n doubles) would pass SYM_PARTIAL_BYTES.
constexpr int64_t SYM_INPLACE_BLOCKS = 96;
constexpr double SYM_PARTIAL_BYTES = 1e9;

static int sym_slots(int64_t n, int64_t nbk) {
  const bool inplace = nbk >= SYM_INPLACE_BLOCKS || (double)nbk * 3.0 * (double)n * 8.0 > SYM_PARTIAL_BYTES;
  return inplace ? 1 : (int)nbk;
}

Plan make_plan(int64_t n, int mode, int kind, bool allow_sym, int64_t ni) {
  Plan pl;
  if (ni < 0) ni = n;
  // Symmetric half-pair kernel for the force paths.  Where
  // it starts and its block sizes are the fastest measured in step sweeps on
  // GB300, counting the epilogue's reads of the partials: from n = 500
  // (split), 1000 (mixed), 1500 (fp64) or 2000 (df64); 32-ion blocks (one
  // warp) first, then 64 from n = 2000-2500, 128 from n = 2500-4096, 256
  // from n = 32768 and 512 from n = 60000; split: 256 from n = 4096 and
  // 512-ion blocks with four P-ions per lane from n = 8000.
  if (allow_sym && kind == 0 &&
      (mode == MODE_FP64 || mode == MODE_DF64 || mode == MODE_MIXED || split_like(mode))) {
    int G;
    bool use;
    if (split_like(mode)) {
      use = n >= 500;
      G = n >= 8000 ? 16 : (n >= 4096 ? 8 : (n >= 2500 ? 4 : (n >= 2000 ? 2 : 1)));
    } else {
      const int64_t from = mode == MODE_MIXED ? 1000 : (mode == MODE_FP64 ? 1500 : 2000);
      const int64_t g2 = mode == MODE_MIXED ? 2000 : 2500;  // 64-ion blocks from here
      const int64_t g4 = mode == MODE_MIXED ? 3000 : 4096;  // 128-ion blocks from here
      use = n >= from;
      G = n >= 60000 ? 16 : (n >= 32768 ? 8 : (n >= g4 ? 4 : (n >= g2 ? 2 : 1)));
    }
    int tb = 0, tr = 0, tbps = 0;
    if (tuning_lookup(4, mode, n, &tb, &tr, &tbps)) {
      use = tr != 0;
      G = tb / 32;
    }
    const int64_t nbk = (n + 32 * G - 1) / (32 * G);
    if (use && nbk <= SYM_MAX_BLOCKS) {
      pl.sym = 1;
      pl.G = G;
      pl.nbk = (int)nbk;
      pl.n_jc = sym_slots(n, nbk);
      pl.block = 256;
      return pl;
    }
  }
  // Symmetric VJP kernel from n = 2500, where it beat the one-sided kernel
  // on GB300 (128-ion blocks below n = 16384, 256 above); tuning kind 5
  // overrides (R = 0 disables).
  if (allow_sym && kind == 2) {
    int G = n >= 16384 ? 8 : 4;
    bool use = n >= 2500;
    int tb = 0, tr = 0, tbps = 0;
    if (tuning_lookup(5, mode, n, &tb, &tr, &tbps)) {
      use = tr != 0;
      G = tb / 32;
    }
    const int64_t nbk = (n + 32 * G - 1) / (32 * G);
    if (use && nbk <= SYM_MAX_BLOCKS) {
      pl.sym = 1;
      pl.G = G;
      pl.nbk = (int)nbk;
      pl.n_jc = sym_slots(n, nbk);
      pl.block = 128;
      return pl;
    }
  }
  int bps;
  if (kind == 0) {
    // force kernel: shapes measured on GB300 (tune.py and step sweeps).  Below
    // n = 8192 a target of 8 blocks per SM: more, shorter j-chunks only add
    // partials for the epilogue once the chunks hold about 30 partners.
    pl.block = n >= 24000 ? 256 : (n >= 3000 ? 128 : (n >= 1500 ? 64 : 32));
    pl.R = (split_like(mode) && n >= 24000) ? 4 : 1;
    bps = n < 8192 ? 8 : 32;
  } else {
    pl.block = n >= 8192 ? 128 : (n >= 2048 ? 64 : 32);
    pl.R = 1;
    bps = pl.block == 32 ? 32 : 16;
  }
  int tb = 0, tr = 0, tbps = 0;
  if (tuning_lookup(kind, mode, n, &tb, &tr, &tbps)) {
    pl.block = tb;
    pl.R = (kind == 0) ? tr : 1;
    bps = tbps;
  }
  const int64_t it = (int64_t)pl.block * pl.R;
  pl.n_it = round_up(n, it);
  // about 16 blocks per SM for large n; small n keeps at least 8 warps per SM
  const int64_t target = (int64_t)device_sm_count() * bps;
  int64_t njc = (target + pl.n_it - 1) / pl.n_it;
  // j-chunks of at least one block of partners; for the force kernel below
  // n = 8192 down to 8 partners, and below n = 128 down to n/16 partners
  // (about 16 chunks), so that many warps share the pair work.  At small n
  // every dependent FP64 instruction costs 64 cycles of latency, so a
  // thread's chain of partners, not throughput, sets the kernel's time; the
  // epilogue adds the chunks with a chain of n_jc/8 + 3.
  const int64_t min_tiles = n >= 8192 ? 4 : 1;
  const int64_t min_chunk = (kind == 0 && n < 8192) ? std::min<int64_t>(8, std::max<int64_t>(1, n / 16))
                                                    : (int64_t)pl.block;
  const int64_t max_jc = std::max<int64_t>(1, n / (min_tiles * min_chunk));
  njc = std::min<int64_t>(std::max<int64_t>(njc, 1), max_jc);
  int64_t chunk = (n + njc - 1) / njc;
  if (chunk >= pl.block) chunk = ((chunk + pl.block - 1) / pl.block) * pl.block;
  pl.jchunk = std::max<int64_t>(chunk, min_chunk);
  pl.n_jc = round_up(n, pl.jchunk);
  // an i-range of ni targets keeps the full plan's chunks and tiles, so each
  // of its ions gets the sums the full launch would give it
  if (ni != n) pl.n_it = round_up(ni, it);
  return pl;
}

}  // namespace nb
