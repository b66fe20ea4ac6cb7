// nb_batched.cu -- persistent velocity-Verlet kernel for an ensemble of
// independent ion systems of uneven size (e.g. Kibble-Zurek quench
// realisations, Sec. I of the paper: many independent numerical experiments
// for defect statistics).
//
// One launch advances every instance by nsteps.  Each instance belongs to
// exactly one CTA, which keeps the instance's positions (and charges) in
// shared memory for the whole run, so no CTA ever waits on another CTA.
// Per step the CTA runs: drift of its ions, __syncthreads, the all-pairs
// Coulomb sum (the FP64 or the double-float pair term of the single-system
// kernels) and the
// kick/trap/friction/Langevin update of each ion, __syncthreads.  Velocities
// and accelerations stay in global memory (L2-resident).
//
// Load balance: instances are packed onto at most one CTA per SM by the
// longest-processing-time rule on N^2 (host side, nb_plan_batched); each
// CTA runs its instances one after another.  The schedule is passed to the
// kernel by value (__grid_constant__), so a launch needs no host-to-device
// copy and can be captured in a CUDA graph.
//
// Instances of at most 4096 ions use a half-pair force phase (bsym_forces
// below); larger instances use the one-sided phase.
// Either way the arithmetic of an ion depends only on its instance (a fixed
// pair order and accumulation order per ion), not on the schedule or the block
// size, so results are bitwise reproducible.
#include <algorithm>
#include <mutex>
#include <vector>

#include "nb_verlet.cuh"

namespace nb {

struct __align__(16) BD4 {
  double x, y, z, w;
};

constexpr int BATCH_MAX_INST = 1024;
constexpr int BATCH_MAX_BINS = 1024;
static_assert(BATCH_MAX_INST == BATCH_LIMIT_INST, "schedule arrays sized for the validated instance limit");
// ions per instance (BATCH_LIMIT_N, checked on the host): 32 B each in shared memory
static_assert(sizeof(Phys) % 16 == 0 && sizeof(Phys) + BATCH_LIMIT_N * sizeof(BD4) <= 227 * 1024,
              "an instance's parameters and positions fit one block's shared memory");

struct BatchSched {
  int n_inst;
  int n_bins;
  int off[BATCH_MAX_INST + 1];                      // ion offsets of the instances
  unsigned short order[BATCH_MAX_INST];             // instances, grouped by bin
  unsigned short bin_start[BATCH_MAX_BINS + 1];     // bin b = order[bin_start[b] .. bin_start[b+1])
};

// FP64 pair term, identical arithmetic to the single-system force kernel.
template <bool QARR>
__device__ __forceinline__ void bpair(double xi, double yi, double zi, const BD4 &pj, double soft2,
                                      double &ax, double &ay, double &az) {
  const double dx = xi - pj.x;
  const double dy = yi - pj.y;
  const double dz = zi - pj.z;
  double s = rinv3_fp64(dx, dy, dz, soft2);
  if (QARR) s *= pj.w;
  ax = fma(dx, s, ax);
  ay = fma(dy, s, ay);
  az = fma(dz, s, az);
}

// Double-float (FP64-class) pair term, as in the single-system df64 kernel;
// w carries q_j as an FP32 (hi, lo) pair in its bits.
template <bool QARR>
__device__ __forceinline__ void bpair_df64(double xi, double yi, double zi, const BD4 &pj,
                                           float s2h, float s2l, float ah[3], float al[3]) {
  float dh[3], dl[3];
  split_f64(xi - pj.x, dh[0], dl[0]);
  split_f64(yi - pj.y, dh[1], dl[1]);
  split_f64(zi - pj.z, dh[2], dl[2]);
  float sh, sl;
  df_rinv3(dh, dl, s2h, s2l, sh, sl);
  if (QARR) {
    const float2 q = *reinterpret_cast<const float2 *>(&pj.w);
    const float ph = sh * q.x;
    sl = fmaf(sh, q.y, fmaf(sl, q.x, fmaf(sh, q.x, -ph)));
    sh = ph;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float ph = dh[k] * sh;
    const float pl = fmaf(dh[k], sl, fmaf(dl[k], sh, fmaf(dh[k], sh, -ph)));
    float s, t;
    two_sum_f(ah[k], ph, s, t);
    ah[k] = s;
    al[k] += t + pl;
  }
}

// ---------------------------------------------------------------------------
// Half-pair (Newton's third law) force phase for instances of at most
// BATCH_SYM_N ions.  The instance is padded to whole 32-ion tiles with
// weight-0 dummies far away; the per-ion sums go to FP64 accumulators in
// shared memory.  A diagonal phase evaluates each tile against itself
// (one-sided); then Tp - 1 rounds of a round-robin schedule (circle method on
// Tp = T rounded up to even tiles, a bye for odd T) pair every two tiles once,
// each tile appearing once per round, so the warps of a round touch disjoint
// accumulators; a barrier separates the rounds.  Within a tile pair a lane
// holds one ion of tile a, reads tile b at the rotated index (lane + r) mod 32
// and rotates tile b's accumulators by shuffle.  The order of every sum is
// fixed by the schedule, not by the block size.
constexpr int BATCH_SYM_N = 4096;
static_assert(sizeof(Phys) + BATCH_SYM_N * (sizeof(BD4) + 3 * sizeof(double)) <= 227 * 1024,
              "the half-pair phase's accumulators fit beside the positions");

__device__ __forceinline__ double bshfl_next(double v, int lane) {
  return __shfl_sync(0xffffffffu, v, (lane + 1) & 31);
}

template <bool W>
__device__ __forceinline__ void bsym_eval(const BD4 &p, const BD4 &q, double soft2, double a[3],
                                          double b[3]) {
  const double dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
  const double s = rinv3_fp64(dx, dy, dz, soft2);
  const double sp = W ? s * q.w : s, sq = W ? s * p.w : s;
  a[0] = fma(dx, sp, a[0]);
  a[1] = fma(dy, sp, a[1]);
  a[2] = fma(dz, sp, a[2]);
  b[0] = fma(-dx, sq, b[0]);
  b[1] = fma(-dy, sq, b[1]);
  b[2] = fma(-dz, sq, b[2]);
}

// The double-float pair term for both ions (df64): P side (ah, al) += w_q d s,
// Q side (bh, bl) -= w_p d s, with the weights as FP32 (hi, lo) pairs in w.
__device__ __forceinline__ void df_scale(float sh, float sl, double w, float &oh, float &ol) {
  const float2 q = *reinterpret_cast<const float2 *>(&w);
  oh = sh * q.x;
  ol = fmaf(sh, q.y, fmaf(sl, q.x, fmaf(sh, q.x, -oh)));
}

template <bool W>
__device__ __forceinline__ void bsym_eval_df64(const BD4 &p, const BD4 &q, float s2h, float s2l,
                                               float ah[3], float al[3], float bh[3], float bl[3]) {
  float dh[3], dl[3];
  split_f64(p.x - q.x, dh[0], dl[0]);
  split_f64(p.y - q.y, dh[1], dl[1]);
  split_f64(p.z - q.z, dh[2], dl[2]);
  float sh, sl;
  df_rinv3(dh, dl, s2h, s2l, sh, sl);
  float sah = sh, sal = sl, sbh = sh, sbl = sl;
  if (W) {
    df_scale(sh, sl, q.w, sah, sal);
    df_scale(sh, sl, p.w, sbh, sbl);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float ph = dh[k] * sah;
    const float pl = fmaf(dh[k], sal, fmaf(dl[k], sah, fmaf(dh[k], sah, -ph)));
    float u, t;
    two_sum_f(ah[k], ph, u, t);
    ah[k] = u;
    al[k] += t + pl;
    float qh = ph, ql = pl;
    if (W) {
      qh = dh[k] * sbh;
      ql = fmaf(dh[k], sbl, fmaf(dl[k], sbh, fmaf(dh[k], sbh, -qh)));
    }
    two_sum_f(bh[k], -qh, u, t);
    bh[k] = u;
    bl[k] += t - ql;
  }
}

// Tiles (a, b) of round rho, pair k, for Tp tiles (circle method).
__device__ __forceinline__ void round_pair(int rho, int k, int Tp, int &a, int &b) {
  if (k == 0) {
    a = rho;
    b = Tp - 1;
  } else {
    a = (rho + k) % (Tp - 1);
    b = (rho - k + Tp - 1) % (Tp - 1);
  }
}

// The force phase: acc[c * npad + i] = sum_j w_j (r_i - r_j) / |r_i - r_j|^3
// for the instance's np32 staged entries (n real ions, weights in w: an FP64
// value for fp64, an FP32 (hi, lo) pair for df64).
template <bool W, bool DF>
__device__ __forceinline__ void bsym_tile_pair(const BD4 &pp, const BD4 *qt, int lane, double soft2,
                                               float s2h, float s2l, double a[3], double b[3]) {
  if (DF) {
    float ah[3] = {0, 0, 0}, al[3] = {0, 0, 0}, bh[3] = {0, 0, 0}, bl[3] = {0, 0, 0};
#pragma unroll 2
    for (int r = 0; r < 32; ++r) {
      bsym_eval_df64<W>(pp, qt[(lane + r) & 31], s2h, s2l, ah, al, bh, bl);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        bh[c] = __shfl_sync(0xffffffffu, bh[c], (lane + 1) & 31);
        bl[c] = __shfl_sync(0xffffffffu, bl[c], (lane + 1) & 31);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      a[c] = f32_to_f64(ah[c]) + f32_to_f64(al[c]);
      b[c] = f32_to_f64(bh[c]) + f32_to_f64(bl[c]);
    }
  } else {
    a[0] = a[1] = a[2] = b[0] = b[1] = b[2] = 0.0;
#pragma unroll 2
    for (int r = 0; r < 32; ++r) {
      bsym_eval<W>(pp, qt[(lane + r) & 31], soft2, a, b);
      b[0] = bshfl_next(b[0], lane);
      b[1] = bshfl_next(b[1], lane);
      b[2] = bshfl_next(b[2], lane);
    }
  }
}

template <bool QARR, bool DF>
__device__ void bsym_forces(const BD4 *sp, double *acc, int npad, int n, int np32, double soft2,
                            float s2h, float s2l) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
  const int T = np32 >> 5;
  const bool ragged = (n & 31) != 0;
  // diagonal tiles, one-sided (the self pair gives 0)
  for (int t = warp; t < T; t += NW) {
    const int i = t * 32 + lane;
    const BD4 pi = sp[i];
    double a[3] = {0.0, 0.0, 0.0};
    const bool w = QARR || (ragged && t == T - 1);
    if (DF) {
      float ah[3] = {0, 0, 0}, al[3] = {0, 0, 0}, bh[3], bl[3];
      for (int j = 0; j < 32; ++j) {
        bh[0] = bh[1] = bh[2] = bl[0] = bl[1] = bl[2] = 0.0f;  // the partner side is not used
        if (w)
          bsym_eval_df64<true>(pi, sp[t * 32 + j], s2h, s2l, ah, al, bh, bl);
        else
          bsym_eval_df64<false>(pi, sp[t * 32 + j], s2h, s2l, ah, al, bh, bl);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) a[c] = f32_to_f64(ah[c]) + f32_to_f64(al[c]);
    } else {
      double dummy[3];
      if (w) {
        for (int j = 0; j < 32; ++j) bsym_eval<true>(pi, sp[t * 32 + j], soft2, a, dummy);
      } else {
        for (int j = 0; j < 32; ++j) bsym_eval<false>(pi, sp[t * 32 + j], soft2, a, dummy);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[c * npad + i] = a[c];
  }
  __syncthreads();
  const int Tp = T + (T & 1);
  for (int rho = 0; rho < Tp - 1; ++rho) {
    for (int k = warp; k < Tp / 2; k += NW) {
      int ta, tb;
      round_pair(rho, k, Tp, ta, tb);
      if (ta >= T || tb >= T) continue;  // the bye of an odd tile count
      const BD4 pp = sp[ta * 32 + lane];
      const BD4 *qt = sp + tb * 32;
      double a[3], b[3];
      if (QARR || (ragged && (ta == T - 1 || tb == T - 1)))
        bsym_tile_pair<true, DF>(pp, qt, lane, soft2, s2h, s2l, a, b);
      else
        bsym_tile_pair<false, DF>(pp, qt, lane, soft2, s2h, s2l, a, b);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        acc[c * npad + ta * 32 + lane] += a[c];
        acc[c * npad + tb * 32 + lane] += b[c];
      }
    }
    __syncthreads();
  }
}

template <bool QARR, bool DF, bool SYM>
__global__ void __launch_bounds__(512, 1) k_batched(Phys pall, const Phys *__restrict__ ptab, StateView s,
                                                  const __grid_constant__ BatchSched sch,
                                                  int64_t step0, int64_t nsteps, int npad, unsigned *err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Phys &pinst = *reinterpret_cast<Phys *>(smem_raw);  // the running instance's parameters
  BD4 *sp = reinterpret_cast<BD4 *>(smem_raw + sizeof(Phys));
  double *acc = reinterpret_cast<double *>(sp + npad);  // SYM: [3][npad]
  const int T = blockDim.x;
  const int tid = threadIdx.x;
  bool bad = false;

  for (int kk = sch.bin_start[blockIdx.x]; kk < sch.bin_start[blockIdx.x + 1]; ++kk) {
    const int inst = sch.order[kk];
    const int64_t i0 = sch.off[inst];
    const int n = sch.off[inst + 1] - sch.off[inst];
    __syncthreads();  // the previous instance is done with shared memory
    if (tid == 0) {
      // the instance's own table entry, or the shared parameters with the
      // instance word offset by the instance's index
      if (ptab) {
        pinst = ptab[inst];
      } else {
        pinst = pall;
        pinst.instance = pall.instance + (unsigned)inst;
      }
    }
    const int np32 = (n + 31) & ~31;
    if (SYM)
      for (int i = n + tid; i < np32; i += T) sp[i] = BD4{1e18, 1e18, 1e18, 0.0};  // weight-0 dummies
    for (int i = tid; i < n; i += T) {
      BD4 r;
      r.x = s.x[i0 + i]; r.y = s.y[i0 + i]; r.z = s.z[i0 + i];
      r.w = QARR ? s.q[i0 + i] : 1.0;
      if (DF && QARR) {  // q as an FP32 (hi, lo) pair for the double-float pair term
        float qh, ql;
        split_f64(s.q[i0 + i], qh, ql);
        *reinterpret_cast<float2 *>(&r.w) = make_float2(qh, ql);
      } else if (DF) {
        *reinterpret_cast<float2 *>(&r.w) = make_float2(1.0f, 0.0f);
      }
      sp[i] = r;
    }
    __syncthreads();
    const Phys &p = pinst;
    const unsigned inst_id = p.instance;
    const double dt = p.dt, hdt2 = 0.5 * dt * dt;
    const double inv = 1.0 / (1.0 + p.gamma * dt / (2.0 * p.mass)), g = p.gamma / p.mass;
    const double sig = p.noise_T > 0.0 ? sqrt(2.0 * p.gamma * KB * p.noise_T * dt) / p.mass : 0.0;
    const double pref_u = p.k_coulomb * p.charge * p.charge / p.mass;
    const double soft2 = p.soft2;
    float s2h = 0.0f, s2l = 0.0f;
    if (DF) split_f64(soft2, s2h, s2l);
    for (int64_t st = 0; st < nsteps; ++st) {
      const int64_t snew = step0 + st + 1;
      const double t = p.t0 + (double)snew * dt;
      // drift: r+ = r + v dt + a dt^2/2 (each thread its own ions)
      for (int i = tid; i < n; i += T) {
        BD4 r = sp[i];
        r.x = r.x + s.vx[i0 + i] * dt + hdt2 * s.ax[i0 + i];
        r.y = r.y + s.vy[i0 + i] * dt + hdt2 * s.ay[i0 + i];
        r.z = r.z + s.vz[i0 + i] * dt + hdt2 * s.az[i0 + i];
        sp[i] = r;
      }
      __syncthreads();
      // forces at r+ and the kick
      if (SYM) bsym_forces<QARR, DF>(sp, acc, npad, n, np32, soft2, s2h, s2l);
      for (int ib = 0; ib < n; ib += T) {
        const int i = ib + tid;
        const BD4 ri = sp[min(i, n - 1)];
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        if (SYM) {
          if (i < n) {
            a0 = acc[i];
            a1 = acc[npad + i];
            a2 = acc[2 * npad + i];
          }
        } else if (DF) {
          float ah[3] = {0.0f, 0.0f, 0.0f}, al[3] = {0.0f, 0.0f, 0.0f};
          for (int j0 = 0; j0 < n; j0 += 256) {  // double-float sums flushed every 256 partners
            const int j1 = min(n, j0 + 256);
            for (int j = j0; j < j1; ++j) bpair_df64<QARR>(ri.x, ri.y, ri.z, sp[j], s2h, s2l, ah, al);
            a0 += f32_to_f64(ah[0]) + f32_to_f64(al[0]);
            a1 += f32_to_f64(ah[1]) + f32_to_f64(al[1]);
            a2 += f32_to_f64(ah[2]) + f32_to_f64(al[2]);
            ah[0] = ah[1] = ah[2] = al[0] = al[1] = al[2] = 0.0f;
          }
        } else {
#pragma unroll 2
          for (int j = 0; j < n; ++j) bpair<QARR>(ri.x, ri.y, ri.z, sp[j], soft2, a0, a1, a2);
        }
        if (i < n) {
          const int64_t gi = i0 + i;
          const double pref = QARR ? p.k_coulomb * s.q[gi] / p.mass : pref_u;
          double tr[3];
          trap_accel(p, t, ri.x, ri.y, ri.z, tr[0], tr[1], tr[2]);
          double xi[3] = {0.0, 0.0, 0.0};
          if (sig > 0.0) normals3(p.seed, inst_id, snew, i, xi);
          const double acc[3] = {a0, a1, a2};
          double *vs[3] = {s.vx, s.vy, s.vz};
          double *as[3] = {s.ax, s.ay, s.az};
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const double u = pref * acc[k] + tr[k];
            double v = (vs[k][gi] + 0.5 * dt * (as[k][gi] + u)) * inv;
            v += sig * xi[k];
            const double a = u - g * v;
            vs[k][gi] = v;
            as[k][gi] = a;
            bad |= not_finite(v) || not_finite(a);
          }
        }
      }
      __syncthreads();
    }
    for (int i = tid; i < n; i += T) {
      s.x[i0 + i] = sp[i].x;
      s.y[i0 + i] = sp[i].y;
      s.z[i0 + i] = sp[i].z;
    }
  }
  if (bad) atomicOr(err, ERR_NONFINITE);
}

// ---------------------------------------------------------------------------
// Longest-processing-time packing of instances (cost n^2) onto n_bins bins:
// instances in decreasing cost (ties by index) go to the currently lightest
// bin (ties by bin index).  Deterministic.
int batched_plan(int n_inst, const int64_t *offsets, int n_bins, unsigned short *order,
                 unsigned short *bin_start, double *max_load, double *mean_load) {
  std::vector<int> idx(n_inst);
  for (int k = 0; k < n_inst; ++k) idx[k] = k;
  auto cost = [&](int k) { const double m = (double)(offsets[k + 1] - offsets[k]); return m * m; };
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost(a) > cost(b); });
  std::vector<double> load(n_bins, 0.0);
  std::vector<std::vector<int>> bins(n_bins);
  for (int k : idx) {
    int best = 0;
    for (int b = 1; b < n_bins; ++b)
      if (load[b] < load[best]) best = b;
    load[best] += cost(k);
    bins[best].push_back(k);
  }
  int pos = 0;
  double mx = 0.0, sum = 0.0;
  for (int b = 0; b < n_bins; ++b) {
    bin_start[b] = (unsigned short)pos;
    for (int k : bins[b]) order[pos++] = (unsigned short)k;
    mx = std::max(mx, load[b]);
    sum += load[b];
  }
  bin_start[n_bins] = (unsigned short)pos;
  if (max_load) *max_load = mx;
  if (mean_load) *mean_load = n_bins ? sum / n_bins : 0.0;
  return pos;
}

cudaError_t launch_batched(const Phys &p, const Phys *ptab, const StateView &s, int n_inst, const int64_t *offsets,
                           int n_bins, int threads, bool allow_sym, int64_t step0, int64_t nsteps, unsigned *err,
                           cudaStream_t st) {
  BatchSched sch;
  sch.n_inst = n_inst;
  sch.n_bins = n_bins;
  int maxn = 0;
  for (int k = 0; k <= n_inst; ++k) sch.off[k] = (int)offsets[k];
  for (int k = 0; k < n_inst; ++k) maxn = std::max(maxn, (int)(offsets[k + 1] - offsets[k]));
  batched_plan(n_inst, offsets, n_bins, sch.order, sch.bin_start, nullptr, nullptr);
  // Instances of at most BATCH_SYM_N ions use the half-pair force phase,
  // which adds the [3][npad] FP64 accumulators to the positions in shared memory.
  const bool df = p.precision == MODE_DF64;
  const bool sym = allow_sym && maxn <= BATCH_SYM_N;
  const int npad = (std::max(maxn, 1) + 31) & ~31;
  const size_t need = sizeof(Phys) + (sym ? (size_t)npad * (sizeof(BD4) + 3 * sizeof(double))
                                          : (size_t)std::max(maxn, 1) * sizeof(BD4));
  // At least 120 KB of shared memory per CTA, so no SM holds two bins: each
  // bin then owns one SM, which is what the LPT packing assumes.
  const size_t smem = std::max(need, (size_t)120 * 1024);
  static std::mutex mu;
  static bool attr_done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_done[dev]) {
      const int lim = 227 * 1024;
      const void *fns[8] = {(const void *)k_batched<true, false, false>, (const void *)k_batched<false, false, false>,
                            (const void *)k_batched<true, true, false>,  (const void *)k_batched<false, true, false>,
                            (const void *)k_batched<true, false, true>,  (const void *)k_batched<false, false, true>,
                            (const void *)k_batched<true, true, true>,   (const void *)k_batched<false, true, true>};
      for (int f = 0; f < 8 && e == cudaSuccess; ++f)
        e = cudaFuncSetAttribute(fns[f], cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
      if (e != cudaSuccess) return e;
      attr_done[dev] = true;
    }
  }
  if (sym && s.q && df)
    k_batched<true, true, true><<<n_bins, threads, smem, st>>>(p, ptab, s, sch, step0, nsteps, npad, err);
  else if (sym && df)
    k_batched<false, true, true><<<n_bins, threads, smem, st>>>(p, ptab, s, sch, step0, nsteps, npad, err);
  else if (sym && s.q)
    k_batched<true, false, true><<<n_bins, threads, smem, st>>>(p, ptab, s, sch, step0, nsteps, npad, err);
  else if (sym)
    k_batched<false, false, true><<<n_bins, threads, smem, st>>>(p, ptab, s, sch, step0, nsteps, npad, err);
  else if (s.q && df)
    k_batched<true, true, false><<<n_bins, threads, smem, st>>>(p, ptab, s, sch, step0, nsteps, npad, err);
  else if (s.q)
    k_batched<true, false, false><<<n_bins, threads, smem, st>>>(p, ptab, s, sch, step0, nsteps, npad, err);
  else if (df)
    k_batched<false, true, false><<<n_bins, threads, smem, st>>>(p, ptab, s, sch, step0, nsteps, npad, err);
  else
    k_batched<false, false, false><<<n_bins, threads, smem, st>>>(p, ptab, s, sch, step0, nsteps, npad, err);
  return cudaGetLastError();
}

}  // namespace nb
