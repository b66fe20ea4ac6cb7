// nb_small.cu -- velocity-Verlet steps (Sec. II) of a small system in one
// thread block: one launch runs many steps, with the positions in shared
// memory and each ion's velocity and acceleration in its own thread's
// registers.
//
// At small n a step of the multi-kernel path (pair kernel, epilogue) costs a
// few microseconds of launch and kernel latency whatever the work, so the
// step rate stops improving as n shrinks.  Here a step costs two block
// barriers on top of its arithmetic, but all of that arithmetic runs on one
// SM, so the path pays off only while one SM's share of the n^2 pair terms
// is shorter than that latency (the host picks it by n and precision).
//
// The block computes the same work items as the one-sided force kernel's
// plan: ion i against the partners of j-chunk jc, in tiles of the plan's
// block size, with the same pair term and the same per-tile flushes
// (nb_pairterm.cuh).  It keeps the chunk partials in shared memory and adds
// them in the epilogue's order (slot_sum3).  It then applies the same kick
// and drift (nb_verlet.cuh).  Each ion's result is therefore bitwise that of
// the multi-kernel path.
#include <mutex>

#include "nb_pairterm.cuh"
#include "nb_verlet.cuh"

namespace nb {

// Partial sum of ion i over the partners [jb, je), in tiles of `tile`
// partners: the arithmetic of one (i, j-chunk) item of k_pair_force.
template <int MODE, bool QARR>
__device__ __forceinline__ void chunk_partial(const D4 *pos, const float4 *sp, int i, int jb, int je,
                                              int tile, double soft2, float soft2f, float s2h,
                                              float s2l, double out[3]) {
  double ad[3] = {0.0, 0.0, 0.0}, cd[3] = {0.0, 0.0, 0.0};
  float af[3] = {0.0f, 0.0f, 0.0f};
  double xi = 0.0, yi = 0.0, zi = 0.0;
  float xh = 0.0f, yh = 0.0f, zh = 0.0f, xl = 0.0f, yl = 0.0f, zl = 0.0f;
  if (split_like(MODE)) {
    const float4 h = sp[2 * i], l = sp[2 * i + 1];
    xh = h.x; yh = h.y; zh = h.z;
    xl = l.x; yl = l.y; zl = l.z;
  } else {
    const D4 e = pos[i];
    xi = e.x; yi = e.y; zi = e.z;
  }
  for (int j0 = jb; j0 < je; j0 += tile) {
    const int cnt = min(tile, je - j0);
    if (MODE == MODE_FP64) {
#pragma unroll 4
      for (int k = 0; k < cnt; ++k) pair_f64<QARR>(xi, yi, zi, pos[j0 + k], soft2, ad[0], ad[1], ad[2]);
    } else if (ladder_mode(MODE)) {
#pragma unroll 4
      for (int k = 0; k < cnt; ++k)
        pair_ladder<MODE, QARR>(xi, yi, zi, pos[j0 + k], soft2, ad[0], ad[1], ad[2]);
    } else if (MODE == MODE_DF64) {
      float al[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll 4
      for (int k = 0; k < cnt; ++k) pair_df64<QARR>(xi, yi, zi, pos[j0 + k], s2h, s2l, af, al);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        ad[c] += f32_to_f64(af[c]) + f32_to_f64(al[c]);
        af[c] = 0.0f;
      }
    } else if (MODE == MODE_MIXED) {
#pragma unroll 4
      for (int k = 0; k < cnt; ++k) {
        const D4 pj = pos[j0 + k];
        const float qf = QARR ? (float)pj.w : 0.0f;
        const float fx = f64_to_f32_rn(xi - pj.x);
        const float fy = f64_to_f32_rn(yi - pj.y);
        const float fz = f64_to_f32_rn(zi - pj.z);
        pair_f32_bulk<QARR>(fx, fy, fz, qf, soft2f, af[0], af[1], af[2]);
      }
    } else {
#pragma unroll 4
      for (int k = 0; k < cnt; ++k) {
        const float4 ph = sp[2 * (j0 + k)];
        const float4 pl = sp[2 * (j0 + k) + 1];
        const float fx = (xh - ph.x) + (xl - pl.x);
        const float fy = (yh - ph.y) + (yl - pl.y);
        const float fz = (zh - ph.z) + (zl - pl.z);
        pair_f32_bulk<QARR, MODE == MODE_SPLIT_RSQ>(fx, fy, fz, ph.w, soft2f, af[0], af[1], af[2]);
      }
    }
    if (MODE == MODE_MIXED || split_like(MODE)) {
#pragma unroll
      for (int c = 0; c < 3; ++c) flush_tile(af[c], ad[c], cd[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) out[c] = (fp64_like(MODE) || MODE == MODE_DF64) ? ad[c] : ad[c] + cd[c];
}

// Stages ion i at positions r in the form the pair terms read: FP64 position
// and weight (w = q_i, or its FP32 (hi, lo) pair for the double-float term),
// and for the split mode the FP32 (hi, lo) parts of the position as
// k_split_positions forms them, with the FP32 charge beside the high part.
template <int MODE, bool QARR>
__device__ __forceinline__ void stage_ion(D4 *pos, float4 *sp, const StateView &s, int i,
                                          const double r[3]) {
  D4 e = make_d4(r[0], r[1], r[2], (QARR && MODE != MODE_DF64) ? s.q[i] : 0.0);
  if (MODE == MODE_DF64 && QARR) {
    float qh, ql;
    split_f64(s.q[i], qh, ql);
    *reinterpret_cast<float2 *>(&e.w) = make_float2(qh, ql);
  }
  pos[i] = e;
  if (split_like(MODE)) {
    float h[3], l[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      h[c] = __double2float_rn(r[c]);
      l[c] = __double2float_rn(r[c] - (double)h[c]);
    }
    sp[2 * i] = make_float4(h[0], h[1], h[2], QARR ? (float)s.q[i] : 0.0f);
    sp[2 * i + 1] = make_float4(l[0], l[1], l[2], 0.0f);
  }
}

// nsteps steps from (x, v, a) at step index step0; thread i < n owns ion i.
// Per step: [barrier] pair items -> chunk partials [barrier] kick and next
// drift of the own ion.  Writes x, v, a back at the end.
template <int MODE, bool QARR>
__global__ void __launch_bounds__(SMALL_THREADS, 1)
    k_small_steps(Phys p, StateView s, int tile, int jchunk, int n_jc, int64_t step0, int64_t nsteps,
                  unsigned *err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = (int)s.n;
  const int tid = threadIdx.x;
  D4 *pos = reinterpret_cast<D4 *>(smem_raw);
  float4 *sp = reinterpret_cast<float4 *>(pos + n);
  double *part = reinterpret_cast<double *>(sp + (split_like(MODE) ? 2 * n : 0));
  const bool own = tid < n;
  const double dt = p.dt;
  const float soft2f = (float)p.soft2;
  float s2h = 0.0f, s2l = 0.0f;
  if (MODE == MODE_DF64) split_f64(p.soft2, s2h, s2l);

  double r[3] = {0.0, 0.0, 0.0}, v[3] = {0.0, 0.0, 0.0}, a[3] = {0.0, 0.0, 0.0};
  const KickConst kc = kick_consts(p, s, own ? tid : 0);  // once for all the launch's steps
  if (own) {
    v[0] = s.vx[tid]; v[1] = s.vy[tid]; v[2] = s.vz[tid];
    a[0] = s.ax[tid]; a[1] = s.ay[tid]; a[2] = s.az[tid];
    r[0] = verlet_drift(s.x[tid], v[0], a[0], dt);
    r[1] = verlet_drift(s.y[tid], v[1], a[1], dt);
    r[2] = verlet_drift(s.z[tid], v[2], a[2], dt);
    stage_ion<MODE, QARR>(pos, sp, s, tid, r);
  }
  bool bad = false;
  const int items = n * n_jc;
  for (int64_t st = 0; st < nsteps; ++st) {
    __syncthreads();  // this step's positions are staged; last step's partials are read
    for (int it = tid; it < items; it += SMALL_THREADS) {
      const int jc = it / n;
      const int i = it - jc * n;
      const int jb = jc * jchunk;
      double o[3];
      chunk_partial<MODE, QARR>(pos, sp, i, jb, min(jb + jchunk, n), tile, p.soft2, soft2f, s2h, s2l, o);
#pragma unroll
      for (int c = 0; c < 3; ++c) part[(jc * 3 + c) * n + i] = o[c];
    }
    __syncthreads();  // partials complete; nobody reads the positions until the next barrier
    if (own) {
      double cs[3];
      slot_sum3(n_jc, [&](int jc, int c) { return part[(jc * 3 + c) * n + tid]; }, cs);
      bad |= verlet_kick_k(p, kc, tid, step0 + st + 1, r, cs, v, a);
      if (st + 1 < nsteps) {
#pragma unroll
        for (int c = 0; c < 3; ++c) r[c] = verlet_drift(r[c], v[c], a[c], dt);
        stage_ion<MODE, QARR>(pos, sp, s, tid, r);
      }
    }
  }
  if (own) {
    s.x[tid] = r[0]; s.y[tid] = r[1]; s.z[tid] = r[2];
    s.vx[tid] = v[0]; s.vy[tid] = v[1]; s.vz[tid] = v[2];
    s.ax[tid] = a[0]; s.ay[tid] = a[1]; s.az[tid] = a[2];
  }
  if (bad) atomicOr(err, ERR_NONFINITE);
}

size_t small_smem_bytes(const Plan &pl, int mode, int64_t n) {
  return (size_t)n * sizeof(D4) + (split_like(mode) ? (size_t)n * 2 * sizeof(float4) : 0) +
         (size_t)pl.n_jc * 3 * (size_t)n * sizeof(double);
}

template <int MODE>
static cudaError_t launch_small_m(const Plan &pl, const Phys &p, const StateView &s, int64_t step0,
                                  int64_t nsteps, unsigned *err, cudaStream_t st) {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!done[dev]) {
      e = cudaFuncSetAttribute(k_small_steps<MODE, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               SMALL_SMEM_MAX);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_small_steps<MODE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 SMALL_SMEM_MAX);
      if (e != cudaSuccess) return e;
      done[dev] = true;
    }
  }
  const size_t smem = small_smem_bytes(pl, MODE, s.n);
  if (s.q)
    k_small_steps<MODE, true><<<1, SMALL_THREADS, smem, st>>>(p, s, pl.block, (int)pl.jchunk, pl.n_jc,
                                                              step0, nsteps, err);
  else
    k_small_steps<MODE, false><<<1, SMALL_THREADS, smem, st>>>(p, s, pl.block, (int)pl.jchunk, pl.n_jc,
                                                               step0, nsteps, err);
  return cudaGetLastError();
}

cudaError_t launch_small_steps(const Plan &pl, int mode, const Phys &p, const StateView &s,
                               int64_t step0, int64_t nsteps, unsigned *err, cudaStream_t st) {
  if (s.n < 1 || s.n > SMALL_MAX_N || pl.sym || small_smem_bytes(pl, mode, s.n) > (size_t)SMALL_SMEM_MAX)
    return cudaErrorInvalidValue;
  switch (mode) {
    case MODE_FP64: return launch_small_m<MODE_FP64>(pl, p, s, step0, nsteps, err, st);
    case MODE_MIXED: return launch_small_m<MODE_MIXED>(pl, p, s, step0, nsteps, err, st);
    case MODE_SPLIT: return launch_small_m<MODE_SPLIT>(pl, p, s, step0, nsteps, err, st);
    case MODE_DF64: return launch_small_m<MODE_DF64>(pl, p, s, step0, nsteps, err, st);
    case MODE_SQRTDIV: return launch_small_m<MODE_SQRTDIV>(pl, p, s, step0, nsteps, err, st);
    case MODE_RSQ: return launch_small_m<MODE_RSQ>(pl, p, s, step0, nsteps, err, st);
    case MODE_RSQ_NR1: return launch_small_m<MODE_RSQ_NR1>(pl, p, s, step0, nsteps, err, st);
    case MODE_RSQ_NR2: return launch_small_m<MODE_RSQ_NR2>(pl, p, s, step0, nsteps, err, st);
    case MODE_SPLIT_RSQ: return launch_small_m<MODE_SPLIT_RSQ>(pl, p, s, step0, nsteps, err, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace nb
