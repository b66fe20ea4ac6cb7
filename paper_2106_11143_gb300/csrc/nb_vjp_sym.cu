// nb_vjp_sym.cu -- symmetric (half-pair) kernel for the pair-force VJP.
//
// For a pair (i, j) with d = r_i - r_j and dl = lam_i - lam_j, the VJP term
//   T = dl r^-3 - 3 (d . dl) r^-5 d
// changes sign under i <-> j (both d and dl do), so one evaluation serves both
// ions: g_i += w_j T and g_j -= w_i T.  The work is organised as in the force
// kernel (nb_sym.cu): block pairs (P, Q), P <= Q, of BI = 32 G ions, drawn
// from the round-robin schedule of nb_symsched.cuh; each warp takes Q-tiles
// and visits the P-tiles in the staggered order pt = (qs + k) mod G, one per
// barrier-separated step, so the warps hold distinct P-tiles and update
// their shared-memory accumulators without atomics.  A lane holds one P-ion
// (position, weight and lam in registers); the Q-tile (64 B per ion) sits
// twice in shared memory, so the entry (lane + r) mod 32 of rotation r is a
// fixed offset from the lane's base; only the Q accumulators rotate, by warp
// shuffle.  Diagonal items (P == Q) are one-sided.  Output: each item adds
// its sums into acc[c * n + i] in round order (nb_symsched.cuh): bitwise
// reproducible with no partial buffer.
//
// Four warps per block and 128-ion blocks at n < 16384 give enough items to
// fill the GPU at the adjoint's sizes (528 items at n = 4096).
//
// DF (NB_DF64): the terms are vjp_term_df's double-floats in the call's
// fixed units, summed on the FP32 pipe per 32-partner tile (the rotating Q
// sums as six floats instead of three doubles) and widened into the FP64
// accumulators once per tile, which takes the per-pair FP64 work from 15 to
// the 6 differences.  Padding ions sit at the origin with weight 0, so their
// terms are finite and vanish.
#include <mutex>

#include "nb_common.cuh"
#include "nb_symsched.cuh"

namespace nb {

constexpr int VJP_THREADS = 128;
constexpr int VJP_W = VJP_THREADS / 32;
constexpr double VJP_FAR = 1e18;

struct __align__(16) VD8 {
  double x, y, z, w, lx, ly, lz, pad;
};

__device__ __forceinline__ double vshfl_next(double v, int lane) {
  return __shfl_sync(0xffffffffu, v, (lane + 1) & 31);
}

// One pair evaluation: P-ion p against Q-ion q; a (P side) += w_q T,
// b (Q side) -= w_p T.
template <bool W>
__device__ __forceinline__ void vjp_eval(const VD8 &p, const VD8 &q, double soft2, double a[3],
                                         double b[3]) {
  double T[3];
  vjp_term_fp64(p.x - q.x, p.y - q.y, p.z - q.z, p.lx - q.lx, p.ly - q.ly, p.lz - q.lz, soft2, T);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (W) {
      a[c] = fma(q.w, T[c], a[c]);
      b[c] = fma(-p.w, T[c], b[c]);
    } else {
      a[c] += T[c];
      b[c] -= T[c];
    }
  }
}

// The same in double-float: (ah, al) += w_q T', (bh, bl) -= w_p T', with the
// weights carried as FP32 (hi, lo) pairs in w.
template <bool W>
__device__ __forceinline__ void vjp_eval_df(const VD8 &p, const VD8 &q, double soft2, int sc, int se,
                                            float ah[3], float al[3], float bh[3], float bl[3]) {
  float th[3], tl[3];
  vjp_term_df(p.x - q.x, p.y - q.y, p.z - q.z, p.lx - q.lx, p.ly - q.ly, p.lz - q.lz, soft2, sc, se, th, tl);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (W) {
      const float2 wq = *reinterpret_cast<const float2 *>(&q.w);
      const float2 wp = *reinterpret_cast<const float2 *>(&p.w);
      float uh, ul;
      dfmul(th[c], tl[c], wq.x, wq.y, uh, ul);
      df_acc(ah[c], al[c], uh, ul);
      dfmul(th[c], tl[c], wp.x, wp.y, uh, ul);
      df_acc(bh[c], bl[c], -uh, -ul);
    } else {
      df_acc(ah[c], al[c], th[c], tl[c]);
      df_acc(bh[c], bl[c], -th[c], -tl[c]);
    }
  }
}

// Staged entry i of a block (g = global index).  Ions past n are weight-0,
// lam-0 dummies: far away for the FP64 term (whose scaling is per pair), at
// the origin for the double-float one (inside its fixed position unit).  DF
// carries the weight as an FP32 (hi, lo) pair.  dup: the Q-side layout, each
// 32-ion tile stored twice back to back.
template <bool QARR, bool DF>
__device__ __forceinline__ void vjp_stage(VD8 *dst, int i, int64_t g, int64_t n, const double *x,
                                          const double *y, const double *z, const double *q,
                                          const double *lx, const double *ly, const double *lz,
                                          bool dup) {
  VD8 e;
  if (g < n) {
    e.x = x[g];
    e.y = y[g];
    e.z = z[g];
    e.w = QARR ? q[g] : 1.0;
    e.lx = lx[g];
    e.ly = ly[g];
    e.lz = lz[g];
    if (DF) {
      float wh = 1.0f, wl = 0.0f;
      if (QARR) split_f64(q[g], wh, wl);
      *reinterpret_cast<float2 *>(&e.w) = make_float2(wh, wl);
    }
  } else {
    e.x = e.y = e.z = DF ? 0.0 : VJP_FAR;
    e.w = 0.0;  // also the FP32 pair (0, 0)
    e.lx = e.ly = e.lz = 0.0;
  }
  e.pad = 0.0;
  if (dup) {
    const int k = (i >> 5) * 64 + (i & 31);
    dst[k] = e;
    dst[k + 32] = e;
  } else {
    dst[i] = e;
  }
}

// Where an item keeps its finished Q sums (and a diagonal item its block's
// sums): at the start of the Q-tile's own 4 KB of staged entries (64 of 64 B
// in the doubled layout), read only by the warp that owns the tile.  Sum c
// of ion i of the block: double [i / 32][c][i mod 32] with a 512-double
// stride per tile.
__device__ __forceinline__ double &vqsum(VD8 *posQ, int c, int i) {
  return reinterpret_cast<double *>(posQ)[(i >> 5) * 512 + c * 32 + (i & 31)];
}

template <bool QARR, bool DF, bool INPLACE>
__global__ void __launch_bounds__(VJP_THREADS, 4) k_vjp_sym(int64_t n, int nbk, int G,
                                                         const double *__restrict__ x,
                                                         const double *__restrict__ y,
                                                         const double *__restrict__ z,
                                                         const double *__restrict__ q,
                                                         const double *__restrict__ lx,
                                                         const double *__restrict__ ly,
                                                         const double *__restrict__ lz, double soft2,
                                                         const int *__restrict__ scales,
                                                         double *__restrict__ acc,
                                                         int *__restrict__ sync, unsigned *err) {
  constexpr bool inplace = INPLACE;  // the output mode, fixed at compile time
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int BI = 32 * G;
  VD8 *posP = reinterpret_cast<VD8 *>(smem_raw);
  VD8 *posQ = posP + BI;                                      // 2 BI entries (dup)
  double *accP = reinterpret_cast<double *>(posQ + 2 * BI);  // [3][BI]
  const SymItem it = sym_block_item(inplace, sync, nbk);
  const int P = it.P, Q = it.Q;
  const int64_t p0 = (int64_t)P * BI, q0 = (int64_t)Q * BI;
  const int np = (int)min((int64_t)BI, n - p0), nq = (int)min((int64_t)BI, n - q0);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int sc = 0, se = 0, out = 0;
  if (DF) {
    sc = vjp_pos_scale(scales[0], soft2);
    se = vjp_lam_scale(scales[1]);
    out = se - 3 * sc;
  }
  for (int i = tid; i < BI; i += VJP_THREADS) {
    vjp_stage<QARR, DF>(posP, i, p0 + i, n, x, y, z, q, lx, ly, lz, false);
    if (P != Q) vjp_stage<QARR, DF>(posQ, i, q0 + i, n, x, y, z, q, lx, ly, lz, true);
    accP[i] = 0.0;
    accP[BI + i] = 0.0;
    accP[2 * BI + i] = 0.0;
  }
  __syncthreads();

  if (P == Q) {  // the block's own pairs, one-sided (the self pair gives T = 0)
    for (int i = tid; i < np; i += VJP_THREADS) {
      const VD8 pi = posP[i];
      double a[3] = {0.0, 0.0, 0.0}, dummy[3];
      if (DF) {
        for (int j0 = 0; j0 < np; j0 += 32) {  // tiles of 32 partners, as off the diagonal
          float ah[3] = {0.0f, 0.0f, 0.0f}, al[3] = {0.0f, 0.0f, 0.0f};
          float bh[3] = {0.0f, 0.0f, 0.0f}, bl[3] = {0.0f, 0.0f, 0.0f};  // not used
          for (int j = j0; j < min(np, j0 + 32); ++j) vjp_eval_df<QARR>(pi, posP[j], soft2, sc, se, ah, al, bh, bl);
#pragma unroll
          for (int c = 0; c < 3; ++c) a[c] += f32_to_f64_scaled(ah[c], out) + f32_to_f64_scaled(al[c], out);
        }
      } else {
        for (int j = 0; j < np; ++j) vjp_eval<QARR>(pi, posP[j], soft2, a, dummy);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) vqsum(posQ, c, i) = a[c];
    }
    __syncthreads();
    sym_output<VJP_THREADS>(inplace, it, n, p0, np, q0, nq, acc, sync, err,
                            [&](int c, int i) { return vqsum(posQ, c, i); }, [&](int c, int i) { return 0.0; });
    return;
  }

  const bool weighted = QARR || np < BI || nq < BI;
  for (int qs = warp; qs < G; qs += VJP_W) {
    const VD8 *qd = posQ + qs * 64 + lane;
    double aq[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < G; ++k) {
      const int pt = (qs + k) % G;
      __syncthreads();  // all warps are at step k: their P-tiles are distinct
      const int ip = pt * 32 + lane;
      const VD8 pp = posP[ip];
      double a[3] = {0.0, 0.0, 0.0}, b[3] = {0.0, 0.0, 0.0};
      if (DF) {
        float ah[3] = {0.0f, 0.0f, 0.0f}, al[3] = {0.0f, 0.0f, 0.0f};
        float bh[3] = {0.0f, 0.0f, 0.0f}, bl[3] = {0.0f, 0.0f, 0.0f};
        if (weighted) {
#pragma unroll 2
          for (int r = 0; r < 32; ++r) {
            vjp_eval_df<true>(pp, qd[r], soft2, sc, se, ah, al, bh, bl);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              bh[c] = __shfl_sync(0xffffffffu, bh[c], (lane + 1) & 31);
              bl[c] = __shfl_sync(0xffffffffu, bl[c], (lane + 1) & 31);
            }
          }
        } else {
#pragma unroll 2
          for (int r = 0; r < 32; ++r) {
            vjp_eval_df<false>(pp, qd[r], soft2, sc, se, ah, al, bh, bl);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              bh[c] = __shfl_sync(0xffffffffu, bh[c], (lane + 1) & 31);
              bl[c] = __shfl_sync(0xffffffffu, bl[c], (lane + 1) & 31);
            }
          }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          a[c] = f32_to_f64_scaled(ah[c], out) + f32_to_f64_scaled(al[c], out);
          b[c] = f32_to_f64_scaled(bh[c], out) + f32_to_f64_scaled(bl[c], out);
        }
      } else if (weighted) {
#pragma unroll 2
        for (int r = 0; r < 32; ++r) {
          vjp_eval<true>(pp, qd[r], soft2, a, b);
          b[0] = vshfl_next(b[0], lane);
          b[1] = vshfl_next(b[1], lane);
          b[2] = vshfl_next(b[2], lane);
        }
      } else {
#pragma unroll 2
        for (int r = 0; r < 32; ++r) {
          vjp_eval<false>(pp, qd[r], soft2, a, b);
          b[0] = vshfl_next(b[0], lane);
          b[1] = vshfl_next(b[1], lane);
          b[2] = vshfl_next(b[2], lane);
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        accP[c * BI + ip] += a[c];
        aq[c] += b[c];
      }
    }
    __syncwarp();  // every lane is done reading the tile
#pragma unroll
    for (int c = 0; c < 3; ++c) vqsum(posQ, c, qs * 32 + lane) = aq[c];
  }
  __syncthreads();
  sym_output<VJP_THREADS>(inplace, it, n, p0, np, q0, nq, acc, sync, err,
                          [&](int c, int i) { return accP[c * BI + i]; },
                          [&](int c, int i) { return vqsum(posQ, c, i); });
}

static size_t vjp_smem_bytes(int G) { return (size_t)32 * G * (3 * sizeof(VD8) + 3 * sizeof(double)); }

cudaError_t launch_vjp_sym(int64_t n, int nbk, int G, const double *x, const double *y,
                           const double *z, const double *q, const double *lx, const double *ly,
                           const double *lz, double soft2, double *part, int *sync, unsigned *err,
                           bool inplace, cudaStream_t st, bool df, const int *scales) {
  if (G != 4 && G != 8) return cudaErrorInvalidValue;
  if (df && !scales) return cudaErrorInvalidValue;
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!done[dev]) {
      const int lim = (int)vjp_smem_bytes(8);
      const void *fns[8] = {(const void *)k_vjp_sym<true, false, false>, (const void *)k_vjp_sym<false, false, false>,
                            (const void *)k_vjp_sym<true, true, false>, (const void *)k_vjp_sym<false, true, false>,
                            (const void *)k_vjp_sym<true, false, true>, (const void *)k_vjp_sym<false, false, true>,
                            (const void *)k_vjp_sym<true, true, true>, (const void *)k_vjp_sym<false, true, true>};
      for (int k = 0; k < 8 && e == cudaSuccess; ++k)
        e = cudaFuncSetAttribute(fns[k], cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
      if (e != cudaSuccess) return e;
      done[dev] = true;
    }
  }
  if (inplace) {
    e = cudaMemsetAsync(sync, 0, sizeof(int) * sym_sync_ints(nbk), st);
    if (e != cudaSuccess) return e;
  }
  const int items = nbk * (nbk + 1) / 2;
  const size_t smem = vjp_smem_bytes(G);
#define NB_VJP_LAUNCH(QA, DFV, IP)                                                                     \
  k_vjp_sym<QA, DFV, IP><<<items, VJP_THREADS, smem, st>>>(n, nbk, G, x, y, z, q, lx, ly, lz, soft2, scales, part, \
                                                           sync, err)
  if (inplace) {
    if (df) {
      if (q) NB_VJP_LAUNCH(true, true, true); else NB_VJP_LAUNCH(false, true, true);
    } else {
      if (q) NB_VJP_LAUNCH(true, false, true); else NB_VJP_LAUNCH(false, false, true);
    }
  } else {
    if (df) {
      if (q) NB_VJP_LAUNCH(true, true, false); else NB_VJP_LAUNCH(false, true, false);
    } else {
      if (q) NB_VJP_LAUNCH(true, false, false); else NB_VJP_LAUNCH(false, false, false);
    }
  }
#undef NB_VJP_LAUNCH
  return cudaGetLastError();
}

}  // namespace nb
