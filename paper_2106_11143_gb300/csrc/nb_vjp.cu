// nb_vjp.cu -- the pair-force VJP kernels.
//
// For a pair (i, j) with d = r_i - r_j and dl = lam_i - lam_j, the VJP term
//   T = dl r^-3 - 3 (d . dl) r^-5 d
// is formed in double-float on the FP32 pipe in the pair's own units
// (vjp_term) and summed per ion, g_i = sum_j w_j T_ij, in block-floating
// double-float sums widened into FP64 once per 32 partners
// (nb_vjpterm.cuh).  The only per-pair FP64 work is the six differences d and
// dl.  NB_FP64 and NB_DF64 share this arithmetic.
//
// One-sided kernel (k_pair_vjp, small n): the (i-tile, j-chunk) grid of the
// force kernel's plan; each thread owns one ion and sums the chunk's
// partners, staged in shared memory, into one partial per chunk.
//
// Half-pair kernel (k_vjp_sym): T changes sign under i <-> j (both d and dl
// do), so one evaluation serves both ions: g_i += w_j T and g_j -= w_i T.  The
// work is organised as in the force kernel (nb_sym.cu): block pairs (P, Q),
// P <= Q, of BI = 32 G ions, drawn from the round-robin schedule of
// nb_symsched.cuh; each warp takes Q-tiles and visits the P-tiles in the
// staggered order pt = (qs + k) mod G, one per barrier-separated step, so the
// warps hold distinct P-tiles and update their shared-memory accumulators
// without atomics.  A lane holds one P-ion (position, weight and lam in
// registers); the Q-tile (64 B per ion) sits twice in shared memory, so the
// entry (lane + r) mod 32 of rotation r is a fixed offset from the lane's
// base; only the Q side's block-floating sums (six floats and their unit)
// rotate, by warp shuffle.  Diagonal items (P == Q) are one-sided.  Output:
// each item adds its sums into acc[c * n + i] in round order
// (nb_symsched.cuh): bitwise reproducible with no partial buffer.
//
// Four warps per block and 128-ion blocks at n < 16384 give enough items to
// fill the GPU at the adjoint's sizes (528 items at n = 4096).
#include <mutex>

#include "nb_vjpterm.cuh"
#include "nb_symsched.cuh"

namespace nb {

constexpr int VJP_THREADS = 128;
constexpr int VJP_W = VJP_THREADS / 32;
constexpr double VJP_FAR = 1e18;

// A staged ion: position, weight, cotangent.  The weight is an FP32 (hi, lo)
// pair in w's bits, scaled by its own exponent ew (vjp_weight).
struct __align__(16) VD8 {
  double x, y, z, w, lx, ly, lz;
  int ew, pad;
};

// One pair evaluation: P-ion p against Q-ion q; (ah, al, ea) += w_q T and,
// with BOTH, (bh, bl, eb) -= w_p T.
template <bool W, bool BOTH>
__device__ __forceinline__ void vjp_eval(const VD8 &p, const VD8 &q, double soft2, float ah[3], float al[3],
                                         int &ea, float bh[3], float bl[3], int &eb) {
  float th[3], tl[3];
  const int out = vjp_term(p.x - q.x, p.y - q.y, p.z - q.z, p.lx - q.lx, p.ly - q.ly, p.lz - q.lz, soft2, th, tl);
  if (W) {
    const float2 wq = *reinterpret_cast<const float2 *>(&q.w);
    const float2 wp = *reinterpret_cast<const float2 *>(&p.w);
    float uh[3], ul[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) dfmul(th[c], tl[c], wq.x, wq.y, uh[c], ul[c]);
    bf_acc(ah, al, ea, uh, ul, out + q.ew);
    if (BOTH) {
#pragma unroll
      for (int c = 0; c < 3; ++c) dfmul(th[c], tl[c], -wp.x, -wp.y, uh[c], ul[c]);
      bf_acc(bh, bl, eb, uh, ul, out + p.ew);
    }
  } else {
    bf_acc(ah, al, ea, th, tl, out);
    if (BOTH) {
      float nh[3], nl[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        nh[c] = -th[c];
        nl[c] = -tl[c];
      }
      bf_acc(bh, bl, eb, nh, nl, out);
    }
  }
}

// Staged entry i of a tile or block (g = global index).  Ions past n are
// weight-0, lam-0 dummies far away.  dup: the half-pair kernel's Q-side
// layout, each 32-ion tile stored twice back to back.
template <bool QARR>
__device__ __forceinline__ void vjp_stage(VD8 *dst, int i, int64_t g, int64_t n, const double *x,
                                          const double *y, const double *z, const double *q,
                                          const double *lx, const double *ly, const double *lz,
                                          bool dup) {
  VD8 e;
  float wh = 0.0f, wl = 0.0f;
  if (g < n) {
    e.x = x[g];
    e.y = y[g];
    e.z = z[g];
    e.lx = lx[g];
    e.ly = ly[g];
    e.lz = lz[g];
    wh = 1.0f;
    e.ew = 0;
    if (QARR) vjp_weight(q[g], wh, wl, e.ew);
  } else {
    e.x = e.y = e.z = VJP_FAR;
    e.lx = e.ly = e.lz = 0.0;
    e.ew = VJP_DEAD;
  }
  *reinterpret_cast<float2 *>(&e.w) = make_float2(wh, wl);
  e.pad = 0;
  if (dup) {
    const int k = (i >> 5) * 64 + (i & 31);
    dst[k] = e;
    dst[k + 32] = e;
  } else {
    dst[i] = e;
  }
}

// ---------------------------------------------------------------------------
// One-sided kernel: part[(jc * 3 + c) * n + i] = sum over the chunk's
// partners j of w_j T_ij (c-th component).
template <bool QARR>
__global__ void __launch_bounds__(256) k_pair_vjp(int64_t n, int64_t jchunk, const double *__restrict__ x,
                                                  const double *__restrict__ y, const double *__restrict__ z,
                                                  const double *__restrict__ q, const double *__restrict__ lx,
                                                  const double *__restrict__ ly, const double *__restrict__ lz,
                                                  double soft2, double *__restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  VD8 *sj = reinterpret_cast<VD8 *>(smem_raw);
  const int B = blockDim.x;
  const int tid = threadIdx.x;
  const int64_t i = (int64_t)blockIdx.x * B + tid;
  const int64_t ic = min(i, n - 1);
  const int64_t jb = (int64_t)blockIdx.y * jchunk;
  const int64_t je = min(jb + jchunk, n);
  VD8 pi;
  pi.x = x[ic];
  pi.y = y[ic];
  pi.z = z[ic];
  pi.lx = lx[ic];
  pi.ly = ly[ic];
  pi.lz = lz[ic];
  pi.w = 0.0;  // the own weight is not used on the one side
  pi.ew = 0;
  pi.pad = 0;
  double g[3] = {0.0, 0.0, 0.0};
  for (int64_t j0 = jb; j0 < je; j0 += B) {
    __syncthreads();
    if (j0 + tid < je) vjp_stage<QARR>(sj, tid, j0 + tid, n, x, y, z, q, lx, ly, lz, false);
    __syncthreads();
    const int cnt = (int)min((int64_t)B, je - j0);
    for (int k0 = 0; k0 < cnt; k0 += 32) {
      float ah[3] = {0.0f, 0.0f, 0.0f}, al[3] = {0.0f, 0.0f, 0.0f};
      int ea = VJP_BF_EMPTY, eb = VJP_BF_EMPTY;
      const int k1 = min(cnt, k0 + 32);
      for (int k = k0; k < k1; ++k) vjp_eval<QARR, false>(pi, sj[k], soft2, ah, al, ea, nullptr, nullptr, eb);
      double t[3];
      bf_widen(ah, al, ea, t);
#pragma unroll
      for (int c = 0; c < 3; ++c) g[c] += t[c];
    }
  }
  if (i < n) {
#pragma unroll
    for (int c = 0; c < 3; ++c) part[((int64_t)blockIdx.y * 3 + c) * n + i] = g[c];
  }
}

// ---------------------------------------------------------------------------
// Half-pair kernel.

// Where an item keeps its finished Q sums (and a diagonal item its block's
// sums): at the start of the Q-tile's own 4 KB of staged entries (64 of 64 B
// in the doubled layout), read only by the warp that owns the tile.  Sum c
// of ion i of the block: double [i / 32][c][i mod 32] with a 512-double
// stride per tile.
__device__ __forceinline__ double &vqsum(VD8 *posQ, int c, int i) {
  return reinterpret_cast<double *>(posQ)[(i >> 5) * 512 + c * 32 + (i & 31)];
}

// 32 rotations of a Q-tile against the lane's P-ion: the P side's sums in
// (ah, al, ea), the Q side's rotating with their ions.
template <bool W>
__device__ __forceinline__ void vjp_tile_pair(const VD8 &pp, const VD8 *qd, int lane, double soft2, double a[3],
                                              double b[3]) {
  float ah[3] = {0.0f, 0.0f, 0.0f}, al[3] = {0.0f, 0.0f, 0.0f};
  float bh[3] = {0.0f, 0.0f, 0.0f}, bl[3] = {0.0f, 0.0f, 0.0f};
  int ea = VJP_BF_EMPTY, eb = VJP_BF_EMPTY;
#pragma unroll 2
  for (int r = 0; r < 32; ++r) {
    vjp_eval<W, true>(pp, qd[r], soft2, ah, al, ea, bh, bl, eb);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      bh[c] = __shfl_sync(0xffffffffu, bh[c], (lane + 1) & 31);
      bl[c] = __shfl_sync(0xffffffffu, bl[c], (lane + 1) & 31);
    }
    eb = __shfl_sync(0xffffffffu, eb, (lane + 1) & 31);
  }
  bf_widen(ah, al, ea, a);
  bf_widen(bh, bl, eb, b);
}

template <bool QARR, bool INPLACE>
__global__ void __launch_bounds__(VJP_THREADS, 4) k_vjp_sym(int64_t n, int nbk, int G,
                                                         const double *__restrict__ x,
                                                         const double *__restrict__ y,
                                                         const double *__restrict__ z,
                                                         const double *__restrict__ q,
                                                         const double *__restrict__ lx,
                                                         const double *__restrict__ ly,
                                                         const double *__restrict__ lz, double soft2,
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
  for (int i = tid; i < BI; i += VJP_THREADS) {
    vjp_stage<QARR>(posP, i, p0 + i, n, x, y, z, q, lx, ly, lz, false);
    if (P != Q) vjp_stage<QARR>(posQ, i, q0 + i, n, x, y, z, q, lx, ly, lz, true);
    accP[i] = 0.0;
    accP[BI + i] = 0.0;
    accP[2 * BI + i] = 0.0;
  }
  __syncthreads();

  if (P == Q) {  // the block's own pairs, one-sided (the self pair gives T = 0)
    for (int i = tid; i < np; i += VJP_THREADS) {
      const VD8 pi = posP[i];
      double a[3] = {0.0, 0.0, 0.0};
      for (int j0 = 0; j0 < np; j0 += 32) {  // tiles of 32 partners, as off the diagonal
        float ah[3] = {0.0f, 0.0f, 0.0f}, al[3] = {0.0f, 0.0f, 0.0f};
        int ea = VJP_BF_EMPTY, eb = VJP_BF_EMPTY;
        for (int j = j0; j < min(np, j0 + 32); ++j)
          vjp_eval<QARR, false>(pi, posP[j], soft2, ah, al, ea, nullptr, nullptr, eb);
        double t[3];
        bf_widen(ah, al, ea, t);
#pragma unroll
        for (int c = 0; c < 3; ++c) a[c] += t[c];
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
      double a[3], b[3];
      if (weighted)
        vjp_tile_pair<true>(pp, qd, lane, soft2, a, b);
      else
        vjp_tile_pair<false>(pp, qd, lane, soft2, a, b);
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
                           bool inplace, cudaStream_t st) {
  if (G != 4 && G != 8) return cudaErrorInvalidValue;
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
      const void *fns[4] = {(const void *)k_vjp_sym<true, false>, (const void *)k_vjp_sym<false, false>,
                            (const void *)k_vjp_sym<true, true>, (const void *)k_vjp_sym<false, true>};
      for (int k = 0; k < 4 && e == cudaSuccess; ++k)
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
#define NB_VJP_LAUNCH(QA, IP)                                                                                  \
  k_vjp_sym<QA, IP><<<items, VJP_THREADS, smem, st>>>(n, nbk, G, x, y, z, q, lx, ly, lz, soft2, part, sync, err)
  if (inplace) {
    if (q) NB_VJP_LAUNCH(true, true); else NB_VJP_LAUNCH(false, true);
  } else {
    if (q) NB_VJP_LAUNCH(true, false); else NB_VJP_LAUNCH(false, false);
  }
#undef NB_VJP_LAUNCH
  return cudaGetLastError();
}

cudaError_t launch_pair_vjp(const Plan &pl, int64_t n, const double *x, const double *y,
                            const double *z, const double *q, const double *lx,
                            const double *ly, const double *lz, double soft2, double *part,
                            unsigned *err, cudaStream_t st) {
  if (pl.sym)
    return launch_vjp_sym(n, pl.nbk, pl.G, x, y, z, q, lx, ly, lz, soft2, part, part_sync(pl, part, n, 3), err,
                          pl.n_jc == 1, st);
  if (pl.block > 256) return cudaErrorInvalidValue;
  const dim3 grid(pl.n_it, pl.n_jc);
  const size_t smem = sizeof(VD8) * pl.block;
  if (q)
    k_pair_vjp<true><<<grid, pl.block, smem, st>>>(n, pl.jchunk, x, y, z, q, lx, ly, lz, soft2, part);
  else
    k_pair_vjp<false><<<grid, pl.block, smem, st>>>(n, pl.jchunk, x, y, z, q, lx, ly, lz, soft2, part);
  return cudaGetLastError();
}

}  // namespace nb
