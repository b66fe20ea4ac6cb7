// nb_integrate.cu -- O(N) kernels of libnb.so: the epilogues that turn the
// pair partial sums into accelerations (Eq. 1), the velocity-Verlet kick and
// drift (Sec. II), the Langevin kick, and the energy reduction.
#include "nb_verlet.cuh"

namespace nb {

static int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

// Sum of the chunk partials of component c for ion i, in chunk order.
__device__ __forceinline__ double chunk_sum(const double *__restrict__ part, int n_jc, int ncomp,
                                           int c, int64_t n, int64_t i) {
  double s = 0.0;
  for (int jc = 0; jc < n_jc; ++jc) s += part[((int64_t)jc * ncomp + c) * n + i];
  return s;
}

// The three components of ion i's chunk partials, part[(jc*3 + c)*n + i],
// summed by slot_sum3 with streaming loads (the partials are read once).
__device__ __forceinline__ void chunk_sum3(const double *__restrict__ part, int n_jc, int64_t n,
                                           int64_t i, double out[3]) {
  const double *p = part + i;
  slot_sum3(n_jc, [&](int jc, int c) { return __ldcs(p + ((int64_t)jc * 3 + c) * n); }, out);
}

// The epilogues run with EPI_THREADS threads per block, one of two ways:
//  - one thread per ion, adding its chunk partials with chunk_sum3;
//  - eight threads per ion (the default): warp u of a block forms slot_sum3's
//    running sum u (chunks u, u+8, ...) for the block's 32 ions, and the
//    eight sums go through shared memory to the first warp, which adds them in
//    slot_sum3's pairing and finishes one ion per lane.  The dependent chain
//    of the sum is spread over eight threads, each warp load reads 256
//    contiguous bytes, and the FP64 tail still serves 32 ions per warp
//    instruction.
// Both give the same sums, bit for bit.  epi_sums returns false for threads
// without an ion (the caller then returns); it holds a block barrier in the
// eight-lane form, so every thread of the block must call it.
constexpr int EPI_THREADS = 256;

template <bool EIGHT>
__device__ __forceinline__ bool epi_sums(const double *__restrict__ part, int n_jc, int64_t n,
                                         int64_t &i, double cs[3]) {
  if (!EIGHT) {
    i = (int64_t)blockIdx.x * EPI_THREADS + threadIdx.x;
    if (i >= n) return false;
    chunk_sum3(part, n_jc, n, i, cs);
    return true;
  }
  // Warp u of the block forms running sum u (slots u, u+8, ...) for the
  // block's 32 ions, one ion per lane: each load of a warp reads one slot of
  // 32 consecutive ions, 256 contiguous bytes (two L1 lines).
  static_assert(EPI_THREADS == 256, "eight warps, one per running sum");
  const int u = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int64_t g = (int64_t)blockIdx.x * 32 + l;
  const int64_t ig = g < n ? g : n - 1;  // every warp reaches the barrier
  cs[0] = cs[1] = cs[2] = 0.0;
  const double *pi = part + ig;
  for (int jc = u; jc < n_jc; jc += 8) {
    const double *q = pi + (int64_t)jc * 3 * n;
    cs[0] += __ldcs(q);
    cs[1] += __ldcs(q + n);
    cs[2] += __ldcs(q + 2 * n);
  }
  __shared__ double csum[3][8][32];
  csum[0][u][l] = cs[0];
  csum[1][u][l] = cs[1];
  csum[2][u][l] = cs[2];
  __syncthreads();
  if (threadIdx.x >= 32) return false;
  i = g;
  if (i >= n) return false;
#pragma unroll
  for (int c = 0; c < 3; ++c) {  // slot_sum3's pairing of the eight running sums
    const double(*s)[32] = csum[c];
    cs[c] = ((s[0][l] + s[1][l]) + (s[2][l] + s[3][l])) + ((s[4][l] + s[5][l]) + (s[6][l] + s[7][l]));
  }
  return true;
}

// Eight threads per ion unless tuning kind 8 says one (R = 0) for this n:
// measured on GB300 the eight-thread form was faster at every n up to 1e5
// with many partial slots (17-32 % of a step at n = 2500-6000; 148 against
// 170 us at 1e5 with 196 slots).  With fewer than eight slots (the in-place
// symmetric kernels leave one) the other seven lanes would have nothing to
// load, so one thread per ion does it.  Both forms add the slots in the same
// order, so the choice never changes a result.
static bool epi_eight(int64_t n, int n_jc) {
  int tb = 0, tr = 0, tbps = 0;
  if (tuning_lookup(8, 0, n, &tb, &tr, &tbps)) return tr == 1;
  return n_jc >= 8;
}
static int epi_blocks(int64_t n, bool eight) { return blocks_for(eight ? 8 * n : n, EPI_THREADS); }

// ---------------------------------------------------------------------------
template <bool EIGHT>
__device__ __forceinline__ void epi_forces(const Phys &p, const StateView &s, const double *part,
                                           int n_jc, int flags, double t, unsigned *err) {
  int64_t i;
  double a[3];
  if (!epi_sums<EIGHT>(part, n_jc, s.n, i, a)) return;
  const double pref = coulomb_pref(p, s, i);
#pragma unroll
  for (int c = 0; c < 3; ++c) a[c] *= pref;
  if (flags & NB_ACC_TOTAL) {
    double tx, ty, tz;
    trap_accel(p, t, s.x[i], s.y[i], s.z[i], tx, ty, tz);
    const double ts = trap_scale(p, s, i);
    const double g = p.gamma / ion_mass(p, s, i);
    a[0] += ts * tx - g * s.vx[i];
    a[1] += ts * ty - g * s.vy[i];
    a[2] += ts * tz - g * s.vz[i];
  }
  s.ax[i] = a[0];
  s.ay[i] = a[1];
  s.az[i] = a[2];
  if (not_finite(a[0]) || not_finite(a[1]) || not_finite(a[2])) atomicOr(err, ERR_NONFINITE);
}
__global__ void __launch_bounds__(EPI_THREADS)
    k_epi_forces(Phys p, StateView s, const double *__restrict__ part, int n_jc, int flags, double t,
                 unsigned *err) {
  epi_forces<false>(p, s, part, n_jc, flags, t, err);
}
__global__ void __launch_bounds__(EPI_THREADS)
    k_epi_forces8(Phys p, StateView s, const double *__restrict__ part, int n_jc, int flags, double t,
                  unsigned *err) {
  epi_forces<true>(p, s, part, n_jc, flags, t, err);
}

cudaError_t launch_epi_forces(const Phys &p, const StateView &s, const double *part, int n_jc,
                              int flags, double t, unsigned *err, cudaStream_t st) {
  const bool eight = epi_eight(s.n, n_jc);
  if (eight)
    k_epi_forces8<<<epi_blocks(s.n, true), EPI_THREADS, 0, st>>>(p, s, part, n_jc, flags, t, err);
  else
    k_epi_forces<<<epi_blocks(s.n, false), EPI_THREADS, 0, st>>>(p, s, part, n_jc, flags, t, err);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
template <bool EIGHT>
__device__ __forceinline__ void epi_vjp(const Phys &p, const StateView &s, const double *part, int n_jc,
                                        const double *lx, const double *ly, const double *lz, double *gx,
                                        double *gy, double *gz, int flags, double t) {
  int64_t i;
  double g[3];
  if (!epi_sums<EIGHT>(part, n_jc, s.n, i, g)) return;
  const double pref = coulomb_pref(p, s, i);
#pragma unroll
  for (int c = 0; c < 3; ++c) g[c] *= pref;
  if (flags & NB_ACC_TOTAL) {
    double tx, ty, tz;  // the trap term is linear: its Jacobian applied to lambda
    trap_accel(p, t, lx[i], ly[i], lz[i], tx, ty, tz);
    const double ts = trap_scale(p, s, i);
    g[0] += ts * tx;
    g[1] += ts * ty;
    g[2] += ts * tz;
  }
  gx[i] = g[0];
  gy[i] = g[1];
  gz[i] = g[2];
}
__global__ void __launch_bounds__(EPI_THREADS)
    k_epi_vjp(Phys p, StateView s, const double *__restrict__ part, int n_jc, const double *__restrict__ lx,
              const double *__restrict__ ly, const double *__restrict__ lz, double *gx, double *gy,
              double *gz, int flags, double t) {
  epi_vjp<false>(p, s, part, n_jc, lx, ly, lz, gx, gy, gz, flags, t);
}
__global__ void __launch_bounds__(EPI_THREADS)
    k_epi_vjp8(Phys p, StateView s, const double *__restrict__ part, int n_jc, const double *__restrict__ lx,
               const double *__restrict__ ly, const double *__restrict__ lz, double *gx, double *gy,
               double *gz, int flags, double t) {
  epi_vjp<true>(p, s, part, n_jc, lx, ly, lz, gx, gy, gz, flags, t);
}

cudaError_t launch_epi_vjp(const Phys &p, const StateView &s, const double *part, int n_jc,
                           const double *lx, const double *ly, const double *lz, double *gx,
                           double *gy, double *gz, int flags, double t, cudaStream_t st) {
  if (epi_eight(s.n, n_jc))
    k_epi_vjp8<<<epi_blocks(s.n, true), EPI_THREADS, 0, st>>>(p, s, part, n_jc, lx, ly, lz, gx, gy, gz, flags, t);
  else
    k_epi_vjp<<<epi_blocks(s.n, false), EPI_THREADS, 0, st>>>(p, s, part, n_jc, lx, ly, lz, gx, gy, gz, flags, t);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// First drift of a run: r+ = r + v dt + a dt^2/2 into (px, py, pz), which may
// alias (x, y, z) (each thread touches only its own ion).
__global__ void k_drift(Phys p, StateView s, double *px, double *py, double *pz) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const double dt = p.dt;
  px[i] = verlet_drift(s.x[i], s.vx[i], s.ax[i], dt);
  py[i] = verlet_drift(s.y[i], s.vy[i], s.ay[i], dt);
  pz[i] = verlet_drift(s.z[i], s.vz[i], s.az[i], dt);
}

cudaError_t launch_drift(const Phys &p, const StateView &s, double *px, double *py, double *pz,
                         cudaStream_t st) {
  const int T = 256;
  k_drift<<<blocks_for(s.n, T), T, 0, st>>>(p, s, px, py, pz);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Verlet epilogue of one step, positions r+ = (cx, cy, cz) at time index snew:
//   a+_cons = Coulomb(r+) + trap(r+, t+)
//   v+ = (v + (a + a+_cons) dt/2) / (1 + gamma dt/(2m))  [+ Langevin kick]
//   a+ = a+_cons - (gamma/m) v+
// then either the next drift r++ = r+ + v+ dt + a+ dt^2/2 into (nx, ny, nz),
// or (last step) r+ copied to the state positions.
// The step index is snew = base + soff with base = *cin (a device counter) or
// 0 when cin is null; with cout non-null, thread 0 stores base + cout_off
// there.  The counter form lets one captured graph of steps be replayed with
// a step index that advances from replay to replay (cin and cout are never
// the same word, so no thread reads what another writes).
template <bool EIGHT>
__device__ __forceinline__ void epi_step(const Phys &p, const StateView &s, const double *cx,
                                         const double *cy, const double *cz, const double *part, int n_jc,
                                         int64_t soff, const int64_t *cin, int64_t *cout, int64_t cout_off,
                                         double *nx, double *ny, double *nz, unsigned *err) {
  int64_t i;
  double cs[3];
  if (!epi_sums<EIGHT>(part, n_jc, s.n, i, cs)) return;
  const int64_t base = cin ? *cin : 0;
  const int64_t snew = base + soff;
  if (cout && i == 0) *cout = base + cout_off;
  const double r[3] = {cx[i], cy[i], cz[i]};
  double v[3] = {s.vx[i], s.vy[i], s.vz[i]};
  double a[3] = {s.ax[i], s.ay[i], s.az[i]};
  const bool bad = verlet_kick(p, s, i, snew, r, cs, v, a);
  s.vx[i] = v[0]; s.vy[i] = v[1]; s.vz[i] = v[2];
  s.ax[i] = a[0]; s.ay[i] = a[1]; s.az[i] = a[2];
  if (nx) {
    nx[i] = verlet_drift(r[0], v[0], a[0], p.dt);
    ny[i] = verlet_drift(r[1], v[1], a[1], p.dt);
    nz[i] = verlet_drift(r[2], v[2], a[2], p.dt);
  } else {
    s.x[i] = r[0]; s.y[i] = r[1]; s.z[i] = r[2];
  }
  if (bad) atomicOr(err, ERR_NONFINITE);
}
__global__ void __launch_bounds__(EPI_THREADS)
    k_epi_step(Phys p, StateView s, const double *__restrict__ cx, const double *__restrict__ cy,
               const double *__restrict__ cz, const double *__restrict__ part, int n_jc, int64_t soff,
               const int64_t *cin, int64_t *cout, int64_t cout_off, double *nx, double *ny, double *nz,
               unsigned *err) {
  epi_step<false>(p, s, cx, cy, cz, part, n_jc, soff, cin, cout, cout_off, nx, ny, nz, err);
}
__global__ void __launch_bounds__(EPI_THREADS)
    k_epi_step8(Phys p, StateView s, const double *__restrict__ cx, const double *__restrict__ cy,
                const double *__restrict__ cz, const double *__restrict__ part, int n_jc, int64_t soff,
                const int64_t *cin, int64_t *cout, int64_t cout_off, double *nx, double *ny, double *nz,
                unsigned *err) {
  epi_step<true>(p, s, cx, cy, cz, part, n_jc, soff, cin, cout, cout_off, nx, ny, nz, err);
}

cudaError_t launch_epi_step(const Phys &p, const StateView &s, const double *cx, const double *cy,
                            const double *cz, const double *part, int n_jc, int64_t snew,
                            double *nx, double *ny, double *nz, unsigned *err, cudaStream_t st,
                            const int64_t *cin, int64_t *cout, int64_t cout_off) {
  if (epi_eight(s.n, n_jc))
    k_epi_step8<<<epi_blocks(s.n, true), EPI_THREADS, 0, st>>>(p, s, cx, cy, cz, part, n_jc, snew, cin, cout,
                                                                cout_off, nx, ny, nz, err);
  else
    k_epi_step<<<epi_blocks(s.n, false), EPI_THREADS, 0, st>>>(p, s, cx, cy, cz, part, n_jc, snew, cin, cout,
                                                                cout_off, nx, ny, nz, err);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Energies.  ENERGY_BLOCKS blocks stride over the ions in a fixed pattern
// and reduce in a fixed tree, so the result is bitwise reproducible.
__device__ __forceinline__ void block_reduce3(double v[3], double *sh) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int c = 0; c < 3; ++c) sh[c * ENERGY_THREADS + tid] = v[c];
  __syncthreads();
  for (int w = ENERGY_THREADS / 2; w > 0; w >>= 1) {
    if (tid < w)
#pragma unroll
      for (int c = 0; c < 3; ++c) sh[c * ENERGY_THREADS + tid] += sh[c * ENERGY_THREADS + tid + w];
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) v[c] = sh[c * ENERGY_THREADS];
}

__global__ void __launch_bounds__(ENERGY_THREADS) k_energy_part(Phys p, StateView s,
                                                                const double *__restrict__ phi,
                                                                int n_jc, double t,
                                                                double *block_part) {
  __shared__ double sh[3 * ENERGY_THREADS];
  double acc[3] = {0.0, 0.0, 0.0};
  double ctrap = 0.0, w2[3];
  for (int k = 0; k < 3; ++k) {
    const double w = p.omega[k] + p.omega_rate[k] * t;
    w2[k] = w * w;
  }
  if (p.trap == NB_TRAP_RF)
    ctrap = 0.5 * p.q_mathieu * p.omega_rf * p.omega_rf * cos(p.omega_rf * t + p.rf_phase);
  const int64_t stride = (int64_t)ENERGY_BLOCKS * ENERGY_THREADS;
  for (int64_t i = (int64_t)blockIdx.x * ENERGY_THREADS + threadIdx.x; i < s.n; i += stride) {
    const double vx = s.vx[i], vy = s.vy[i], vz = s.vz[i];
    const double x = s.x[i], y = s.y[i], z = s.z[i];
    const double mi = ion_mass(p, s, i), ts = trap_scale(p, s, i);
    acc[0] += 0.5 * mi * (vx * vx + vy * vy + vz * vz);
    if (p.trap == NB_TRAP_RF)
      acc[1] += 0.5 * mi * ts * (ctrap * (x * x - y * y) + w2[2] * z * z);
    else
      acc[1] += 0.5 * mi * ts * (w2[0] * x * x + w2[1] * y * y + w2[2] * z * z);
    const double qi = s.q ? s.q[i] : p.charge;
    const double qw = s.q ? qi : qi * p.charge;  // phi carries w_j = q_j or 1
    acc[2] += 0.5 * p.k_coulomb * qw * chunk_sum(phi, n_jc, 1, 0, s.n, i);
  }
  block_reduce3(acc, sh);
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; ++c) block_part[blockIdx.x * 3 + c] = acc[c];
}

__global__ void __launch_bounds__(ENERGY_THREADS) k_energy_final(const double *__restrict__ block_part,
                                                                 double *out4) {
  __shared__ double sh[3 * ENERGY_THREADS];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < ENERGY_BLOCKS; b += ENERGY_THREADS)
    for (int c = 0; c < 3; ++c) acc[c] += block_part[b * 3 + c];
  block_reduce3(acc, sh);
  if (threadIdx.x == 0) {
    out4[0] = acc[0];
    out4[1] = acc[1];
    out4[2] = acc[2];
    out4[3] = acc[0] + acc[1] + acc[2];
  }
}

cudaError_t launch_energy(const Phys &p, const StateView &s, const double *phi_part, int n_jc,
                          double t, double *block_part, double *out4, cudaStream_t st) {
  k_energy_part<<<ENERGY_BLOCKS, ENERGY_THREADS, 0, st>>>(p, s, phi_part, n_jc, t, block_part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_energy_final<<<1, ENERGY_THREADS, 0, st>>>(block_part, out4);
  return cudaGetLastError();
}

}  // namespace nb

namespace nb {

// out[i] = scale * sum over chunks of part[jc*n + i], in chunk order.
__global__ void k_chunk_sum1(int64_t n, const double *__restrict__ part, int n_jc, double scale,
                             double *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = scale * chunk_sum(part, n_jc, 1, 0, n, i);
}

cudaError_t launch_chunk_sum1(int64_t n, const double *part, int n_jc, double scale, double *out,
                              cudaStream_t st) {
  const int T = 256;
  k_chunk_sum1<<<blocks_for(n, T), T, 0, st>>>(n, part, n_jc, scale, out);
  return cudaGetLastError();
}

}  // namespace nb
