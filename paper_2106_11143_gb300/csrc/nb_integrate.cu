// nb_integrate.cu -- O(N) kernels of libnb.so: the epilogues that turn the
// pair partial sums into accelerations (Eq. 1), the velocity-Verlet kick and
// drift (Sec. II), the Langevin kick, and the energy reduction.
#include "nb_common.cuh"

namespace nb {

static int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

// Sum of the chunk partials of component c for ion i, in chunk order.
__device__ __forceinline__ double chunk_sum(const double *__restrict__ part, int n_jc, int ncomp,
                                           int c, int64_t n, int64_t i) {
  double s = 0.0;
  for (int jc = 0; jc < n_jc; ++jc) s += part[((int64_t)jc * ncomp + c) * n + i];
  return s;
}

// The three components of chunk_sum at once, each summed in the same
// ascending-chunk order (bitwise equal to three chunk_sum calls); eight chunks'
// loads are issued before their adds, so that a thread keeps 24 loads in
// flight over the symmetric plan's hundreds of slots.
__device__ __forceinline__ void chunk_sum3(const double *__restrict__ part, int n_jc, int64_t n,
                                           int64_t i, double out[3]) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  const int64_t stride = 3 * n;
  const double *p = part + i;
  int jc = 0;
  for (; jc + 8 <= n_jc; jc += 8, p += 8 * stride) {
    double v[8][3];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      v[u][0] = __ldcs(p + u * stride);
      v[u][1] = __ldcs(p + u * stride + n);
      v[u][2] = __ldcs(p + u * stride + 2 * n);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      s0 += v[u][0];
      s1 += v[u][1];
      s2 += v[u][2];
    }
  }
  for (; jc < n_jc; ++jc, p += stride) {
    s0 += p[0];
    s1 += p[n];
    s2 += p[2 * n];
  }
  out[0] = s0;
  out[1] = s1;
  out[2] = s2;
}

// Coulomb prefactor k_C q_i w / m_i, where the pair sums carry w_j = q_j when
// per-ion charges are given and w_j = 1 otherwise.
__device__ __forceinline__ double coulomb_pref(const Phys &p, const StateView &s, int64_t i) {
  const double m = ion_mass(p, s, i);
  return s.q ? p.k_coulomb * s.q[i] / m : p.k_coulomb * p.charge * p.charge / m;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) from its definition:
// ten rounds of two 32x32 -> 64-bit products with the multipliers
// 0xD2511F53 and 0xCD9E8D57, key bumped by 0x9E3779B9 / 0xBB67AE85.
__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// Three N(0,1) draws for (seed, instance, step, ion): Box-Muller on the four
// Philox words mapped to (0,1) as (k + 1/2) 2^-32.
__device__ __forceinline__ void normals3(unsigned long long seed, unsigned instance,
                                         int64_t step, int64_t ion, double out[3]) {
  uint32_t c[4] = {(uint32_t)ion, (uint32_t)((uint64_t)step & 0xffffffffu),
                   (uint32_t)((uint64_t)step >> 32), instance};
  philox(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
  const double s = 2.3283064365386963e-10;
  const double u0 = ((double)c[0] + 0.5) * s, u1 = ((double)c[1] + 0.5) * s;
  const double u2 = ((double)c[2] + 0.5) * s, u3 = ((double)c[3] + 0.5) * s;
  const double m0 = sqrt(-2.0 * log(u0)), m1 = sqrt(-2.0 * log(u2));
  double s1, c1, s3, c3;
  sincospi(2.0 * u1, &s1, &c1);
  sincospi(2.0 * u3, &s3, &c3);
  out[0] = m0 * c1;
  out[1] = m0 * s1;
  out[2] = m1 * c3;
}

// ---------------------------------------------------------------------------
__global__ void k_epi_forces(Phys p, StateView s, const double *__restrict__ part, int n_jc,
                             int flags, double t, unsigned *err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const double pref = coulomb_pref(p, s, i);
  double a[3];
  chunk_sum3(part, n_jc, s.n, i, a);
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

cudaError_t launch_epi_forces(const Phys &p, const StateView &s, const double *part, int n_jc,
                              int flags, double t, unsigned *err, cudaStream_t st) {
  const int T = 256;
  k_epi_forces<<<blocks_for(s.n, T), T, 0, st>>>(p, s, part, n_jc, flags, t, err);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__global__ void k_epi_vjp(Phys p, StateView s, const double *__restrict__ part, int n_jc,
                          const double *__restrict__ lx, const double *__restrict__ ly,
                          const double *__restrict__ lz, double *gx, double *gy, double *gz,
                          int flags, double t) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const double pref = coulomb_pref(p, s, i);
  double g[3];
  chunk_sum3(part, n_jc, s.n, i, g);
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

cudaError_t launch_epi_vjp(const Phys &p, const StateView &s, const double *part, int n_jc,
                           const double *lx, const double *ly, const double *lz, double *gx,
                           double *gy, double *gz, int flags, double t, cudaStream_t st) {
  const int T = 256;
  k_epi_vjp<<<blocks_for(s.n, T), T, 0, st>>>(p, s, part, n_jc, lx, ly, lz, gx, gy, gz, flags, t);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// First drift of a run: r+ = r + v dt + a dt^2/2 into (px, py, pz), which may
// alias (x, y, z) (each thread touches only its own ion).
__global__ void k_drift(Phys p, StateView s, double *px, double *py, double *pz) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const double dt = p.dt, h = 0.5 * dt * dt;
  px[i] = s.x[i] + s.vx[i] * dt + h * s.ax[i];
  py[i] = s.y[i] + s.vy[i] * dt + h * s.ay[i];
  pz[i] = s.z[i] + s.vz[i] * dt + h * s.az[i];
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
__global__ void k_epi_step(Phys p, StateView s, const double *__restrict__ cx,
                           const double *__restrict__ cy, const double *__restrict__ cz,
                           const double *__restrict__ part, int n_jc, int64_t snew, double *nx,
                           double *ny, double *nz, unsigned *err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const double dt = p.dt;
  const double t = p.t0 + (double)snew * dt;
  const double pref = coulomb_pref(p, s, i);
  const double r[3] = {cx[i], cy[i], cz[i]};
  double tr[3];
  trap_accel(p, t, r[0], r[1], r[2], tr[0], tr[1], tr[2]);
  const double ts = trap_scale(p, s, i);
  tr[0] *= ts;
  tr[1] *= ts;
  tr[2] *= ts;
  const double mi = ion_mass(p, s, i);
  const double c = p.gamma * dt / (2.0 * mi);
  const double g = p.gamma / mi;
  double xi[3] = {0.0, 0.0, 0.0};
  double sig = 0.0;
  if (p.noise_T > 0.0) {
    sig = sqrt(2.0 * p.gamma * KB * p.noise_T * dt) / mi;
    normals3(p.seed, p.instance, snew, i, xi);
  }
  double *vs[3] = {s.vx, s.vy, s.vz};
  double *as[3] = {s.ax, s.ay, s.az};
  double *ns[3] = {nx, ny, nz};
  double *xs[3] = {s.x, s.y, s.z};
  double cs[3];
  chunk_sum3(part, n_jc, s.n, i, cs);
  bool bad = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double ucons = pref * cs[k] + tr[k];
    double v = (vs[k][i] + 0.5 * dt * (as[k][i] + ucons)) / (1.0 + c);
    v += sig * xi[k];
    const double a = ucons - g * v;
    vs[k][i] = v;
    as[k][i] = a;
    if (nx)
      ns[k][i] = r[k] + v * dt + 0.5 * dt * dt * a;
    else
      xs[k][i] = r[k];
    bad |= not_finite(v) || not_finite(a);
  }
  if (bad) atomicOr(err, ERR_NONFINITE);
}

cudaError_t launch_epi_step(const Phys &p, const StateView &s, const double *cx, const double *cy,
                            const double *cz, const double *part, int n_jc, int64_t snew,
                            double *nx, double *ny, double *nz, unsigned *err, cudaStream_t st) {
  const int T = 256;
  k_epi_step<<<blocks_for(s.n, T), T, 0, st>>>(p, s, cx, cy, cz, part, n_jc, snew, nx, ny, nz, err);
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
