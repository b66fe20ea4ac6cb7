/*
 * nb_oracle.c -- plain, slow, obviously correct FP64 CPU oracle for the
 * trapped-ion direct N-body method of Pedregosa-Gutierrez & Dempsey,
 * "Direct N-Body problem optimisation using the AVX-512 instruction set"
 * (arXiv 2106.11143).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, constant
 * table or helper with the CUDA library.
 *
 * What it computes, and where the paper defines it:
 *   - Coulomb acceleration: Eq. 1 (Sec. II), the sum over j != i of
 *     Q^2 k_C / m * (r_i - r_j) / |r_i - r_j|^3, evaluated exactly as the
 *     Sec. III double loop does (1/sqrt(r^2 + softening), cubed), with the
 *     self pair excluded and the softening added to r^2.  Per-particle
 *     charges q_j generalise the single-species Q (Sec. II).
 *     Each component is summed in j order with Neumaier compensation so the
 *     result is close to correctly rounded regardless of summation order.
 *   - Trap force: Eq. 1.  Static harmonic -omega_k^2 x_k, or the linear RF
 *     trap written with the Mathieu q (a = 0): a_x = -(q Omega^2/2) cos(Omega t
 *     + phase) x, a_y = +(q Omega^2/2) cos(...) y, a_z = -omega_z^2 z.
 *   - Friction: Eq. 1, -(Gamma/m) v.
 *   - Velocity Verlet with constant dt: Sec. II (position update, new
 *     acceleration, velocity update with the mean of old and new
 *     acceleration).  The friction term makes the new acceleration depend on
 *     the new velocity; the velocity update is solved for it in closed form.
 *   - Energies (kinetic, trap, Coulomb) and the adjoint (reverse-mode
 *     derivative) of the Verlet trajectory: not in the paper; plain
 *     definitions written out.
 *   - Langevin noise: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
 *     written from its published definition, plus the Box-Muller transform.
 *
 * Compile: gcc -std=c11 -O2 -ffp-contract=off -fopenmp -shared -fPIC.
 * No -ffast-math: IEEE semantics are part of the definition.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CODATA 2018 exact Boltzmann constant (J/K). */
static const double OR_KB = 1.380649e-23;
static const double OR_PI = 3.14159265358979323846;

typedef struct {
  double k_coulomb;  /* 1/(4 pi eps0) */
  double mass;       /* kg */
  double charge;     /* C, used when the per-particle charge array is NULL */
  double soft2;      /* softening added to r^2 (m^2) */
  int32_t trap;      /* 0 = static harmonic, 1 = linear RF trap */
  int32_t pad0;
  double omega[3];   /* rad/s; in RF mode only omega[2] (axial) is used */
  double omega_rate[3]; /* rad/s^2: omega_k(t) = omega[k] + omega_rate[k] t */
  double q_mathieu;  /* RF Mathieu q */
  double omega_rf;   /* RF angular frequency (rad/s) */
  double rf_phase;   /* rad */
  double gamma;      /* friction coefficient (kg/s) */
  double dt;         /* s */
  double t0;         /* time of step 0 (s): t = t0 + step*dt */
  double noise_T;    /* Langevin temperature (K); 0 disables the noise */
  uint64_t seed;     /* Philox key */
  uint32_t instance; /* ensemble member index, part of the Philox counter */
  uint32_t pad1;
} or_params;

/* ------------------------------------------------------------------ */
/* Neumaier (improved Kahan-Babuska) compensated summation.            */
typedef struct { double s, c; } or_sum;
static void or_add(or_sum *a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}
static double or_val(or_sum a) { return a.s + a.c; }

void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
int or_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static double or_charge(const or_params *p, const double *q, int64_t i) {
  return q ? q[i] : p->charge;
}

/* Per-ion mass for two-species systems (Sec. II: two species interact as
 * three N-body problems, 1-1, 2-2 and 1-2; with a per-ion charge and mass the
 * single all-pairs sum covers all three).  NULL = params mass for all.     */
static const double *g_mass = NULL;
void or_set_masses(const double *m) { g_mass = m; }
static double or_mass(const or_params *p, int64_t i) { return g_mass ? g_mass[i] : p->mass; }

/* The trap's electric field is fixed, so an ion's trap acceleration scales
 * with its charge-to-mass ratio relative to the reference species that the
 * trap parameters describe (params charge and mass).                      */
static double or_trap_scale(const or_params *p, const double *q, int64_t i) {
  return (or_charge(p, q, i) / or_mass(p, i)) / (p->charge / p->mass);
}

/* ------------------------------------------------------------------ */
/* Coulomb acceleration of every particle in [i0, i1) from all n.
 * ax/ay/az receive k_C q_i/m * sum_{j != i} q_j d_ij / s_ij^3 with
 * d_ij = r_i - r_j and s_ij^2 = |d_ij|^2 + soft2 (Sec. III listing, Eq. 1).
 * phi (nullable) receives sum_{j != i} q_j / s_ij (no k_C factor).
 * absf (nullable) receives the conditioning sum k_C |q_i|/m *
 * sum_{j != i} |q_j| |d_ij| / s_ij^3 (the magnitudes of the pair terms).
 * reverse != 0 sums j in descending order (used to measure how much two
 * correct summation orders differ).                                      */
void or_coulomb_range(const or_params *p, int64_t n, int64_t i0, int64_t i1,
                      const double *x, const double *y, const double *z,
                      const double *q, double *ax, double *ay, double *az,
                      double *phi, double *absf, int reverse) {
  int64_t i;
#pragma omp parallel for schedule(static)
  for (i = i0; i < i1; i++) {
    or_sum sx = {0, 0}, sy = {0, 0}, sz = {0, 0}, sp = {0, 0}, sa = {0, 0};
    for (int64_t jj = 0; jj < n; jj++) {
      int64_t j = reverse ? (n - 1 - jj) : jj;
      if (j == i) continue; /* the self pair carries no force */
      double dx = x[i] - x[j];
      double dy = y[i] - y[j];
      double dz = z[i] - z[j];
      double r2 = dx * dx + dy * dy + dz * dz + p->soft2;
      double inv = 1.0 / sqrt(r2);
      double inv3 = inv * inv * inv;
      double qj = or_charge(p, q, j);
      double s = qj * inv3;
      or_add(&sx, dx * s);
      or_add(&sy, dy * s);
      or_add(&sz, dz * s);
      if (phi) or_add(&sp, qj * inv);
      if (absf) or_add(&sa, fabs(qj) * sqrt(dx * dx + dy * dy + dz * dz) * inv3);
    }
    double qi = or_charge(p, q, i);
    double pref = p->k_coulomb * qi / or_mass(p, i);
    ax[i - i0] = pref * or_val(sx);
    ay[i - i0] = pref * or_val(sy);
    az[i - i0] = pref * or_val(sz);
    if (phi) phi[i - i0] = or_val(sp);
    if (absf) absf[i - i0] = fabs(pref) * or_val(sa);
  }
}

void or_coulomb(const or_params *p, int64_t n, const double *x, const double *y,
                const double *z, const double *q, double *ax, double *ay,
                double *az, double *phi, double *absf, int reverse) {
  or_coulomb_range(p, n, 0, n, x, y, z, q, ax, ay, az, phi, absf, reverse);
}

/* ------------------------------------------------------------------ */
/* Trap acceleration at time t (Eq. 1).                                  */
static double or_omega(const or_params *p, int k, double t) {
  return p->omega[k] + p->omega_rate[k] * t;
}

static void or_trap_one(const or_params *p, double t, double x, double y,
                        double z, double *tx, double *ty, double *tz) {
  if (p->trap == 1) {
    double c = 0.5 * p->q_mathieu * p->omega_rf * p->omega_rf *
               cos(p->omega_rf * t + p->rf_phase);
    double wz = or_omega(p, 2, t);
    *tx = -c * x;
    *ty = c * y;
    *tz = -wz * wz * z;
  } else {
    double wx = or_omega(p, 0, t), wy = or_omega(p, 1, t), wz = or_omega(p, 2, t);
    *tx = -wx * wx * x;
    *ty = -wy * wy * y;
    *tz = -wz * wz * z;
  }
}

void or_trap(const or_params *p, double t, int64_t n, const double *x,
             const double *y, const double *z, double *ax, double *ay,
             double *az) {
  for (int64_t i = 0; i < n; i++) or_trap_one(p, t, x[i], y[i], z[i], &ax[i], &ay[i], &az[i]);
}

/* Total acceleration used as the Verlet state: Coulomb + trap(t) -
 * (gamma/m) v (Eq. 1).  v may be NULL (treated as zero).                */
void or_accel(const or_params *p, double t, int64_t n, const double *x,
              const double *y, const double *z, const double *vx,
              const double *vy, const double *vz, const double *q, double *ax,
              double *ay, double *az, int reverse) {
  or_coulomb(p, n, x, y, z, q, ax, ay, az, NULL, NULL, reverse);
  for (int64_t i = 0; i < n; i++) {
    double tx, ty, tz;
    double g = p->gamma / or_mass(p, i);
    double ts = or_trap_scale(p, q, i);
    or_trap_one(p, t, x[i], y[i], z[i], &tx, &ty, &tz);
    ax[i] += ts * tx;
    ay[i] += ts * ty;
    az[i] += ts * tz;
    if (vx) {
      ax[i] -= g * vx[i];
      ay[i] -= g * vy[i];
      az[i] -= g * vz[i];
    }
  }
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64
 * multiplications by M0 = 0xD2511F53 and M1 = 0xCD9E8D57, with the key
 * bumped by the Weyl constants W0 = 0x9E3779B9, W1 = 0xBB67AE85 between
 * rounds.                                                                */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                      uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; r++) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    if (r < 9) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Three standard normals for (seed, instance, step, ion) via Box-Muller on
 * the four Philox words mapped to (0,1) as (k + 0.5) 2^-32.  Counter layout:
 * {ion, step low word, step high word, instance}; key = seed words.       */
void or_normals3(uint64_t seed, uint32_t instance, int64_t step, int64_t ion,
                 double out[3]) {
  uint32_t ctr[4] = {(uint32_t)ion, (uint32_t)((uint64_t)step & 0xffffffffu),
                     (uint32_t)((uint64_t)step >> 32), instance};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t r[4];
  or_philox4x32_10(ctr, key, r);
  const double s = 2.3283064365386963e-10; /* 2^-32 */
  double u0 = ((double)r[0] + 0.5) * s, u1 = ((double)r[1] + 0.5) * s;
  double u2 = ((double)r[2] + 0.5) * s, u3 = ((double)r[3] + 0.5) * s;
  double m0 = sqrt(-2.0 * log(u0)), m1 = sqrt(-2.0 * log(u2));
  out[0] = m0 * cos(2.0 * OR_PI * u1);
  out[1] = m0 * sin(2.0 * OR_PI * u1);
  out[2] = m1 * cos(2.0 * OR_PI * u3);
}

/* ------------------------------------------------------------------ */
/* Velocity Verlet (Sec. II) for nsteps steps.  State on entry: positions,
 * velocities and the total acceleration a(t) at t = t0 + step*dt.
 *   r+ = r + v dt + (dt^2/2) a
 *   a+ = a_coulomb(r+) + a_trap(r+, t+dt) - (gamma/m) v+
 *   v+ = v + (dt/2)(a + a+)
 * The last line contains v+ on both sides through the friction term; with
 * c = gamma dt / (2m) it is solved as v+ = (v + (dt/2)(a + a+_cons))/(1+c),
 * a+_cons being a+ without friction.  With noise_T > 0 a Langevin kick
 * sqrt(2 gamma kB T dt)/m * xi is added to v+ afterwards, xi ~ N(0,1) per
 * component from or_normals3 with the step index of the new state.
 * `step` is advanced by nsteps.                                            */
int or_run(const or_params *p, int64_t n, const double *q, double *x, double *y,
           double *z, double *vx, double *vy, double *vz, double *ax,
           double *ay, double *az, int64_t *step, int64_t nsteps, int reverse) {
  double dt = p->dt;
  double *cx = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  if (!cx) return 1;
  double *cy = cx + n, *cz = cy + n;
  for (int64_t s = 0; s < nsteps; s++) {
    int64_t snew = *step + 1;
    double tnew = p->t0 + (double)snew * dt;
    for (int64_t i = 0; i < n; i++) {
      x[i] = x[i] + vx[i] * dt + 0.5 * dt * dt * ax[i];
      y[i] = y[i] + vy[i] * dt + 0.5 * dt * dt * ay[i];
      z[i] = z[i] + vz[i] * dt + 0.5 * dt * dt * az[i];
    }
    or_coulomb(p, n, x, y, z, q, cx, cy, cz, NULL, NULL, reverse);
    for (int64_t i = 0; i < n; i++) {
      double tx, ty, tz;
      double mi = or_mass(p, i), ts = or_trap_scale(p, q, i);
      double c = p->gamma * dt / (2.0 * mi);
      double g = p->gamma / mi;
      double sig = 0.0;
      if (p->noise_T > 0.0) sig = sqrt(2.0 * p->gamma * OR_KB * p->noise_T * dt) / mi;
      or_trap_one(p, tnew, x[i], y[i], z[i], &tx, &ty, &tz);
      double ux = cx[i] + ts * tx, uy = cy[i] + ts * ty, uz = cz[i] + ts * tz;
      double nvx = (vx[i] + 0.5 * dt * (ax[i] + ux)) / (1.0 + c);
      double nvy = (vy[i] + 0.5 * dt * (ay[i] + uy)) / (1.0 + c);
      double nvz = (vz[i] + 0.5 * dt * (az[i] + uz)) / (1.0 + c);
      if (sig > 0.0) {
        double xi[3];
        or_normals3(p->seed, p->instance, snew, i, xi);
        nvx += sig * xi[0];
        nvy += sig * xi[1];
        nvz += sig * xi[2];
      }
      vx[i] = nvx; vy[i] = nvy; vz[i] = nvz;
      ax[i] = ux - g * nvx;
      ay[i] = uy - g * nvy;
      az[i] = uz - g * nvz;
    }
    *step = snew;
  }
  free(cx);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Energies at time t = t0 + step*dt: out = {kinetic, trap, Coulomb, total}.
 * kinetic = (m/2) sum v^2; trap = the potential whose negative gradient
 * (per unit mass) is the Eq. 1 trap term; Coulomb = (k_C/2) sum_i q_i phi_i. */
void or_energy(const or_params *p, int64_t step, int64_t n, const double *x,
               const double *y, const double *z, const double *vx,
               const double *vy, const double *vz, const double *q,
               double out[4]) {
  double t = p->t0 + (double)step * p->dt;
  or_sum ke = {0, 0}, tp = {0, 0}, cp = {0, 0};
  double *phi = (double *)malloc(sizeof(double) * 4 * (size_t)(n > 0 ? n : 1));
  double *t1 = phi + n, *t2 = t1 + n, *t3 = t2 + n;
  or_coulomb(p, n, x, y, z, q, t1, t2, t3, phi, NULL, 0);
  for (int64_t i = 0; i < n; i++) {
    double mi = or_mass(p, i), ts = or_trap_scale(p, q, i);
    or_add(&ke, 0.5 * mi * (vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i]));
    if (p->trap == 1) {
      double c = 0.5 * p->q_mathieu * p->omega_rf * p->omega_rf *
                 cos(p->omega_rf * t + p->rf_phase);
      double wz = or_omega(p, 2, t);
      or_add(&tp, 0.5 * mi * ts * (c * (x[i] * x[i] - y[i] * y[i]) + wz * wz * z[i] * z[i]));
    } else {
      double wx = or_omega(p, 0, t), wy = or_omega(p, 1, t), wz = or_omega(p, 2, t);
      or_add(&tp, 0.5 * mi * ts *
                      (wx * wx * x[i] * x[i] + wy * wy * y[i] * y[i] + wz * wz * z[i] * z[i]));
    }
    or_add(&cp, 0.5 * p->k_coulomb * or_charge(p, q, i) * phi[i]);
  }
  out[0] = or_val(ke);
  out[1] = or_val(tp);
  out[2] = or_val(cp);
  out[3] = out[0] + out[1] + out[2];
  free(phi);
}

/* ------------------------------------------------------------------ */
/* Vector-Jacobian product of the position-dependent acceleration.
 * With f(d) = d / s^3, s^2 = |d|^2 + soft2, the Jacobian block is
 * M(d) = I/s^3 - 3 d d^T / s^5 (symmetric, even in d), so
 *   (J^T lam)_i = k_C q_i/m sum_{j != i} q_j M(d_ij)(lam_i - lam_j)
 * plus, when include_trap is set, the trap's diagonal term at time t.   */
void or_forces_vjp(const or_params *p, double t, int64_t n, const double *x,
                   const double *y, const double *z, const double *q,
                   const double *lx, const double *ly, const double *lz,
                   double *gx, double *gy, double *gz, int include_trap) {
  int64_t i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < n; i++) {
    or_sum sx = {0, 0}, sy = {0, 0}, sz = {0, 0};
    for (int64_t j = 0; j < n; j++) {
      if (j == i) continue;
      double dx = x[i] - x[j], dy = y[i] - y[j], dz = z[i] - z[j];
      double r2 = dx * dx + dy * dy + dz * dz + p->soft2;
      double inv = 1.0 / sqrt(r2);
      double inv3 = inv * inv * inv;
      double inv5 = inv3 * inv * inv;
      double ex = lx[i] - lx[j], ey = ly[i] - ly[j], ez = lz[i] - lz[j];
      double dot = dx * ex + dy * ey + dz * ez;
      double qj = or_charge(p, q, j);
      or_add(&sx, qj * (ex * inv3 - 3.0 * dx * dot * inv5));
      or_add(&sy, qj * (ey * inv3 - 3.0 * dy * dot * inv5));
      or_add(&sz, qj * (ez * inv3 - 3.0 * dz * dot * inv5));
    }
    double pref = p->k_coulomb * or_charge(p, q, i) / or_mass(p, i);
    double ts = or_trap_scale(p, q, i);
    gx[i] = pref * or_val(sx);
    gy[i] = pref * or_val(sy);
    gz[i] = pref * or_val(sz);
    if (include_trap) {
      double tx0 = gx[i], ty0 = gy[i], tz0 = gz[i];
      if (p->trap == 1) {
        double c = 0.5 * p->q_mathieu * p->omega_rf * p->omega_rf *
                   cos(p->omega_rf * t + p->rf_phase);
        double wz = or_omega(p, 2, t);
        gx[i] = tx0 + ts * (-c * lx[i]);
        gy[i] = ty0 + ts * (c * ly[i]);
        gz[i] = tz0 + ts * (-wz * wz * lz[i]);
      } else {
        double wx = or_omega(p, 0, t), wy = or_omega(p, 1, t), wz = or_omega(p, 2, t);
        gx[i] = tx0 + ts * (-wx * wx * lx[i]);
        gy[i] = ty0 + ts * (-wy * wy * ly[i]);
        gz[i] = tz0 + ts * (-wz * wz * lz[i]);
      }
    }
  }
}

/* ------------------------------------------------------------------ */
/* Loss and gradient of a velocity-Verlet trajectory (static harmonic trap,
 * no friction, no noise).  Forward: a_0 = A(x_0), then nsteps Verlet steps.
 * Loss L = E_coulomb(x_T) + E_trap(x_T) + sum_i |x_T,i - target_i|^2.
 * Reverse sweep, for n = T-1 .. 0 with carried cotangents (xb, vb, ab):
 *   ab_{n+1} += dt/2 vb_{n+1}
 *   xb_{n+1} += J(x_{n+1})^T ab_{n+1};  wb_k += sum_i ab_{n+1,i,k} (-2 w_k x_{n+1,i,k})
 *   vb_n = vb_{n+1} + dt xb_{n+1};  ab_n = dt/2 vb_{n+1} + dt^2/2 xb_{n+1};
 *   xb_n = xb_{n+1}
 * and finally xb_0 += J(x_0)^T ab_0 with the matching omega term.
 * Every state is stored (plain, memory-hungry, fine for an oracle).
 * grad_x0, grad_v0: 3n each, SoA (x block, y block, z block).  Returns 0
 * on success, 2 on unsupported parameters, 1 on allocation failure.       */
int or_trajectory_grad(const or_params *p, int64_t n, const double *q,
                       const double *x0, const double *v0, int64_t nsteps,
                       const double *target, double *loss, double *grad_x0,
                       double *grad_v0, double grad_omega[3]) {
  if (g_mass || p->trap != 0 || p->gamma != 0.0 || p->noise_T != 0.0 ||
      p->omega_rate[0] != 0.0 || p->omega_rate[1] != 0.0 || p->omega_rate[2] != 0.0)
    return 2;
  size_t N3 = 3 * (size_t)n;
  double *X = (double *)malloc(sizeof(double) * N3 * (size_t)(nsteps + 1));
  double *v = (double *)malloc(sizeof(double) * N3);
  double *a = (double *)malloc(sizeof(double) * N3);
  double *xb = (double *)malloc(sizeof(double) * N3);
  double *vb = (double *)malloc(sizeof(double) * N3);
  double *ab = (double *)malloc(sizeof(double) * N3);
  double *g = (double *)malloc(sizeof(double) * N3);
  if (!X || !v || !a || !xb || !vb || !ab || !g) return 1;
  double dt = p->dt;
  memcpy(X, x0, sizeof(double) * N3);
  memcpy(v, v0, sizeof(double) * N3);
  /* forward */
  or_accel(p, p->t0, n, X, X + n, X + 2 * n, NULL, NULL, NULL, q, a, a + n, a + 2 * n, 0);
  for (int64_t s = 0; s < nsteps; s++) {
    double *xc = X + N3 * (size_t)s, *xn = X + N3 * (size_t)(s + 1);
    for (size_t k = 0; k < N3; k++) xn[k] = xc[k] + v[k] * dt + 0.5 * dt * dt * a[k];
    double *an = g; /* reuse as scratch */
    or_accel(p, p->t0, n, xn, xn + n, xn + 2 * n, NULL, NULL, NULL, q, an, an + n, an + 2 * n, 0);
    for (size_t k = 0; k < N3; k++) {
      v[k] = v[k] + 0.5 * dt * (a[k] + an[k]);
      a[k] = an[k];
    }
  }
  double *xT = X + N3 * (size_t)nsteps;
  /* loss and its gradient at x_T:  dL/dx = -m A(x_T) + 2 (x_T - target) */
  double e[4];
  or_energy(p, 0, n, xT, xT + n, xT + 2 * n, v, v + n, v + 2 * n, q, e);
  or_sum ls = {0, 0};
  or_add(&ls, e[1]);
  or_add(&ls, e[2]);
  for (size_t k = 0; k < N3; k++) {
    double d = xT[k] - target[k];
    or_add(&ls, d * d);
    xb[k] = -p->mass * a[k] + 2.0 * d;
    vb[k] = 0.0;
    ab[k] = 0.0;
  }
  *loss = or_val(ls);
  double wb[3];
  for (int k = 0; k < 3; k++) {
    or_sum s = {0, 0};
    for (int64_t i = 0; i < n; i++) or_add(&s, p->mass * p->omega[k] * xT[(size_t)k * n + i] * xT[(size_t)k * n + i]);
    wb[k] = or_val(s);
  }
  /* reverse sweep */
  for (int64_t s = nsteps - 1; s >= -1; s--) {
    double *xn = X + N3 * (size_t)(s + 1);
    if (s >= 0)
      for (size_t k = 0; k < N3; k++) ab[k] += 0.5 * dt * vb[k];
    or_forces_vjp(p, p->t0, n, xn, xn + n, xn + 2 * n, q, ab, ab + n, ab + 2 * n, g, g + n, g + 2 * n, 1);
    for (int k = 0; k < 3; k++) {
      or_sum sw = {0, 0};
      for (int64_t i = 0; i < n; i++)
        or_add(&sw, ab[(size_t)k * n + i] * (-2.0 * p->omega[k] * xn[(size_t)k * n + i]));
      wb[k] += or_val(sw);
    }
    for (size_t k = 0; k < N3; k++) xb[k] += g[k];
    if (s < 0) break;
    for (size_t k = 0; k < N3; k++) {
      double vbn = vb[k] + dt * xb[k];
      ab[k] = 0.5 * dt * vb[k] + 0.5 * dt * dt * xb[k];
      vb[k] = vbn;
    }
  }
  memcpy(grad_x0, xb, sizeof(double) * N3);
  memcpy(grad_v0, vb, sizeof(double) * N3);
  for (int k = 0; k < 3; k++) grad_omega[k] = wb[k];
  free(X); free(v); free(a); free(xb); free(vb); free(ab); free(g);
  return 0;
}
