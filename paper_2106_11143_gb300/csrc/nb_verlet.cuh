// nb_verlet.cuh -- per-ion pieces of the velocity-Verlet step (Sec. II) shared
// by every kernel that advances ions: the Langevin normals (Philox4x32-10 and
// Box-Muller), the Coulomb prefactor, the drift and the kick.  The
// multi-kernel step (nb_integrate.cu), the single-block step (nb_small.cu)
// and the ensemble kernel (nb_batched.cu) all inline these same functions, so
// an ion given the same inputs gets the same bits on every path.
#pragma once

#include "nb_common.cuh"

namespace nb {

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

// Coulomb prefactor k_C q_i w / m_i, where the pair sums carry w_j = q_j when
// per-ion charges are given and w_j = 1 otherwise.
__device__ __forceinline__ double coulomb_pref(const Phys &p, const StateView &s, int64_t i) {
  const double m = ion_mass(p, s, i);
  return s.q ? p.k_coulomb * s.q[i] / m : p.k_coulomb * p.charge * p.charge / m;
}

// Sum of the n_jc chunk partials (x, y, z) of one ion, as eight interleaved
// running sums (chunk jc goes to sum jc mod 8) added pairwise at the end.
// The dependent chain is n_jc/8 + 3 FP64 adds instead of n_jc: at small n the
// latency of that chain, not the bandwidth, bounds the epilogue.  ld(jc, c)
// returns component c of chunk jc; the loads of eight chunks are issued
// before their adds.
template <class LD>
__device__ __forceinline__ void slot_sum3(int n_jc, LD ld, double out[3]) {
  double s[8][3];
#pragma unroll
  for (int u = 0; u < 8; ++u) s[u][0] = s[u][1] = s[u][2] = 0.0;
  int jc = 0;
  for (; jc + 8 <= n_jc; jc += 8) {
    double v[8][3];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      v[u][0] = ld(jc + u, 0);
      v[u][1] = ld(jc + u, 1);
      v[u][2] = ld(jc + u, 2);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      s[u][0] += v[u][0];
      s[u][1] += v[u][1];
      s[u][2] += v[u][2];
    }
  }
#pragma unroll
  for (int u = 0; u < 7; ++u)
    if (jc + u < n_jc) {
      s[u][0] += ld(jc + u, 0);
      s[u][1] += ld(jc + u, 1);
      s[u][2] += ld(jc + u, 2);
    }
#pragma unroll
  for (int c = 0; c < 3; ++c)
    out[c] = ((s[0][c] + s[1][c]) + (s[2][c] + s[3][c])) + ((s[4][c] + s[5][c]) + (s[6][c] + s[7][c]));
}

// Drift of one coordinate: r + v dt + a dt^2/2.
__device__ __forceinline__ double verlet_drift(double r, double v, double a, double dt) {
  return r + v * dt + 0.5 * dt * dt * a;
}

// The kick's per-ion constants, which depend only on the ion and the
// parameters: the Coulomb prefactor, the trap scale of its species, the
// friction factors 1 / (1 + gamma dt/(2 m_i)) and gamma/m_i, and the Langevin
// amplitude.  Several are FP64 divisions, long dependent chains on GB300, so a
// kernel that kicks the same ion many times forms them once; the values are
// the same wherever they are formed.
struct KickConst {
  double pref, ts, inv, g, sig;
};
__device__ __forceinline__ KickConst kick_consts(const Phys &p, const StateView &s, int64_t i) {
  KickConst k;
  k.pref = coulomb_pref(p, s, i);
  k.ts = trap_scale(p, s, i);
  const double mi = ion_mass(p, s, i);
  k.inv = 1.0 / (1.0 + p.gamma * p.dt / (2.0 * mi));
  k.g = p.gamma / mi;
  k.sig = p.noise_T > 0.0 ? sqrt(2.0 * p.gamma * KB * p.noise_T * p.dt) / mi : 0.0;
  return k;
}

// Kick of ion i at positions r (step index snew, time t0 + snew dt), given
// its pair sum cs = sum_j w_j (r_i - r_j) / s_ij^3 and its constants kc:
//   a+_cons = k_C q_i/m_i cs + trap(r, t)   (Eq. 1)
//   v+ = (v + (a + a+_cons) dt/2) * [1 / (1 + gamma dt/(2 m_i))]  [+ Langevin kick]
//   a+ = a+_cons - (gamma/m_i) v+
// v and a hold the ion's velocity and acceleration on entry and the new ones
// on return.  Returns true if any of them is not finite.
__device__ __forceinline__ bool verlet_kick_k(const Phys &p, const KickConst &kc, int64_t i,
                                              int64_t snew, const double r[3], const double cs[3],
                                              double v[3], double a[3]) {
  const double dt = p.dt;
  const double t = p.t0 + (double)snew * dt;
  double tr[3];
  trap_accel(p, t, r[0], r[1], r[2], tr[0], tr[1], tr[2]);
  tr[0] *= kc.ts;
  tr[1] *= kc.ts;
  tr[2] *= kc.ts;
  double xi[3] = {0.0, 0.0, 0.0};
  if (p.noise_T > 0.0) normals3(p.seed, p.instance, snew, i, xi);
  bool bad = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double ucons = kc.pref * cs[k] + tr[k];
    double vn = (v[k] + 0.5 * dt * (a[k] + ucons)) * kc.inv;
    vn += kc.sig * xi[k];
    const double an = ucons - kc.g * vn;
    v[k] = vn;
    a[k] = an;
    bad |= not_finite(vn) || not_finite(an);
  }
  return bad;
}

// The kick with its constants formed on the spot; ion i of the view is ion
// s.ion0 + i of the system, which keys its Langevin draws.
__device__ __forceinline__ bool verlet_kick(const Phys &p, const StateView &s, int64_t i,
                                            int64_t snew, const double r[3], const double cs[3],
                                            double v[3], double a[3]) {
  return verlet_kick_k(p, kick_consts(p, s, i), s.ion0 + i, snew, r, cs, v, a);
}

}  // namespace nb
