// nb_adjoint.cu -- loss of a velocity-Verlet trajectory and its gradient by
// the discrete adjoint (reverse sweep) of the Sec. II integrator, with
// checkpoints every K steps and recomputation in between.
//
// Forward (Sec. II, Eq. 1 with a static harmonic trap, no friction or noise):
//   a_0 = A(x_0);  x_{n+1} = x_n + dt v_n + dt^2/2 a_n;  a_{n+1} = A(x_{n+1});
//   v_{n+1} = v_n + dt/2 (a_n + a_{n+1}).
// Loss L = E_coulomb(x_T) + E_trap(x_T) + sum_i |x_T,i - target_i|^2.
// Reverse sweep with cotangents (xb, vb, ab), n = T-1 .. 0:
//   ab_{n+1} += dt/2 vb_{n+1}
//   xb_{n+1} += J(x_{n+1})^T ab_{n+1};   wb_k += sum_i ab_{n+1,i,k} (-2 w_k x_{n+1,i,k})
//   vb_n = vb_{n+1} + dt xb_{n+1};  ab_n = dt/2 vb_{n+1} + dt^2/2 xb_{n+1};  xb_n = xb_{n+1}
// and finally xb_0 += J(x_0)^T ab_0 with its omega term.  The first line of
// each iteration is fused into the epilogue of the previous one.  J^T ab is
// the pair VJP kernel plus the diagonal trap term.  The omega terms are
// accumulated per ion and reduced once at the end (deterministic).
#include "nb_common.cuh"

namespace nb {

static int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

__device__ __forceinline__ double pref_of(const Phys &p, const double *q, int64_t i) {
  return q ? p.k_coulomb * q[i] / p.mass : p.k_coulomb * p.charge * p.charge / p.mass;
}

__device__ __forceinline__ double csum(const double *__restrict__ part, int n_jc, int c, int64_t n,
                                       int64_t i) {
  double s = 0.0;
  for (int jc = 0; jc < n_jc; ++jc) s += part[((int64_t)jc * 3 + c) * n + i];
  return s;
}

struct Vec3 {
  double *x, *y, *z;
};
struct CVec3 {
  const double *x, *y, *z;
};

// Gradient of the loss at x_T:  xb = -m a_T + 2 (x_T - target)  (a_T is the
// total acceleration, i.e. minus the gradient of the potential over m);
// vb = ab = 0;  wacc_{i,k} = m w_k x_{T,i,k}^2 (direct omega dependence of E_trap).
__global__ void k_adj_init(Phys p, int64_t n, CVec3 xT, CVec3 aT, CVec3 tgt, Vec3 xb, Vec3 vb,
                           Vec3 ab, Vec3 wacc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double *xs[3] = {xT.x, xT.y, xT.z}, *as[3] = {aT.x, aT.y, aT.z}, *ts[3] = {tgt.x, tgt.y, tgt.z};
  double *xbs[3] = {xb.x, xb.y, xb.z}, *vbs[3] = {vb.x, vb.y, vb.z}, *abs_[3] = {ab.x, ab.y, ab.z};
  double *ws[3] = {wacc.x, wacc.y, wacc.z};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double x = xs[k][i];
    xbs[k][i] = -p.mass * as[k][i] + 2.0 * (x - ts[k][i]);
    vbs[k][i] = 0.0;
    abs_[k][i] = 0.0;
    ws[k][i] = p.mass * p.omega[k] * x * x;
  }
}

// One reverse step at positions x = x_{n+1} with lambda = ab (read in place):
//   g = J^T ab;  xb += g;  wacc += ab (-2 w x);
// and unless `last`:  vb' = vb + dt xb;  ab = dt/2 vb + dt^2/2 xb (+ dt/2 vb'
// when `more`, the next iteration's first line);  vb = vb'.
__global__ void k_adj_epi(Phys p, int64_t n, const double *q, CVec3 x,
                          const double *__restrict__ part, int n_jc, Vec3 xb, Vec3 vb, Vec3 ab,
                          Vec3 wacc, int last, int more) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double pref = pref_of(p, q, i);
  const double dt = p.dt;
  const double *xs[3] = {x.x, x.y, x.z};
  double *xbs[3] = {xb.x, xb.y, xb.z}, *vbs[3] = {vb.x, vb.y, vb.z}, *abs_[3] = {ab.x, ab.y, ab.z};
  double *ws[3] = {wacc.x, wacc.y, wacc.z};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double lam = abs_[k][i];
    const double w2 = p.omega[k] * p.omega[k];
    const double g = pref * csum(part, n_jc, k, n, i) - w2 * lam;
    const double xbn = xbs[k][i] + g;
    ws[k][i] += lam * (-2.0 * p.omega[k] * xs[k][i]);
    xbs[k][i] = xbn;
    if (!last) {
      const double vbo = vbs[k][i];
      const double vbn = vbo + dt * xbn;
      double a = 0.5 * dt * vbo + 0.5 * dt * dt * xbn;
      if (more) a += 0.5 * dt * vbn;
      abs_[k][i] = a;
      vbs[k][i] = vbn;
    }
  }
}

// Outputs: gx0 = s xb, gv0 = s vb, and per-block partial sums of wacc.
constexpr int ADJ_BLOCKS = 128;
constexpr int ADJ_THREADS = 256;

__global__ void __launch_bounds__(ADJ_THREADS) k_adj_out(int64_t n, CVec3 xb, CVec3 vb, CVec3 wacc,
                                                         const double *gscale, Vec3 gx, Vec3 gv,
                                                         double *bpart) {
  __shared__ double sh[3 * ADJ_THREADS];
  const double s = gscale ? *gscale : 1.0;
  double acc[3] = {0.0, 0.0, 0.0};
  const int64_t stride = (int64_t)ADJ_BLOCKS * ADJ_THREADS;
  for (int64_t i = (int64_t)blockIdx.x * ADJ_THREADS + threadIdx.x; i < n; i += stride) {
    gx.x[i] = s * xb.x[i]; gx.y[i] = s * xb.y[i]; gx.z[i] = s * xb.z[i];
    gv.x[i] = s * vb.x[i]; gv.y[i] = s * vb.y[i]; gv.z[i] = s * vb.z[i];
    acc[0] += wacc.x[i];
    acc[1] += wacc.y[i];
    acc[2] += wacc.z[i];
  }
  const int tid = threadIdx.x;
  for (int c = 0; c < 3; ++c) sh[c * ADJ_THREADS + tid] = acc[c];
  __syncthreads();
  for (int w = ADJ_THREADS / 2; w > 0; w >>= 1) {
    if (tid < w)
      for (int c = 0; c < 3; ++c) sh[c * ADJ_THREADS + tid] += sh[c * ADJ_THREADS + tid + w];
    __syncthreads();
  }
  if (tid == 0)
    for (int c = 0; c < 3; ++c) bpart[blockIdx.x * 3 + c] = sh[c * ADJ_THREADS];
}

__global__ void k_adj_out_final(const double *__restrict__ bpart, const double *gscale, double *gw) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const double s = gscale ? *gscale : 1.0;
    for (int c = 0; c < 3; ++c) {
      double t = 0.0;
      for (int b = 0; b < ADJ_BLOCKS; ++b) t += bpart[b * 3 + c];
      gw[c] = s * t;
    }
  }
}

// Loss: per-block partials of (k_C/2) q_i w phi_i + (m/2) sum_k w_k^2 x_k^2 + |x - target|^2.
__global__ void __launch_bounds__(ADJ_THREADS) k_loss_part(Phys p, int64_t n, const double *q, CVec3 x,
                                                           CVec3 tgt, const double *__restrict__ phi,
                                                           int n_jc, double *bpart) {
  __shared__ double sh[ADJ_THREADS];
  double acc = 0.0;
  const int64_t stride = (int64_t)ADJ_BLOCKS * ADJ_THREADS;
  for (int64_t i = (int64_t)blockIdx.x * ADJ_THREADS + threadIdx.x; i < n; i += stride) {
    double ph = 0.0;
    for (int jc = 0; jc < n_jc; ++jc) ph += phi[(int64_t)jc * n + i];
    const double qi = q ? q[i] : p.charge;
    const double qw = q ? qi : qi * p.charge;
    const double xv[3] = {x.x[i], x.y[i], x.z[i]};
    const double tv[3] = {tgt.x[i], tgt.y[i], tgt.z[i]};
    double e = 0.5 * p.k_coulomb * qw * ph;
    for (int k = 0; k < 3; ++k) {
      e += 0.5 * p.mass * p.omega[k] * p.omega[k] * xv[k] * xv[k];
      const double d = xv[k] - tv[k];
      e += d * d;
    }
    acc += e;
  }
  const int tid = threadIdx.x;
  sh[tid] = acc;
  __syncthreads();
  for (int w = ADJ_THREADS / 2; w > 0; w >>= 1) {
    if (tid < w) sh[tid] += sh[tid + w];
    __syncthreads();
  }
  if (tid == 0) bpart[blockIdx.x] = sh[0];
}

__global__ void k_loss_final(const double *__restrict__ bpart, double *loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < ADJ_BLOCKS; ++b) t += bpart[b];
    *loss = t;
  }
}

// ---------------------------------------------------------------------------
cudaError_t launch_adj_init(const Phys &p, int64_t n, const double *const xT[3],
                            const double *const aT[3], const double *const tgt[3], double *const xb[3],
                            double *const vb[3], double *const ab[3], double *const wacc[3],
                            cudaStream_t st) {
  k_adj_init<<<nblk(n, 256), 256, 0, st>>>(p, n, CVec3{xT[0], xT[1], xT[2]}, CVec3{aT[0], aT[1], aT[2]},
                                           CVec3{tgt[0], tgt[1], tgt[2]}, Vec3{xb[0], xb[1], xb[2]},
                                           Vec3{vb[0], vb[1], vb[2]}, Vec3{ab[0], ab[1], ab[2]},
                                           Vec3{wacc[0], wacc[1], wacc[2]});
  return cudaGetLastError();
}

cudaError_t launch_adj_epi(const Phys &p, int64_t n, const double *q, const double *const x[3],
                           const double *part, int n_jc, double *const xb[3], double *const vb[3],
                           double *const ab[3], double *const wacc[3], int last, int more,
                           cudaStream_t st) {
  k_adj_epi<<<nblk(n, 256), 256, 0, st>>>(p, n, q, CVec3{x[0], x[1], x[2]}, part, n_jc,
                                          Vec3{xb[0], xb[1], xb[2]}, Vec3{vb[0], vb[1], vb[2]},
                                          Vec3{ab[0], ab[1], ab[2]}, Vec3{wacc[0], wacc[1], wacc[2]},
                                          last, more);
  return cudaGetLastError();
}

cudaError_t launch_adj_out(int64_t n, double *const xb[3], double *const vb[3], double *const wacc[3],
                           const double *gscale, double *gx0, double *gv0, double *gw, double *bpart,
                           cudaStream_t st) {
  k_adj_out<<<ADJ_BLOCKS, ADJ_THREADS, 0, st>>>(n, CVec3{xb[0], xb[1], xb[2]}, CVec3{vb[0], vb[1], vb[2]},
                                                CVec3{wacc[0], wacc[1], wacc[2]}, gscale,
                                                Vec3{gx0, gx0 + n, gx0 + 2 * n},
                                                Vec3{gv0, gv0 + n, gv0 + 2 * n}, bpart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_adj_out_final<<<1, 32, 0, st>>>(bpart, gscale, gw);
  return cudaGetLastError();
}

cudaError_t launch_loss(const Phys &p, int64_t n, const double *q, const double *const x[3],
                        const double *const tgt[3], const double *phi_part, int n_jc, double *bpart,
                        double *loss, cudaStream_t st) {
  k_loss_part<<<ADJ_BLOCKS, ADJ_THREADS, 0, st>>>(p, n, q, CVec3{x[0], x[1], x[2]},
                                                  CVec3{tgt[0], tgt[1], tgt[2]}, phi_part, n_jc, bpart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_loss_final<<<1, 32, 0, st>>>(bpart, loss);
  return cudaGetLastError();
}

}  // namespace nb
