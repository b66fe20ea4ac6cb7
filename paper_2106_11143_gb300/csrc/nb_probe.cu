// nb_probe.cu -- element-wise probes of the pair arithmetic (steps a1-a3 of
// one pair): the r^-3 that each precision mode forms from a displacement,
// and the raw FP32 reciprocal-square-root seed it starts from.  They run the
// same device functions as the pair kernels, so a caller can measure a mode's
// error distribution against an exact reference over any set of inputs.
#include "nb_common.cuh"

namespace nb {

template <int MODE>
__global__ void k_rinv3_probe(int64_t n, const double *__restrict__ dx, const double *__restrict__ dy,
                              const double *__restrict__ dz, double soft2, double *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = dx[i], y = dy[i], z = dz[i];
  double s;
  if (MODE == MODE_FP64) {
    s = rinv3_fp64(x, y, z, soft2);
  } else if (fp64_like(MODE)) {
    s = ladder_rinv3<MODE>(fma(x, x, fma(y, y, fma(z, z, soft2))));
  } else if (MODE == MODE_DF64) {
    float dh[3], dl[3], s2h, s2l, sh, sl;
    split_f64(x, dh[0], dl[0]);
    split_f64(y, dh[1], dl[1]);
    split_f64(z, dh[2], dl[2]);
    split_f64(soft2, s2h, s2l);
    df_rinv3(dh, dl, s2h, s2l, sh, sl);
    s = f32_to_f64(sh) + f32_to_f64(sl);
  } else {  // both mixed modes: the FP32 bulk of the displacement cast to FP32
    s = f32_to_f64(f32_rinv3(f64_to_f32_rn(x), f64_to_f32_rn(y), f64_to_f32_rn(z), (float)soft2));
  }
  out[i] = s;
}

__global__ void k_rsqrt_seed_probe(int64_t n, const float *__restrict__ x, float *__restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x[i]));
  y[i] = r;
}

template <int MODE>
static cudaError_t launch_probe(int64_t n, const double *dx, const double *dy, const double *dz,
                                double soft2, double *out, cudaStream_t st) {
  const int T = 256;
  k_rinv3_probe<MODE><<<(unsigned)((n + T - 1) / T), T, 0, st>>>(n, dx, dy, dz, soft2, out);
  return cudaGetLastError();
}

}  // namespace nb

using namespace nb;

extern "C" nb_status nb_rinv3_probe(int precision, int64_t n, const double *dx, const double *dy,
                                    const double *dz, double soft2, double *out, void *stream) {
  if (n < 0 || n > ((int64_t)1 << 36) || !(soft2 >= 0.0) || precision < NB_FP64 ||
      precision > NB_FP64_RSQ_NR2)
    return NB_EINVAL;
  if (n == 0) return NB_OK;
  if (!dx || !dy || !dz || !out) return NB_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  switch (precision) {
    case NB_FP64: e = launch_probe<MODE_FP64>(n, dx, dy, dz, soft2, out, st); break;
    case NB_MIXED: e = launch_probe<MODE_MIXED>(n, dx, dy, dz, soft2, out, st); break;
    case NB_MIXED_SPLIT: e = launch_probe<MODE_SPLIT>(n, dx, dy, dz, soft2, out, st); break;
    case NB_DF64: e = launch_probe<MODE_DF64>(n, dx, dy, dz, soft2, out, st); break;
    case NB_FP64_SQRTDIV: e = launch_probe<MODE_SQRTDIV>(n, dx, dy, dz, soft2, out, st); break;
    case NB_FP64_RSQ: e = launch_probe<MODE_RSQ>(n, dx, dy, dz, soft2, out, st); break;
    case NB_FP64_RSQ_NR1: e = launch_probe<MODE_RSQ_NR1>(n, dx, dy, dz, soft2, out, st); break;
    default: e = launch_probe<MODE_RSQ_NR2>(n, dx, dy, dz, soft2, out, st); break;
  }
  if (e != cudaSuccess) return NB_ECUDA;
  count_launches(1);
  return NB_OK;
}

extern "C" nb_status nb_rsqrt_seed_probe(int64_t n, const float *x, float *y, void *stream) {
  if (n < 0 || n > ((int64_t)1 << 36)) return NB_EINVAL;
  if (n == 0) return NB_OK;
  if (!x || !y) return NB_EINVAL;
  const int T = 256;
  k_rsqrt_seed_probe<<<(unsigned)((n + T - 1) / T), T, 0, (cudaStream_t)stream>>>(n, x, y);
  if (cudaGetLastError() != cudaSuccess) return NB_ECUDA;
  count_launches(1);
  return NB_OK;
}
