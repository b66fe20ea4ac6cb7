// nb_probe.cu -- element-wise probes of the pair arithmetic (steps a1-a3 of
// one pair): the r^-3 that each precision mode forms from a displacement,
// and the raw FP32 reciprocal-square-root seed it starts from.  They run the
// same device functions as the pair kernels, so a caller can measure a mode's
// error distribution against an exact reference over any set of inputs.
#include <algorithm>
#include <map>
#include <utility>
#include <vector>

#include "nb_common.cuh"
#include "nb_symsched.cuh"

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
  } else if (ladder_mode(MODE)) {
    s = ladder_rinv3<MODE>(fma(x, x, fma(y, y, fma(z, z, soft2))));
  } else if (MODE == MODE_DF64) {
    float dh[3], dl[3], s2h, s2l, sh, sl;
    split_f64(x, dh[0], dl[0]);
    split_f64(y, dh[1], dl[1]);
    split_f64(z, dh[2], dl[2]);
    split_f64(soft2, s2h, s2l);
    df_rinv3(dh, dl, s2h, s2l, sh, sl);
    s = f32_to_f64(sh) + f32_to_f64(sl);
  } else {  // the mixed modes: the FP32 bulk of the displacement cast to FP32
    s = f32_to_f64(f32_rinv3<MODE == MODE_SPLIT_RSQ>(f64_to_f32_rn(x), f64_to_f32_rn(y), f64_to_f32_rn(z),
                                                     (float)soft2));
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
      precision > NB_MIXED_SPLIT_RSQ)
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
    case NB_FP64_RSQ_NR2: e = launch_probe<MODE_RSQ_NR2>(n, dx, dy, dz, soft2, out, st); break;
    default: e = launch_probe<MODE_SPLIT_RSQ>(n, dx, dy, dz, soft2, out, st); break;
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

// ---------------------------------------------------------------------------
// Pipe throughput probe: the rate at which every SM retires one instruction
// kind (the denominator of the ALU rooflines).  Each thread runs CH
// independent dependence chains of the instruction, issued from inline PTX
// so that the compiler keeps every one, for `iters` rounds of 8; thread 0 of
// each block records its SM and the SM clock before and after, between two
// block barriers.  The chains use shared or per-chain operands (DIST).  The
// attainable rate depends on the shape through register-bank conflicts: on
// GB300 four FP64 FMA chains with their own operands reach 2.0 lanes/clk/SM
// where eight with shared operands settle at 1.68, while FP32 FMA chains
// reach 125 lanes/clk/SM with shared operands and 85 with their own.  The
// entry point runs three shapes and reports the fastest.
namespace nb {

constexpr int PIPE_THREADS = 512;
constexpr int PIPE_BLOCKS_PER_SM = 2;
constexpr int PIPE_UNROLL = 8;

template <int KIND>
__device__ __forceinline__ void pipe_op(double &a, float &f, double b, double c, float fb, float fc) {
  if (KIND == 0) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a) : "d"(b), "d"(c));
  if (KIND == 1) asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(a) : "d"(c));
  if (KIND == 2) asm volatile("mul.rn.f64 %0, %0, %1;" : "+d"(a) : "d"(b));
  if (KIND == 3) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f) : "f"(fb), "f"(fc));
  if (KIND == 4) asm volatile("add.rn.f32 %0, %0, %1;" : "+f"(f) : "f"(fc));
  if (KIND == 5) asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(f));
}

template <int KIND, int CH, bool DIST>
__global__ void __launch_bounds__(PIPE_THREADS) k_pipe_probe(int64_t iters, double b, double c,
                                                             unsigned long long *clk, double *sink) {
  constexpr bool F64 = KIND <= 2;
  double a[CH], bk[CH], ck[CH];
  float f[CH], fbk[CH], fck[CH];
#pragma unroll
  for (int k = 0; k < CH; ++k) {
    a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    f[k] = 1.0f + 1e-3f * (float)(threadIdx.x + k);
    bk[k] = (DIST && KIND != 2) ? b + 1e-9 * k : b;
    ck[k] = DIST ? c * (1 + k) : c;
    fbk[k] = (float)bk[k];
    fck[k] = (float)ck[k];
  }
  __syncthreads();
  unsigned long long t0 = 0;
  if (threadIdx.x == 0) t0 = clock64();
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < PIPE_UNROLL; ++u)
#pragma unroll
      for (int k = 0; k < CH; ++k) pipe_op<KIND>(a[k], f[k], bk[k], ck[k], fbk[k], fck[k]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long t1 = clock64();
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    clk[3 * blockIdx.x] = smid;
    clk[3 * blockIdx.x + 1] = t0;
    clk[3 * blockIdx.x + 2] = t1;
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < CH; ++k) s += F64 ? a[k] : (double)f[k];
  if (s == 12345.678) sink[0] = s;  // keeps the chains observable
}

// One timed launch of shape (CH, DIST): lanes per clock per SM (median over
// SMs) and the span's SM clock in MHz.
template <int KIND, int CH, bool DIST>
static cudaError_t pipe_shape(int sms, int64_t iters, unsigned long long *clk, double *sink, cudaStream_t st,
                              double *rate, double *mhz) {
  const int blocks = sms * PIPE_BLOCKS_PER_SM;
  const double b = (KIND == 2) ? 1.0 : 0.999999, c = (KIND == 1) ? 1e-300 : 1e-7;
  // the chains' iteration count scales so that every shape issues the same work
  const int64_t it = iters * 4 / CH;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    k_pipe_probe<KIND, CH, DIST><<<blocks, PIPE_THREADS, 0, st>>>(it, b, c, clk, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  std::vector<unsigned long long> h(3 * (size_t)blocks);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), clk, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  count_launches(1);
  std::map<unsigned long long, std::pair<unsigned long long, unsigned long long>> span;
  std::map<unsigned long long, int> nblk;
  for (int bl = 0; bl < blocks; ++bl) {
    const unsigned long long sm = h[3 * bl], t0 = h[3 * bl + 1], t1 = h[3 * bl + 2];
    auto p = span.find(sm);
    if (p == span.end()) span[sm] = {t0, t1};
    else p->second = {std::min(p->second.first, t0), std::max(p->second.second, t1)};
    ++nblk[sm];
  }
  std::vector<double> r;
  double cyc_max = 0.0;
  for (auto &kv : span) {
    const double cyc = (double)(kv.second.second - kv.second.first);
    const double ops = (double)nblk[kv.first] * PIPE_THREADS * (double)it * PIPE_UNROLL * CH;
    if (cyc > 0.0) r.push_back(ops / cyc);
    cyc_max = std::max(cyc_max, cyc);
  }
  if (r.empty()) return cudaErrorUnknown;
  std::sort(r.begin(), r.end());
  *rate = r[r.size() / 2];
  *mhz = ms > 0.0f ? cyc_max / (ms * 1e3) : 0.0;
  return cudaSuccess;
}

template <int KIND>
static cudaError_t pipe_best(int sms, int64_t iters, unsigned long long *clk, double *sink, cudaStream_t st,
                             double out[3]) {
  double r[3] = {0, 0, 0}, m[3] = {0, 0, 0};
  cudaError_t e = pipe_shape<KIND, 4, true>(sms, iters, clk, sink, st, &r[0], &m[0]);
  if (e == cudaSuccess) e = pipe_shape<KIND, 4, false>(sms, iters, clk, sink, st, &r[1], &m[1]);
  if (e == cudaSuccess) e = pipe_shape<KIND, 8, false>(sms, iters, clk, sink, st, &r[2], &m[2]);
  if (e != cudaSuccess) return e;
  int k = 0;
  for (int j = 1; j < 3; ++j)
    if (r[j] > r[k]) k = j;
  out[0] = r[k];
  out[1] = m[k];
  out[2] = k;
  return cudaSuccess;
}

// Probe of the half-pair kernels' bounded wait: one thread publishes
// `committed` rounds for block 0 (a release store, as sym_commit does) and
// then waits, as sym_commit does, until block 0 has committed `round`.  A
// wait for a round nobody commits runs out its spin limit, sets
// ERR_TIMEOUT in the error word and ends normally.
__global__ void k_sym_wait_probe(int *sync, int committed, int round, unsigned *err, int *ok) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st_release(sync + 1, committed);
  const bool done = sym_wait(sync, 0, round, err);
  if (!done) atomicOr(err, ERR_TIMEOUT);
  ok[0] = done ? 1 : 0;
}

cudaError_t launch_sym_wait_probe(int *sync, int committed, int round, unsigned *err, int *ok, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(sync, 0, 2 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_sym_wait_probe<<<1, 32, 0, st>>>(sync, committed, round, err, ok);
  return cudaGetLastError();
}

}  // namespace nb

extern "C" nb_status nb_pipe_probe(int32_t kind, int64_t iters, double out[3], void *stream) {
  if (kind < 0 || kind > 5) return fail(NB_EINVAL, "nb_pipe_probe: unknown kind %d", kind);
  if (iters < 2 || iters > ((int64_t)1 << 24)) return fail(NB_EINVAL, "nb_pipe_probe: iters out of range");
  if (!out) return fail(NB_EINVAL, "nb_pipe_probe: out is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const int sms = device_sm_count();
  const int blocks = sms * PIPE_BLOCKS_PER_SM;
  unsigned long long *clk = nullptr;
  cudaError_t e = cudaMalloc(&clk, sizeof(unsigned long long) * 3 * blocks + sizeof(double));
  if (e == cudaSuccess) {
    double *sink = reinterpret_cast<double *>(clk + 3 * blocks);
    switch (kind) {
      case 0: e = pipe_best<0>(sms, iters, clk, sink, st, out); break;
      case 1: e = pipe_best<1>(sms, iters, clk, sink, st, out); break;
      case 2: e = pipe_best<2>(sms, iters, clk, sink, st, out); break;
      case 3: e = pipe_best<3>(sms, iters, clk, sink, st, out); break;
      case 4: e = pipe_best<4>(sms, iters, clk, sink, st, out); break;
      default: e = pipe_best<5>(sms, iters, clk, sink, st, out); break;
    }
  }
  if (clk) cudaFree(clk);
  if (e != cudaSuccess) return fail(NB_ECUDA, "nb_pipe_probe: %s", cudaGetErrorString(e));
  return NB_OK;
}
