// nb_noalloc.cu -- nb_energy_noalloc: the energy computation of nb_energy
// for callers that must not allocate device memory.
//
// Why it exists.  nb_energy takes its scratch (the per-chunk potential
// partial sums and the reduction partials) from a library arena that it
// grows with cudaMalloc.  Some callers cannot allow that:
//  - cudaMalloc can synchronise the whole device, which a latency-bound
//    monitoring loop that samples energies between integration steps
//    cannot tolerate;
//  - a host framework may already own all device memory through its own
//    pool or caching allocator, so a raw cudaMalloc can fail, or can take
//    memory the framework has budgeted for something else.
// This entry point allocates nothing.  Its scratch is one file-scope device
// array of fixed size, created when the library is loaded and held by
// every GPU that loads the library until the process exits.
//
// Sharing rule.  Every call uses the same array.  Calls whose work can
// overlap on the GPU (different streams, or different host threads without
// ordering) race on it and give wrong results; serialise them.  Each call
// overwrites every scratch word it reads before reading it, so nothing has
// to start at zero and the contents left by the previous call do not matter.
#include <mutex>

#include "nb_common.cuh"

namespace nb {

// Scratch capacity: 8 MiB of doubles.  It bounds n through the launch plan of
// the potential kernel: n_jc * n + 3 * ENERGY_BLOCKS + 4 doubles must fit.
// With the default plan on a 152-SM GB300 that holds for every n up to about
// 1,000,000 (n_jc * n is about the SM count times the plan's blocks per SM
// times its block size); a potential-kernel tuning override (nb_set_tuning
// kind 1) or a GPU with more SMs can lower the limit.
constexpr size_t NOALLOC_SCRATCH_DOUBLES = (size_t)1 << 20;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[MAX_DEVICES] = {nullptr};

// Device address of g_noalloc_scratch on the current device.  In host code
// the symbol names a host-side stand-in, not device memory, so the address
// is looked up once per device with that device current and cached.
cudaError_t noalloc_scratch(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace nb

using namespace nb;

extern "C" nb_status nb_energy_noalloc(const nb_params *params, const nb_system *sys,
                                       double out[4], void *stream) {
  NvtxRange range_("nb_energy_noalloc");
  // The same host-side checks as nb_energy, before any CUDA call.
  NB_TRY(check_params(params));
  NB_TRY(check_system(sys, true, false));
  if (!out) return fail(NB_EINVAL, "out is NULL");
  const int64_t n = sys->n;
  if (n == 0) {
    out[0] = out[1] = out[2] = out[3] = 0.0;
    return NB_OK;
  }
  const Plan pl = make_plan(n, MODE_FP64, 1);
  const size_t need = (size_t)pl.n_jc * (size_t)n + 3 * ENERGY_BLOCKS + 4;
  if (need > NOALLOC_SCRATCH_DOUBLES)
    return fail(NB_EINVAL,
                "nb_energy_noalloc: n = %lld needs %zu scratch doubles, above its fixed %zu "
                "(8 MiB); use nb_energy",
                (long long)n, need, NOALLOC_SCRATCH_DOUBLES);
  double *scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess)
    return fail(NB_ECUDA, "nb_energy_noalloc: cudaGetSymbolAddress of the scratch array failed: %s",
                cudaGetErrorString(e));
  double *ppart = scratch;
  double *bpart = ppart + (size_t)pl.n_jc * (size_t)n;
  double *out4 = bpart + 3 * ENERGY_BLOCKS;
  const Phys p = to_phys(params);
  const StateView v = to_view(sys);
  const double t = params->t0 + (double)sys->step * params->dt;
  cudaStream_t st = (cudaStream_t)stream;
  e = launch_pair_phi(pl, n, sys->x, sys->y, sys->z, sys->q, params->charge, params->soft2, ppart, st);
  if (e == cudaSuccess) e = launch_energy(p, v, ppart, pl.n_jc, t, bpart, out4, st);
  if (e == cudaSuccess) {
    count_launches(3);
    e = cudaMemcpyAsync(out, out4, 4 * sizeof(double), cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess)
    return fail(NB_ECUDA, "nb_energy_noalloc: %s", cudaGetErrorString(e));
  return NB_OK;
}
