// nb_api.cu -- host side of the C ABI declared in include/nb.h.
//
// Argument validation, per-(device, stream) scratch arenas, launch planning
// and the orchestration of the pair and epilogue kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <array>
#include <atomic>
#include <map>
#include <vector>
#include <mutex>
#include <string>
#include <utility>

#include "nb_common.cuh"
#include "nb_symsched.cuh"

namespace nb {

cudaError_t launch_chunk_sum1(int64_t n, const double *part, int n_jc, double scale, double *out,
                              cudaStream_t st);
// Bounded-wait probe (nb_probe.cu): sync holds 2 ints, ok 1 int, device.
cudaError_t launch_sym_wait_probe(int *sync, int committed, int round, unsigned *err, int *ok, cudaStream_t st);

namespace {
thread_local std::string g_last_error;
}  // namespace

nb_status fail(nb_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

namespace {

#define NB_CUDA_TRY(call)                                                              \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(NB_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                  __FILE__, __LINE__);                                                 \
  } while (0)

// A captured window of nb_step (STEP_WINDOW steps), replayed for the middle
// steps of a long call at small n, and the bytes of every kernel argument it
// was captured with (it is valid while they are unchanged).
struct StepGraph {
  std::vector<unsigned char> key;
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels = 0;  // kernel launches per replay
  uint64_t last = 0;     // the arena's use counter at its last replay
};
constexpr size_t STEP_WINDOW_CACHE = 4;  // windows kept per stream (least recently used goes)

// Scratch owned by the library for one (device, stream).
struct Arena {
  char *buf = nullptr;
  size_t cap = 0;
  unsigned *err = nullptr;  // 256 B: device error word at 0, step counters at 64 and 72
  cudaStream_t cap_st = nullptr;  // private stream the step windows are captured on
  std::vector<StepGraph> windows;  // at most STEP_WINDOW_CACHE
  uint64_t uses = 0;
  // nb_step_batched_each: the device table of per-instance parameters
  // (BATCH_LIMIT_INST entries) and the nb_params it was last filled from
  Phys *ptab = nullptr;
  std::vector<nb_params> ptab_src;
  std::vector<Phys> ptab_stage;
};

int64_t *step_counters(Arena *a) { return reinterpret_cast<int64_t *>(reinterpret_cast<char *>(a->err) + 64); }

std::mutex g_mu;
std::map<std::pair<int, cudaStream_t>, Arena> g_arenas;

// Returns the arena of the current device and `st` with at least `bytes`
// of scratch.  Growing synchronises `st` before the old buffer is freed.
nb_status get_arena(cudaStream_t st, size_t bytes, Arena **out) {
  int dev = 0;
  NB_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  Arena &a = g_arenas[std::make_pair(dev, st)];
  if (!a.err) {
    if (cudaMalloc(&a.err, 256) != cudaSuccess) return fail(NB_ENOMEM, "cudaMalloc(error word) failed");
    NB_CUDA_TRY(cudaMemsetAsync(a.err, 0, 256, st));
  }
  if (a.cap < bytes) {
    if (a.buf) {
      NB_CUDA_TRY(cudaStreamSynchronize(st));
      NB_CUDA_TRY(cudaFree(a.buf));
      a.buf = nullptr;
      a.cap = 0;
    }
    const size_t want = bytes + bytes / 8;  // headroom against repeated growth
    if (cudaMalloc(&a.buf, want) != cudaSuccess) {
      cudaGetLastError();
      return fail(NB_ENOMEM, "cudaMalloc(%zu bytes of scratch) failed", want);
    }
    a.cap = want;
  }
  *out = &a;
  return NB_OK;
}

// Carves aligned sub-buffers out of an arena.
struct Carver {
  size_t off = 0;
  char *base = nullptr;
  template <class T>
  T *take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
    off += count * sizeof(T);
    return p;
  }
};

bool finite(double v) { return std::isfinite(v); }
bool aligned8(const void *ptr) { return ((uintptr_t)ptr & 7u) == 0; }

nb_status check_array(const void *ptr, const char *name) {
  if (!ptr) return fail(NB_EINVAL, "%s is NULL", name);
  if (!aligned8(ptr)) return fail(NB_EINVAL, "%s is not 8-byte aligned", name);
  return NB_OK;
}

}  // namespace

nb_status check_params(const nb_params *p) {
  if (!p) return fail(NB_EINVAL, "params is NULL");
  if (!(p->mass > 0.0) || !finite(p->mass)) return fail(NB_EINVAL, "mass must be positive and finite");
  if (!finite(p->k_coulomb) || !finite(p->charge) || !finite(p->soft2) || p->soft2 < 0.0)
    return fail(NB_EINVAL, "k_coulomb, charge and soft2 must be finite (soft2 >= 0)");
  if (p->trap != NB_TRAP_HARMONIC && p->trap != NB_TRAP_RF) return fail(NB_EINVAL, "unknown trap %d", p->trap);
  if (p->precision < NB_FP64 || p->precision > NB_MIXED_SPLIT_RSQ)
    return fail(NB_EINVAL, "unknown precision %d", p->precision);
  for (int k = 0; k < 3; ++k)
    if (!finite(p->omega[k]) || !finite(p->omega_rate[k])) return fail(NB_EINVAL, "omega must be finite");
  if (!finite(p->q_mathieu) || !finite(p->omega_rf) || !finite(p->rf_phase) || !finite(p->gamma) ||
      !finite(p->dt) || !finite(p->t0) || !finite(p->noise_T))
    return fail(NB_EINVAL, "trap, friction and time parameters must be finite");
  if (p->gamma < 0.0 || p->noise_T < 0.0) return fail(NB_EINVAL, "gamma and noise_T must be >= 0");
  if (p->noise_T > 0.0 && p->gamma == 0.0) return fail(NB_EINVAL, "noise_T > 0 needs gamma > 0");
  if (p->reserved != 0) return fail(NB_EINVAL, "params.reserved must be 0");
  return NB_OK;
}

nb_status check_system(const nb_system *s, bool need_v, bool need_a) {
  if (!s) return fail(NB_EINVAL, "system is NULL");
  if (s->n < 0) return fail(NB_EINVAL, "n must be >= 0");
  if (s->n > ((int64_t)1 << 31)) return fail(NB_EINVAL, "n above 2^31 is not supported");
  if (s->n == 0) return NB_OK;
  NB_TRY(check_array(s->x, "x"));
  NB_TRY(check_array(s->y, "y"));
  NB_TRY(check_array(s->z, "z"));
  if (need_v) {
    NB_TRY(check_array(s->vx, "vx"));
    NB_TRY(check_array(s->vy, "vy"));
    NB_TRY(check_array(s->vz, "vz"));
  }
  if (need_a) {
    NB_TRY(check_array(s->ax, "ax"));
    NB_TRY(check_array(s->ay, "ay"));
    NB_TRY(check_array(s->az, "az"));
  }
  if (s->q && !aligned8(s->q)) return fail(NB_EINVAL, "q is not 8-byte aligned");
  if (s->m && !aligned8(s->m)) return fail(NB_EINVAL, "m is not 8-byte aligned");
  return NB_OK;
}

Phys to_phys(const nb_params *p) {
  Phys f;
  f.k_coulomb = p->k_coulomb;
  f.mass = p->mass;
  f.charge = p->charge;
  f.soft2 = p->soft2;
  f.trap = p->trap;
  f.precision = p->precision;
  for (int k = 0; k < 3; ++k) {
    f.omega[k] = p->omega[k];
    f.omega_rate[k] = p->omega_rate[k];
  }
  f.q_mathieu = p->q_mathieu;
  f.omega_rf = p->omega_rf;
  f.rf_phase = p->rf_phase;
  f.gamma = p->gamma;
  f.dt = p->dt;
  f.t0 = p->t0;
  f.noise_T = p->noise_T;
  f.seed = p->seed;
  f.instance = p->instance;
  return f;
}

StateView to_view(const nb_system *s) {
  StateView v;
  v.n = s->n;
  v.x = s->x; v.y = s->y; v.z = s->z;
  v.vx = s->vx; v.vy = s->vy; v.vz = s->vz;
  v.ax = s->ax; v.ay = s->ay; v.az = s->az;
  v.q = s->q;
  v.m = s->m;
  return v;
}

namespace {

// Scratch need of one force evaluation.
size_t force_bytes(const Plan &pl, int mode, int64_t n, bool extra_pos, bool phi, const Plan &plp) {
  Carver c;
  c.take<double>(part_doubles(pl, n, 3));
  if (split_like(mode)) c.take<float>(6 * (size_t)n);
  if (extra_pos) c.take<double>(3 * (size_t)n);
  if (phi) c.take<double>((size_t)plp.n_jc * n);
  return c.off + 256;
}

// Force evaluation at positions (x, y, z) into `part`.
nb_status pair_forces(const Plan &pl, int mode, int64_t n, const double *x, const double *y,
                      const double *z, const double *q, double soft2, double *part, float *split,
                      unsigned *err, cudaStream_t st) {
  PosF32 pf{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  if (split_like(mode)) {
    NB_CUDA_TRY(launch_split_positions(n, x, y, z, split, st));
    count_launches(1);
    pf = PosF32{split, split + n, split + 2 * n, split + 3 * n, split + 4 * n, split + 5 * n};
  }
  timing_begin(st);
  NB_CUDA_TRY(launch_pair_force(pl, mode, n, x, y, z, q, pf, soft2, part, err, st));
  timing_end(st);
  count_launches(1);
  return NB_OK;
}

// ---------------------------------------------------------------------------
// Instrumentation state.
std::atomic<uint64_t> g_launches{0};
thread_local uint64_t *g_count_sink = nullptr;  // set while a step window is captured
std::mutex g_tmu;
std::vector<cudaEvent_t> g_ev;  // pairs: start, stop
int64_t g_ev_cap = 0, g_ev_used = 0;

}  // namespace

void count_launches(uint64_t k) {
  if (g_count_sink) {  // captured into a graph, counted when it is replayed
    *g_count_sink += k;
    return;
  }
  g_launches.fetch_add(k, std::memory_order_relaxed);
}

void record_error(const char *msg) { g_last_error = msg; }

void timing_begin(cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_tmu);
  if (g_ev_used < g_ev_cap) cudaEventRecord(g_ev[2 * g_ev_used], st);
}

void timing_end(cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_tmu);
  if (g_ev_used < g_ev_cap) {
    cudaEventRecord(g_ev[2 * g_ev_used + 1], st);
    ++g_ev_used;
  }
}

// ---------------------------------------------------------------------------
// Step windows: at small n a step is a few short kernels and the per-launch
// cost bounds the step rate, so nb_step captures STEP_WINDOW steps once into a
// CUDA graph and replays it for the middle steps of a call.
namespace {

constexpr int64_t STEP_WINDOW = 8;        // steps per replay (even: the position buffers alternate)
constexpr int64_t STEP_GRAPH_N = 4096;    // default: windows for n up to this
constexpr int64_t STEP_GRAPH_STEPS = 32;  // default: and calls of at least this many steps

bool timing_active() {
  std::lock_guard<std::mutex> lk(g_tmu);
  return g_ev_used < g_ev_cap;
}

// Whether this nb_step call replays windows.  Tuning kind 6 overrides the
// default (R = 1 use, 0 not; block = the least nsteps).  Never while the
// caller's stream is itself being captured or kernel timing is on.
bool use_step_graph(int mode, int64_t n, int64_t nsteps, cudaStream_t st) {
  int tb = 0, tr = 0, tbps = 0;
  bool on = n <= STEP_GRAPH_N;
  int64_t least = STEP_GRAPH_STEPS;
  if (tuning_lookup(6, mode, n, &tb, &tr, &tbps)) {
    on = tr == 1;
    least = tb;
  }
  if (!on || nsteps < std::max<int64_t>(least, STEP_WINDOW + 2) || timing_active()) return false;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs == cudaStreamCaptureStatusNone;
}

// Single-block steps (nb_small.cu) for small systems: one launch runs many
// steps, but all pair terms of a step run on one SM, so the path wins only
// below a size that grows with the pair term's throughput.  Defaults: the
// largest n, per precision, at which it was faster than the multi-kernel
// steps on GB300.  Tuning kind 7 overrides them (R = 1 use, 0 not) within
// the kernel's limits.  Not while kernel timing is on (it times pair
// kernels).
// Steps per launch: at most 16384, and about 2^28 pair terms per launch at
// larger n, so that one launch stays well under a second.
int64_t small_steps_per_launch(int64_t n) {
  return std::max<int64_t>(64, std::min<int64_t>(16384, ((int64_t)1 << 28) / (n * n)));
}

int64_t small_default_n(int mode) {
  switch (mode) {
    case MODE_SQRTDIV: return 16;  // an FP64 square root and division per pair
    case MODE_DF64: return 48;     // its pair term runs on the FP32 pipe
    default: return 32;
  }
}

bool use_small_steps(const Plan &pl, int mode, int64_t n) {
  if (pl.sym || n > SMALL_MAX_N || small_smem_bytes(pl, mode, n) > (size_t)SMALL_SMEM_MAX || timing_active())
    return false;
  int tb = 0, tr = 0, tbps = 0;
  if (tuning_lookup(7, mode, n, &tb, &tr, &tbps)) return tr == 1;
  return n <= small_default_n(mode);
}

// The bytes of every argument the kernels of a window take: a cached window
// is replayed only while they are unchanged.
struct KeyBytes {
  std::vector<unsigned char> b;
  template <class T>
  void put(const T &v) {
    const unsigned char *p = reinterpret_cast<const unsigned char *>(&v);
    b.insert(b.end(), p, p + sizeof(T));
  }
};

static_assert(sizeof(Phys) == 160 && sizeof(StateView) == 104 && sizeof(Plan) == 40,
              "a new field of Phys, StateView or Plan must join window_key");

std::vector<unsigned char> window_key(const Plan &pl, int mode, const Phys &p, const StateView &v,
                                      double *const *A, double *const *B, const double *part,
                                      const float *split, const Arena *a) {
  KeyBytes k;
  k.put(mode);
  k.put(tuning_generation());
  k.put(pl.block); k.put(pl.R); k.put(pl.jchunk); k.put(pl.n_it); k.put(pl.n_jc); k.put(pl.sym); k.put(pl.G); k.put(pl.nbk);
  k.put(p.k_coulomb); k.put(p.mass); k.put(p.charge); k.put(p.soft2); k.put(p.trap); k.put(p.precision);
  for (int c = 0; c < 3; ++c) {
    k.put(p.omega[c]);
    k.put(p.omega_rate[c]);
  }
  k.put(p.q_mathieu); k.put(p.omega_rf); k.put(p.rf_phase); k.put(p.gamma); k.put(p.dt); k.put(p.t0);
  k.put(p.noise_T); k.put(p.seed); k.put(p.instance);
  k.put(v.n); k.put(v.x); k.put(v.y); k.put(v.z); k.put(v.vx); k.put(v.vy); k.put(v.vz);
  k.put(v.ax); k.put(v.ay); k.put(v.az); k.put(v.q); k.put(v.m); k.put(v.ion0);
  for (int c = 0; c < 3; ++c) {
    k.put(A[c]);
    k.put(B[c]);
  }
  k.put(part); k.put(split); k.put(a->err);
  return k.b;
}

// Captures one window on the arena's private stream: STEP_WINDOW steps of
// pair forces and epilogue, the position buffers alternating A -> B -> A.
// The epilogues take the step index from the two counters c0, c1: the first
// reads c0 (the index of the step before the window) and stores
// c0 + STEP_WINDOW in c1; the others read c1 with offsets, and the last
// copies c1 to c0, so each replay continues where the previous one ended.
nb_status capture_window(Arena *a, const Plan &pl, int mode, const Phys &p, const StateView &v,
                         double *const *A, double *const *B, double *part, float *split,
                         double soft2, StepGraph *out) {
  if (!a->cap_st) NB_CUDA_TRY(cudaStreamCreateWithFlags(&a->cap_st, cudaStreamNonBlocking));
  cudaStream_t cs = a->cap_st;
  int64_t *c = step_counters(a);
  NB_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  uint64_t kernels = 0;
  g_count_sink = &kernels;
  nb_status rc = NB_OK;
  cudaError_t e = cudaSuccess;
  for (int64_t k = 1; k <= STEP_WINDOW && rc == NB_OK && e == cudaSuccess; ++k) {
    double *const *P = (k % 2) ? A : B;
    double *const *Nx = (k % 2) ? B : A;
    rc = pair_forces(pl, mode, v.n, P[0], P[1], P[2], v.q, soft2, part, split, a->err, cs);
    if (rc != NB_OK) break;
    const int64_t *cin = k == 1 ? c : c + 1;
    const int64_t soff = k == 1 ? 1 : k - STEP_WINDOW;
    int64_t *cout = k == 1 ? c + 1 : (k == STEP_WINDOW ? c : nullptr);
    const int64_t cout_off = k == 1 ? STEP_WINDOW : 0;
    e = launch_epi_step(p, v, P[0], P[1], P[2], part, pl.n_jc, soff, Nx[0], Nx[1], Nx[2], a->err, cs,
                        cin, cout, cout_off);
    count_launches(1);
  }
  g_count_sink = nullptr;
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(cs, &g);
  if (rc != NB_OK || e != cudaSuccess || ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (rc != NB_OK) return rc;
    return fail(NB_ECUDA, "capturing the step window failed: %s",
                cudaGetErrorString(e != cudaSuccess ? e : ee));
  }
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) return fail(NB_ECUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(ie));
  out->exec = exec;
  out->kernels = kernels;
  return NB_OK;
}

// The cached window with this key, captured (evicting the least recently
// used one when the cache is full) if there is none.
nb_status find_window(Arena *a, std::vector<unsigned char> &key, const Plan &pl, int mode, const Phys &p,
                      const StateView &v, double *const *A, double *const *B, double *part, float *split,
                      double soft2, StepGraph **out) {
  ++a->uses;
  for (StepGraph &g : a->windows)
    if (g.key == key) {
      g.last = a->uses;
      *out = &g;
      return NB_OK;
    }
  StepGraph fresh;
  NB_TRY(capture_window(a, pl, mode, p, v, A, B, part, split, soft2, &fresh));
  fresh.key.swap(key);
  fresh.last = a->uses;
  if (a->windows.size() >= STEP_WINDOW_CACHE) {
    auto lru = std::min_element(a->windows.begin(), a->windows.end(),
                                [](const StepGraph &x, const StepGraph &y) { return x.last < y.last; });
    cudaGraphExecDestroy(lru->exec);  // a pending launch of it still completes
    *lru = std::move(fresh);
    *out = &*lru;
  } else {
    a->windows.push_back(std::move(fresh));
    *out = &a->windows.back();
  }
  return NB_OK;
}

}  // namespace

}  // namespace nb

using namespace nb;

extern "C" {

nb_status nb_forces(const nb_params *params, const nb_system *sys, double *phi, int flags,
                    void *stream) {
  NvtxRange range_("nb_forces");
  NB_TRY(check_params(params));
  NB_TRY(check_system(sys, (flags & NB_ACC_TOTAL) != 0, true));
  if (flags & ~NB_ACC_TOTAL) return fail(NB_EINVAL, "unknown flags 0x%x", flags);
  if (phi && !aligned8(phi)) return fail(NB_EINVAL, "phi is not 8-byte aligned");
  const int64_t n = sys->n;
  if (n == 0) return NB_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int mode = params->precision;
  const Plan pl = make_plan(n, mode, 0);
  const Plan plp = make_plan(n, MODE_FP64, 1);
  Arena *a = nullptr;
  NB_TRY(get_arena(st, force_bytes(pl, mode, n, false, phi != nullptr, plp), &a));
  Carver cv;
  cv.base = a->buf;
  double *part = cv.take<double>(part_doubles(pl, n, 3));
  float *split = split_like(mode) ? cv.take<float>(6 * (size_t)n) : nullptr;
  double *ppart = phi ? cv.take<double>((size_t)plp.n_jc * n) : nullptr;
  const Phys p = to_phys(params);
  const StateView v = to_view(sys);
  const double t = params->t0 + (double)sys->step * params->dt;
  NB_TRY(pair_forces(pl, mode, n, sys->x, sys->y, sys->z, sys->q, params->soft2, part, split, a->err, st));
  NB_CUDA_TRY(launch_epi_forces(p, v, part, pl.n_jc, flags, t, a->err, st));
  count_launches(1);
  if (phi) {
    NB_CUDA_TRY(launch_pair_phi(plp, n, sys->x, sys->y, sys->z, sys->q, params->charge, params->soft2, ppart, st));
    // the pair sums carry w_j = q_j, or 1 for a single species
    NB_CUDA_TRY(launch_chunk_sum1(n, ppart, plp.n_jc, sys->q ? 1.0 : params->charge, phi, st));
    count_launches(2);
  }
  return NB_OK;
}

nb_status nb_step(const nb_params *params, nb_system *sys, int64_t nsteps, void *stream) {
  NvtxRange range_("nb_step");
  NB_TRY(check_params(params));
  NB_TRY(check_system(sys, true, true));
  if (nsteps < 0) return fail(NB_EINVAL, "nsteps must be >= 0");
  if (!(params->dt > 0.0)) return fail(NB_EINVAL, "dt must be > 0");
  const int64_t n = sys->n;
  if (n == 0 || nsteps == 0) {
    sys->step += nsteps;
    return NB_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int mode = params->precision;
  const Plan pl = make_plan(n, mode, 0);
  Arena *a = nullptr;
  if (use_small_steps(pl, mode, n)) {
    NvtxRange sub_("nb_step: single-block steps");
    NB_TRY(get_arena(st, 256, &a));
    const Phys p = to_phys(params);
    const StateView v = to_view(sys);
    for (int64_t done = 0; done < nsteps;) {
      const int64_t k = std::min(nsteps - done, small_steps_per_launch(n));
      NB_CUDA_TRY(launch_small_steps(pl, mode, p, v, sys->step + done, k, a->err, st));
      count_launches(1);
      done += k;
    }
    sys->step += nsteps;
    return NB_OK;
  }
  NB_TRY(get_arena(st, force_bytes(pl, mode, n, true, false, pl), &a));
  Carver cv;
  cv.base = a->buf;
  double *part = cv.take<double>(part_doubles(pl, n, 3));
  float *split = split_like(mode) ? cv.take<float>(6 * (size_t)n) : nullptr;
  double *other = cv.take<double>(3 * (size_t)n);
  double *ubuf[3] = {sys->x, sys->y, sys->z};
  double *obuf[3] = {other, other + n, other + 2 * n};
  // Position buffer of step s: chosen so that the last step reads the
  // library buffer and writes the final positions into the caller's arrays.
  auto buf = [&](int64_t s) -> double ** { return ((nsteps - 1 - s) % 2 == 0) ? obuf : ubuf; };
  const Phys p = to_phys(params);
  const StateView v = to_view(sys);
  // Steps 0 .. nsteps-2 write the next drift, the last one the final state.
  // With step windows, the middle steps after `pre` eager ones are `reps`
  // replays of one captured window.
  const bool windows = use_step_graph(mode, n, nsteps, st);
  const int64_t pre = windows ? 1 + (nsteps - 2) % STEP_WINDOW : nsteps - 1;
  const int64_t reps = windows ? (nsteps - 1 - pre) / STEP_WINDOW : 0;
  int64_t *ctr = step_counters(a);
  double **b0 = buf(0);
  NB_CUDA_TRY(launch_drift(p, v, b0[0], b0[1], b0[2], st));
  count_launches(1);
  for (int64_t s = 0; s < pre; ++s) {
    double **P = buf(s), **Nx = buf(s + 1);
    NB_TRY(pair_forces(pl, mode, n, P[0], P[1], P[2], sys->q, params->soft2, part, split, a->err, st));
    const int64_t snew = sys->step + s + 1;
    int64_t *cout = (windows && s + 1 == pre) ? ctr : nullptr;  // the windows' starting index
    NB_CUDA_TRY(launch_epi_step(p, v, P[0], P[1], P[2], part, pl.n_jc, snew, Nx[0], Nx[1], Nx[2], a->err, st,
                                nullptr, cout, snew));
    count_launches(1);
  }
  if (reps > 0) {
    NvtxRange sub_("nb_step: step windows");
    std::vector<unsigned char> key = window_key(pl, mode, p, v, buf(pre), buf(pre + 1), part, split, a);
    StepGraph *wg = nullptr;
    NB_TRY(find_window(a, key, pl, mode, p, v, buf(pre), buf(pre + 1), part, split, params->soft2, &wg));
    for (int64_t r = 0; r < reps; ++r) NB_CUDA_TRY(cudaGraphLaunch(wg->exec, st));
    count_launches(wg->kernels * (uint64_t)reps);
  }
  double **P = buf(nsteps - 1);
  NB_TRY(pair_forces(pl, mode, n, P[0], P[1], P[2], sys->q, params->soft2, part, split, a->err, st));
  NB_CUDA_TRY(launch_epi_step(p, v, P[0], P[1], P[2], part, pl.n_jc, sys->step + nsteps, nullptr, nullptr, nullptr,
                              a->err, st));
  count_launches(1);
  sys->step += nsteps;
  return NB_OK;
}

nb_status nb_energy(const nb_params *params, const nb_system *sys, double out[4], void *stream) {
  NvtxRange range_("nb_energy");
  NB_TRY(check_params(params));
  NB_TRY(check_system(sys, true, false));
  if (!out) return fail(NB_EINVAL, "out is NULL");
  const int64_t n = sys->n;
  if (n == 0) {
    out[0] = out[1] = out[2] = out[3] = 0.0;
    return NB_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const Plan pl = make_plan(n, MODE_FP64, 1);
  Carver need;
  need.take<double>((size_t)pl.n_jc * n);
  need.take<double>(3 * ENERGY_BLOCKS);
  need.take<double>(4);
  Arena *a = nullptr;
  NB_TRY(get_arena(st, need.off + 256, &a));
  Carver cv;
  cv.base = a->buf;
  double *ppart = cv.take<double>((size_t)pl.n_jc * n);
  double *bpart = cv.take<double>(3 * ENERGY_BLOCKS);
  double *out4 = cv.take<double>(4);
  const Phys p = to_phys(params);
  const StateView v = to_view(sys);
  const double t = params->t0 + (double)sys->step * params->dt;
  NB_CUDA_TRY(launch_pair_phi(pl, n, sys->x, sys->y, sys->z, sys->q, params->charge, params->soft2, ppart, st));
  NB_CUDA_TRY(launch_energy(p, v, ppart, pl.n_jc, t, bpart, out4, st));
  count_launches(3);
  NB_CUDA_TRY(cudaMemcpyAsync(out, out4, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  NB_CUDA_TRY(cudaStreamSynchronize(st));
  return NB_OK;
}

}  // extern "C"

namespace nb {
namespace {

// The view of ions [i0, i1) of a system: pointers offset by i0, n = i1 - i0,
// ion0 = i0 (the global index that keys the Langevin draws).
StateView range_view(const nb_system *sys, int64_t i0, int64_t i1) {
  StateView v = to_view(sys);
  auto off = [&](double *a) { return a ? a + i0 : a; };
  v.n = i1 - i0;
  v.x = off(v.x); v.y = off(v.y); v.z = off(v.z);
  v.vx = off(v.vx); v.vy = off(v.vy); v.vz = off(v.vz);
  v.ax = off(v.ax); v.ay = off(v.ay); v.az = off(v.az);
  v.q = v.q ? v.q + i0 : nullptr;
  v.m = v.m ? v.m + i0 : nullptr;
  v.ion0 = i0;
  return v;
}

nb_status check_range(const nb_system *sys, int64_t i0, int64_t i1) {
  if (i0 < 0 || i1 < i0 || i1 > sys->n) return fail(NB_EINVAL, "range [%lld, %lld) not within [0, %lld)",
                                                    (long long)i0, (long long)i1, (long long)sys->n);
  return NB_OK;
}

// Coulomb sums of ions [i0, i1) from all n ions into `part` (the one-sided
// kernel with the full plan's chunks), the FP32 position split first for
// NB_MIXED_SPLIT.  Returns the plan used.
nb_status range_pair_sums(const nb_params *params, const nb_system *sys, int64_t i0, int64_t i1,
                          cudaStream_t st, Arena **arena, double **part_out, Plan *plan_out) {
  const int64_t n = sys->n, ni = i1 - i0;
  const int mode = params->precision;
  const Plan pl = make_plan(n, mode, 0, false, ni);
  Carver need;
  need.take<double>((size_t)pl.n_jc * 3 * ni);
  if (split_like(mode)) need.take<float>(6 * (size_t)n);
  NB_TRY(get_arena(st, need.off + 256, arena));
  Carver cv;
  cv.base = (*arena)->buf;
  double *part = cv.take<double>((size_t)pl.n_jc * 3 * ni);
  PosF32 pf{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  if (split_like(mode)) {
    float *split = cv.take<float>(6 * (size_t)n);
    NB_CUDA_TRY(launch_split_positions(n, sys->x, sys->y, sys->z, split, st));
    count_launches(1);
    pf = PosF32{split, split + n, split + 2 * n, split + 3 * n, split + 4 * n, split + 5 * n};
  }
  timing_begin(st);
  NB_CUDA_TRY(launch_pair_force_range(pl, mode, n, i0, ni, sys->x, sys->y, sys->z, sys->q, pf, params->soft2,
                                      part, st));
  timing_end(st);
  count_launches(1);
  *part_out = part;
  *plan_out = pl;
  return NB_OK;
}

}  // namespace
}  // namespace nb

extern "C" {

nb_status nb_forces_range(const nb_params *params, const nb_system *sys, int64_t i0, int64_t i1, int flags,
                          void *stream) {
  NvtxRange range_("nb_forces_range");
  NB_TRY(check_params(params));
  NB_TRY(check_system(sys, (flags & NB_ACC_TOTAL) != 0, true));
  if (flags & ~NB_ACC_TOTAL) return fail(NB_EINVAL, "unknown flags 0x%x", flags);
  NB_TRY(check_range(sys, i0, i1));
  if (i1 == i0) return NB_OK;
  cudaStream_t st = (cudaStream_t)stream;
  Arena *a = nullptr;
  double *part = nullptr;
  Plan pl;
  NB_TRY(range_pair_sums(params, sys, i0, i1, st, &a, &part, &pl));
  const double t = params->t0 + (double)sys->step * params->dt;
  NB_CUDA_TRY(launch_epi_forces(to_phys(params), range_view(sys, i0, i1), part, pl.n_jc, flags, t, a->err, st));
  count_launches(1);
  return NB_OK;
}

nb_status nb_step_range_drift(const nb_params *params, nb_system *sys, int64_t i0, int64_t i1, void *stream) {
  NvtxRange range_("nb_step_range_drift");
  NB_TRY(check_params(params));
  NB_TRY(check_system(sys, true, true));
  NB_TRY(check_range(sys, i0, i1));
  if (!(params->dt > 0.0)) return fail(NB_EINVAL, "dt must be > 0");
  if (i1 == i0) return NB_OK;
  const StateView v = range_view(sys, i0, i1);
  NB_CUDA_TRY(launch_drift(to_phys(params), v, v.x, v.y, v.z, (cudaStream_t)stream));
  count_launches(1);
  return NB_OK;
}

nb_status nb_step_range_kick(const nb_params *params, nb_system *sys, int64_t i0, int64_t i1, void *stream) {
  NvtxRange range_("nb_step_range_kick");
  NB_TRY(check_params(params));
  NB_TRY(check_system(sys, true, true));
  NB_TRY(check_range(sys, i0, i1));
  if (!(params->dt > 0.0)) return fail(NB_EINVAL, "dt must be > 0");
  if (i1 > i0) {
    cudaStream_t st = (cudaStream_t)stream;
    Arena *a = nullptr;
    double *part = nullptr;
    Plan pl;
    NB_TRY(range_pair_sums(params, sys, i0, i1, st, &a, &part, &pl));
    const StateView v = range_view(sys, i0, i1);
    NB_CUDA_TRY(launch_epi_step(to_phys(params), v, v.x, v.y, v.z, part, pl.n_jc, sys->step + 1, nullptr, nullptr,
                                nullptr, a->err, st));
    count_launches(1);
  }
  sys->step += 1;
  return NB_OK;
}

nb_status nb_forces_vjp(const nb_params *params, const nb_system *sys, const double *lx,
                        const double *ly, const double *lz, double *gx, double *gy, double *gz,
                        int flags, void *stream) {
  NvtxRange range_("nb_forces_vjp");
  NB_TRY(check_params(params));
  NB_TRY(check_system(sys, false, false));
  if (flags & ~NB_ACC_TOTAL) return fail(NB_EINVAL, "unknown flags 0x%x", flags);
  const int64_t n = sys->n;
  if (n == 0) return NB_OK;
  NB_TRY(check_array(lx, "lx"));
  NB_TRY(check_array(ly, "ly"));
  NB_TRY(check_array(lz, "lz"));
  NB_TRY(check_array(gx, "gx"));
  NB_TRY(check_array(gy, "gy"));
  NB_TRY(check_array(gz, "gz"));
  cudaStream_t st = (cudaStream_t)stream;
  const Plan pl = make_plan(n, MODE_FP64, 2);
  Arena *a = nullptr;
  NB_TRY(get_arena(st, part_doubles(pl, n, 3) * sizeof(double) + 512, &a));
  double *part = reinterpret_cast<double *>(a->buf);
  const Phys p = to_phys(params);
  const StateView v = to_view(sys);
  const double t = params->t0 + (double)sys->step * params->dt;
  NB_CUDA_TRY(launch_pair_vjp(pl, n, sys->x, sys->y, sys->z, sys->q, lx, ly, lz, params->soft2, part, a->err, st));
  NB_CUDA_TRY(launch_epi_vjp(p, v, part, pl.n_jc, lx, ly, lz, gx, gy, gz, flags, t, st));
  count_launches(2);
  return NB_OK;
}

namespace {

// Checks shared by both ensemble calls: the packed system, the instance
// offsets and the step count; `p` is one instance's parameters.
nb_status check_batched(const nb_params *p, int32_t n_inst, const int64_t *offsets,
                        const nb_system *packed, int64_t nsteps) {
  NB_TRY(check_system(packed, true, true));
  if (p->precision != NB_FP64 && p->precision != NB_DF64)
    return fail(NB_ENOTSUP, "the ensemble kernel supports NB_FP64 and NB_DF64");
  if (packed->m) return fail(NB_ENOTSUP, "the ensemble kernel has one species (m must be NULL)");
  if (nsteps < 0) return fail(NB_EINVAL, "nsteps must be >= 0");
  if (!(p->dt > 0.0)) return fail(NB_EINVAL, "dt must be > 0");
  if (n_inst < 0 || n_inst > BATCH_LIMIT_INST)
    return fail(NB_EINVAL, "n_inst must be in [0, %d]", BATCH_LIMIT_INST);
  if (n_inst > 0 && !offsets) return fail(NB_EINVAL, "offsets is NULL");
  if (n_inst > 0) {
    if (offsets[0] != 0 || offsets[n_inst] != packed->n)
      return fail(NB_EINVAL, "offsets must start at 0 and end at n");
    for (int k = 0; k < n_inst; ++k) {
      const int64_t m = offsets[k + 1] - offsets[k];
      if (m < 0) return fail(NB_EINVAL, "offsets must be non-decreasing");
      if (m > BATCH_LIMIT_N)
        return fail(NB_EINVAL, "instance %d has %lld ions, above the ensemble limit %d", k,
                    (long long)m, BATCH_LIMIT_N);
    }
  }
  return NB_OK;
}

// One persistent launch of the ensemble kernel; ptab = nullptr shares `p`.
nb_status run_batched(const nb_params *p, const Phys *ptab, int32_t n_inst, const int64_t *offsets,
                      nb_system *packed, int64_t nsteps, Arena *a, cudaStream_t st) {
  int threads = 512, R = 1, bps = 1;  // fastest on GB300 with the half-pair phase
  tuning_lookup(3, p->precision, packed->n, &threads, &R, &bps);
  const int n_bins = std::min(n_inst, device_sm_count());
  // a tuning entry with R = 0 keeps the one-sided force phase
  NB_CUDA_TRY(launch_batched(to_phys(p), ptab, to_view(packed), n_inst, offsets, n_bins, threads, R != 0,
                             packed->step, nsteps, a->err, st));
  count_launches(1);
  packed->step += nsteps;
  return NB_OK;
}

}  // namespace

nb_status nb_step_batched(const nb_params *params, int32_t n_inst, const int64_t *offsets,
                          nb_system *packed, int64_t nsteps, void *stream) {
  NvtxRange range_("nb_step_batched");
  NB_TRY(check_params(params));
  NB_TRY(check_batched(params, n_inst, offsets, packed, nsteps));
  if (n_inst == 0 || packed->n == 0 || nsteps == 0) {
    packed->step += nsteps;
    return NB_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  Arena *a = nullptr;
  NB_TRY(get_arena(st, 256, &a));
  return run_batched(params, nullptr, n_inst, offsets, packed, nsteps, a, st);
}

nb_status nb_step_batched_each(const nb_params *per_inst, int32_t n_inst, const int64_t *offsets,
                               nb_system *packed, int64_t nsteps, void *stream) {
  NvtxRange range_("nb_step_batched_each");
  if (n_inst < 0 || n_inst > BATCH_LIMIT_INST)
    return fail(NB_EINVAL, "n_inst must be in [0, %d]", BATCH_LIMIT_INST);
  if (n_inst > 0 && !per_inst) return fail(NB_EINVAL, "per_inst is NULL");
  for (int k = 0; k < n_inst; ++k) {
    const nb_status rc = check_params(&per_inst[k]);
    if (rc != NB_OK) return fail(rc, "per_inst[%d]: %s", k, g_last_error.c_str());
    if (per_inst[k].precision != per_inst[0].precision)
      return fail(NB_EINVAL, "per_inst[%d].precision differs from per_inst[0]'s", k);
    if (!(per_inst[k].dt > 0.0)) return fail(NB_EINVAL, "per_inst[%d].dt must be > 0", k);
  }
  nb_params shape{};  // stands in for the instances' common fields when n_inst == 0
  shape.precision = n_inst > 0 ? per_inst[0].precision : NB_FP64;
  shape.dt = 1.0;
  NB_TRY(check_batched(&shape, n_inst, offsets, packed, nsteps));
  if (n_inst == 0 || packed->n == 0 || nsteps == 0) {
    packed->step += nsteps;
    return NB_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  Arena *a = nullptr;
  NB_TRY(get_arena(st, 256, &a));
  const bool same = a->ptab && a->ptab_src.size() == (size_t)n_inst &&
                    std::memcmp(a->ptab_src.data(), per_inst, n_inst * sizeof(nb_params)) == 0;
  if (!same) {
    // a graph capture records the launch, which reads the table at replay
    // time; a host-to-device copy of new contents is not captured
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    NB_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone)
      return fail(NB_EINVAL, "per-instance parameters differ from the stream's last uncaptured call; "
                             "make one uncaptured call with them before capturing");
    if (!a->ptab && cudaMalloc(&a->ptab, BATCH_LIMIT_INST * sizeof(Phys)) != cudaSuccess) {
      cudaGetLastError();
      a->ptab = nullptr;
      return fail(NB_ENOMEM, "cudaMalloc(per-instance parameter table) failed");
    }
    a->ptab_stage.resize(n_inst);
    for (int k = 0; k < n_inst; ++k) a->ptab_stage[k] = to_phys(&per_inst[k]);
    // pageable source: the call returns once the bytes are staged; the copy
    // to the device is ordered after the stream's earlier work, which may
    // still read the old table
    NB_CUDA_TRY(cudaMemcpyAsync(a->ptab, a->ptab_stage.data(), n_inst * sizeof(Phys),
                                cudaMemcpyHostToDevice, st));
    a->ptab_src.assign(per_inst, per_inst + n_inst);
  }
  return run_batched(&per_inst[0], a->ptab, n_inst, offsets, packed, nsteps, a, st);
}

nb_status nb_plan_batched(int32_t n_inst, const int64_t *offsets, int32_t n_bins,
                          uint16_t *order, uint16_t *bin_start, double *max_load,
                          double *mean_load) {
  if (n_inst < 0 || n_inst > BATCH_LIMIT_INST || n_bins < 1 || n_bins > BATCH_LIMIT_INST)
    return fail(NB_EINVAL, "n_inst must be in [0, %d] and n_bins in [1, %d]", BATCH_LIMIT_INST,
                BATCH_LIMIT_INST);
  if (!offsets || !order || !bin_start) return fail(NB_EINVAL, "NULL argument");
  for (int k = 0; k < n_inst; ++k)
    if (offsets[k + 1] < offsets[k]) return fail(NB_EINVAL, "offsets must be non-decreasing");
  batched_plan(n_inst, offsets, n_bins, order, bin_start, max_load, mean_load);
  return NB_OK;
}

nb_status nb_plan_info(int32_t kind, int32_t precision, int64_t n, int64_t out[8]) {
  if (!out) return fail(NB_EINVAL, "out is NULL");
  if (kind < 0 || kind > 2) return fail(NB_EINVAL, "kind must be 0 (force), 1 (potential) or 2 (VJP)");
  if (precision < NB_FP64 || precision > NB_MIXED_SPLIT_RSQ) return fail(NB_EINVAL, "bad precision");
  if (n < 1) return fail(NB_EINVAL, "n must be >= 1");
  const Plan pl = make_plan(n, kind == 0 ? precision : MODE_FP64, kind);
  out[0] = pl.block;
  out[1] = pl.R;
  out[2] = pl.jchunk;
  out[3] = pl.sym ? pl.nbk : pl.n_it;
  out[4] = pl.n_jc;
  out[5] = pl.sym;
  out[6] = pl.G;
  out[7] = kind == 0 && use_small_steps(pl, precision, n) ? 1 : 0;
  return NB_OK;
}

nb_status nb_sym_schedule(int32_t nbk, int32_t *P, int32_t *Q, int32_t *round) {
  if (nbk < 1 || nbk > 60000) return fail(NB_EINVAL, "nbk must be in 1..60000");
  if (!P || !Q || !round) return fail(NB_EINVAL, "output arrays must not be NULL");
  const int64_t items = (int64_t)nbk * (nbk + 1) / 2;
  for (int64_t t = 0; t < items; ++t) {
    const SymItem it = sym_item((int)t, nbk);
    P[t] = it.P;
    Q[t] = it.Q;
    round[t] = it.round;
  }
  return NB_OK;
}

nb_status nb_set_tuning(int32_t kind, int32_t precision, int64_t n_lo, int64_t n_hi, int32_t block,
                        int32_t R, int32_t blocks_per_sm) {
  if (block == 0) {
    tuning_clear();
    return NB_OK;
  }
  if (kind < 0 || kind > 8) return fail(NB_EINVAL, "kind must be 0..8");
  if (precision < NB_FP64 || precision > NB_MIXED_SPLIT_RSQ) return fail(NB_EINVAL, "bad precision");
  if (n_lo < 0 || n_hi < n_lo) return fail(NB_EINVAL, "bad n range");
  if (kind == 4) {
    if (block != 32 && block != 64 && block != 128 && block != 256 && block != 512 && block != 1024)
      return fail(NB_EINVAL, "symmetric block must be 32, 64, 128, 256, 512 or 1024 ions");
    if (R != 0 && R != 1) return fail(NB_EINVAL, "R must be 1 (use) or 0 (disable)");
  } else if (kind == 5) {
    if (block != 128 && block != 256) return fail(NB_EINVAL, "symmetric VJP block must be 128 or 256 ions");
    if (R != 0 && R != 1) return fail(NB_EINVAL, "R must be 1 (use) or 0 (disable)");
  } else if (kind == 8) {
    if (block < 1) return fail(NB_EINVAL, "block must be >= 1 (it is not used)");
    if (R != 0 && R != 1) return fail(NB_EINVAL, "R must be 1 (eight lanes) or 0 (one lane)");
  } else if (kind == 7) {
    if (block < 1) return fail(NB_EINVAL, "block must be >= 1 (it is not used)");
    if (R != 0 && R != 1) return fail(NB_EINVAL, "R must be 1 (use) or 0 (disable)");
  } else if (kind == 6) {
    if (block < 1) return fail(NB_EINVAL, "block (the least nsteps) must be >= 1");
    if (R != 0 && R != 1) return fail(NB_EINVAL, "R must be 1 (use) or 0 (disable)");
  } else if (kind == 3) {
    if (block < 32 || block > 512 || block % 32) return fail(NB_EINVAL, "block must be 32..512, a multiple of 32");
  } else {
    if (block != 32 && block != 64 && block != 128 && block != 256)
      return fail(NB_EINVAL, "block must be 32, 64, 128 or 256");
    if (R != 1 && R != 2 && R != 4) return fail(NB_EINVAL, "R must be 1, 2 or 4");
    if (kind != 0 && R != 1) return fail(NB_EINVAL, "R > 1 is for the force kernel only");
    if (blocks_per_sm < 1 || blocks_per_sm > 256) return fail(NB_EINVAL, "blocks_per_sm must be 1..256");
  }
  tuning_set(kind, precision, n_lo, n_hi, block, R, blocks_per_sm);
  return NB_OK;
}

// ---------------------------------------------------------------------------
// Trajectory loss and adjoint gradient (static harmonic trap, no friction or
// noise, FP64 pair arithmetic).

namespace nb {
namespace {

nb_status check_adjoint(const nb_params *p) {
  NB_TRY(check_params(p));
  if (p->trap != NB_TRAP_HARMONIC || p->gamma != 0.0 || p->noise_T != 0.0 ||
      p->omega_rate[0] != 0.0 || p->omega_rate[1] != 0.0 || p->omega_rate[2] != 0.0)
    return fail(NB_ENOTSUP, "the trajectory adjoint supports the static harmonic trap without friction or noise");
  if (p->precision != NB_FP64 && p->precision != NB_DF64)
    return fail(NB_ENOTSUP, "the trajectory adjoint takes NB_FP64 or NB_DF64 force arithmetic");
  if (!(p->dt > 0.0)) return fail(NB_EINVAL, "dt must be > 0");
  return NB_OK;
}

int64_t n_segments(int64_t nsteps, int64_t every) {
  return nsteps == 0 ? 1 : (nsteps + every - 1) / every;
}

}  // namespace
}  // namespace nb

extern "C" int64_t nb_traj_ckpt_doubles(int64_t n, int64_t nsteps, int64_t every) {
  if (n < 0 || nsteps < 0 || every < 1) return -1;
  return n_segments(nsteps, every) * 9 * n;
}

extern "C" nb_status nb_traj_forward(const nb_params *params, nb_system *sys, int64_t nsteps,
                                     int64_t every, double *ckpt, const double *target, double *loss,
                                     void *stream) {
  NvtxRange range_("nb_traj_forward");
  NB_TRY(check_adjoint(params));
  NB_TRY(check_system(sys, true, true));
  if (sys->m) return fail(NB_ENOTSUP, "the trajectory adjoint has one species (m must be NULL)");
  if (nsteps < 0 || every < 1) return fail(NB_EINVAL, "nsteps must be >= 0 and every >= 1");
  const int64_t n = sys->n;
  if (n == 0) return fail(NB_EINVAL, "the trajectory loss needs n >= 1");
  NB_TRY(check_array(ckpt, "ckpt"));
  NB_TRY(check_array(target, "target"));
  NB_TRY(check_array(loss, "loss"));
  cudaStream_t st = (cudaStream_t)stream;
  NB_TRY(nb_forces(params, sys, nullptr, NB_ACC_TOTAL, stream));
  const int64_t S = n_segments(nsteps, every);
  const size_t N8 = (size_t)n * sizeof(double);
  for (int64_t seg = 0; seg < S; ++seg) {
    double *c = ckpt + (size_t)seg * 9 * n;
    double *src[9] = {sys->x, sys->y, sys->z, sys->vx, sys->vy, sys->vz, sys->ax, sys->ay, sys->az};
    for (int k = 0; k < 9; ++k)
      NB_CUDA_TRY(cudaMemcpyAsync(c + (size_t)k * n, src[k], N8, cudaMemcpyDeviceToDevice, st));
    const int64_t len = std::min(every, nsteps - seg * every);
    if (len > 0) NB_TRY(nb_step(params, sys, len, stream));
  }
  const Plan plp = make_plan(n, MODE_FP64, 1);
  Carver need;
  need.take<double>((size_t)plp.n_jc * n);
  need.take<double>(ADJ_PART_BLOCKS);
  Arena *a = nullptr;
  NB_TRY(get_arena(st, need.off + 256, &a));
  Carver cv;
  cv.base = a->buf;
  double *ppart = cv.take<double>((size_t)plp.n_jc * n);
  double *bpart = cv.take<double>(ADJ_PART_BLOCKS);
  const double *xT[3] = {sys->x, sys->y, sys->z};
  const double *tg[3] = {target, target + n, target + 2 * n};
  NB_CUDA_TRY(launch_pair_phi(plp, n, sys->x, sys->y, sys->z, sys->q, params->charge, params->soft2, ppart, st));
  NB_CUDA_TRY(launch_loss(to_phys(params), n, sys->q, xT, tg, ppart, plp.n_jc, bpart, loss, st));
  count_launches(3);
  return NB_OK;
}

extern "C" nb_status nb_traj_backward(const nb_params *params, const nb_system *sys, int64_t nsteps,
                                      int64_t every, const double *ckpt, const double *target,
                                      const double *gscale, double *gx0, double *gv0, double *gomega,
                                      void *stream) {
  NvtxRange range_("nb_traj_backward");
  NB_TRY(check_adjoint(params));
  if (!sys) return fail(NB_EINVAL, "system is NULL");
  if (sys->m) return fail(NB_ENOTSUP, "the trajectory adjoint has one species (m must be NULL)");
  if (nsteps < 0 || every < 1) return fail(NB_EINVAL, "nsteps must be >= 0 and every >= 1");
  const int64_t n = sys->n;
  if (n < 1) return fail(NB_EINVAL, "the trajectory loss needs n >= 1");
  if (sys->q && !aligned8(sys->q)) return fail(NB_EINVAL, "q is not 8-byte aligned");
  NB_TRY(check_array(ckpt, "ckpt"));
  NB_TRY(check_array(target, "target"));
  NB_TRY(check_array(gx0, "gx0"));
  NB_TRY(check_array(gv0, "gv0"));
  NB_TRY(check_array(gomega, "gomega"));
  if (gscale && !aligned8(gscale)) return fail(NB_EINVAL, "gscale is not 8-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  const int mode = params->precision;  // the forward's force arithmetic, for the recompute
  const Plan pl = make_plan(n, mode, 0);
  const Plan plv = make_plan(n, MODE_FP64, 2);
  const int64_t S = n_segments(nsteps, every);
  const int64_t slots = std::min(every, std::max<int64_t>(nsteps, 1)) + 2;
  Carver need;
  need.take<double>((size_t)slots * 3 * n);
  need.take<double>(18 * (size_t)n);
  need.take<double>(part_doubles(pl, n, 3));
  need.take<double>(part_doubles(plv, n, 3));
  need.take<double>(3 * ADJ_PART_BLOCKS);
  Arena *a = nullptr;
  NB_TRY(get_arena(st, need.off + 256, &a));
  Carver cv;
  cv.base = a->buf;
  double *segbuf = cv.take<double>((size_t)slots * 3 * n);
  double *st18 = cv.take<double>(18 * (size_t)n);
  double *fpart = cv.take<double>(part_doubles(pl, n, 3));
  double *vpart = cv.take<double>(part_doubles(plv, n, 3));
  double *bpart = cv.take<double>(3 * ADJ_PART_BLOCKS);
  auto arr3 = [&](double *base) { return std::array<double *, 3>{base, base + n, base + 2 * n}; };
  const auto v3 = arr3(st18), a3 = arr3(st18 + 3 * n), xb = arr3(st18 + 6 * n), vb = arr3(st18 + 9 * n),
             ab = arr3(st18 + 12 * n), wacc = arr3(st18 + 15 * n);
  auto slot = [&](int64_t k) { return arr3(segbuf + (size_t)k * 3 * n); };
  const double *tg[3] = {target, target + n, target + 2 * n};
  const Phys p = to_phys(params);
  const size_t N8 = (size_t)n * sizeof(double);
  PosF32 nopf{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  for (int64_t seg = S - 1; seg >= 0; --seg) {
    const int64_t start = seg * every;
    const int64_t len = std::min(every, nsteps - start);
    const double *c = ckpt + (size_t)seg * 9 * n;
    const auto s0 = slot(0);
    for (int k = 0; k < 3; ++k) {
      NB_CUDA_TRY(cudaMemcpyAsync(s0[k], c + (size_t)k * n, N8, cudaMemcpyDeviceToDevice, st));
      NB_CUDA_TRY(cudaMemcpyAsync(v3[k], c + (size_t)(3 + k) * n, N8, cudaMemcpyDeviceToDevice, st));
      NB_CUDA_TRY(cudaMemcpyAsync(a3[k], c + (size_t)(6 + k) * n, N8, cudaMemcpyDeviceToDevice, st));
    }
    // recompute the segment from the checkpointed state (x, v, a): positions of
    // steps start .. start+len into slots 0 .. len, bitwise as in the forward
    StateView sv;
    sv.n = n;
    sv.x = s0[0]; sv.y = s0[1]; sv.z = s0[2];
    sv.vx = v3[0]; sv.vy = v3[1]; sv.vz = v3[2];
    sv.ax = a3[0]; sv.ay = a3[1]; sv.az = a3[2];
    sv.q = sys->q;
    if (len > 0) {
      const auto s1 = slot(1);
      NB_CUDA_TRY(launch_drift(p, sv, s1[0], s1[1], s1[2], st));
      count_launches(1);
      for (int64_t m = 0; m < len; ++m) {
        const auto P = slot(m + 1), Nx = slot(m + 2);
        NB_CUDA_TRY(launch_pair_force(pl, mode, n, P[0], P[1], P[2], sys->q, nopf, params->soft2, fpart, a->err, st));
        NB_CUDA_TRY(launch_epi_step(p, sv, P[0], P[1], P[2], fpart, pl.n_jc, start + m + 1, Nx[0], Nx[1], Nx[2],
                                    a->err, st));
        count_launches(2);
      }
    }
    if (seg == S - 1) {
      const auto sT = slot(len);
      const double *xT[3] = {sT[0], sT[1], sT[2]};
      const double *aT[3] = {a3[0], a3[1], a3[2]};
      NB_CUDA_TRY(launch_adj_init(p, n, xT, aT, tg, xb.data(), vb.data(), ab.data(), wacc.data(), st));
      count_launches(1);
    }
    // reverse sweep over the segment
    for (int64_t m = len - 1; m >= 0; --m) {
      const auto X = slot(m + 1);
      NB_CUDA_TRY(launch_pair_vjp(plv, n, X[0], X[1], X[2], sys->q, ab[0], ab[1], ab[2], params->soft2, vpart, a->err,
                                  st));
      const double *xc[3] = {X[0], X[1], X[2]};
      NB_CUDA_TRY(launch_adj_epi(p, n, sys->q, xc, vpart, plv.n_jc, xb.data(), vb.data(), ab.data(),
                                 wacc.data(), 0, (start + m) >= 1 ? 1 : 0, st));
      count_launches(2);
    }
  }
  // x_0 term: J(x_0)^T ab_0 (slot 0 holds x_0 after segment 0's recompute)
  const auto X0 = slot(0);
  NB_CUDA_TRY(launch_pair_vjp(plv, n, X0[0], X0[1], X0[2], sys->q, ab[0], ab[1], ab[2], params->soft2, vpart, a->err,
                              st));
  const double *x0c[3] = {X0[0], X0[1], X0[2]};
  NB_CUDA_TRY(launch_adj_epi(p, n, sys->q, x0c, vpart, plv.n_jc, xb.data(), vb.data(), ab.data(), wacc.data(),
                             1, 0, st));
  NB_CUDA_TRY(launch_adj_out(n, xb.data(), vb.data(), wacc.data(), gscale, gx0, gv0, gomega, bpart, st));
  count_launches(4);
  return NB_OK;
}

nb_status nb_sym_wait_probe(int32_t committed, int32_t round, int32_t *ok, void *stream) {
  if (!ok) return fail(NB_EINVAL, "ok is NULL");
  if (committed < 0 || round < 0) return fail(NB_EINVAL, "committed and round must be >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  Arena *a = nullptr;
  NB_TRY(get_arena(st, 256, &a));
  int *sync = reinterpret_cast<int *>(a->buf);
  int *dev_ok = sync + 2;
  NB_CUDA_TRY(launch_sym_wait_probe(sync, committed, round, a->err, dev_ok, st));
  count_launches(1);
  int h = 0;
  NB_CUDA_TRY(cudaMemcpyAsync(&h, dev_ok, sizeof(int), cudaMemcpyDeviceToHost, st));
  NB_CUDA_TRY(cudaStreamSynchronize(st));
  *ok = h;
  return NB_OK;
}

nb_status nb_sync_status(void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  NB_CUDA_TRY(cudaStreamSynchronize(st));
  int dev = 0;
  NB_CUDA_TRY(cudaGetDevice(&dev));
  unsigned *err = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_arenas.find(std::make_pair(dev, st));
    if (it == g_arenas.end() || !it->second.err) return NB_OK;
    err = it->second.err;
  }
  unsigned h = 0;
  NB_CUDA_TRY(cudaMemcpy(&h, err, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (h) NB_CUDA_TRY(cudaMemset(err, 0, sizeof(unsigned)));
  if (h & ERR_TIMEOUT) return fail(NB_ETIMEOUT, "a bounded device wait gave up");
  if (h & ERR_NONFINITE) return fail(NB_ENONFINITE, "a non-finite acceleration or velocity was produced");
  return NB_OK;
}

nb_status nb_release(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  int cur = 0;
  cudaGetDevice(&cur);
  nb_status rc = NB_OK;
  for (auto &kv : g_arenas) {
    if (cudaSetDevice(kv.first.first) != cudaSuccess) { rc = NB_ECUDA; continue; }
    cudaDeviceSynchronize();
    for (StepGraph &g : kv.second.windows)
      if (g.exec && cudaGraphExecDestroy(g.exec) != cudaSuccess) rc = NB_ECUDA;
    if (kv.second.cap_st && cudaStreamDestroy(kv.second.cap_st) != cudaSuccess) rc = NB_ECUDA;
    if (kv.second.buf && cudaFree(kv.second.buf) != cudaSuccess) rc = NB_ECUDA;
    if (kv.second.ptab && cudaFree(kv.second.ptab) != cudaSuccess) rc = NB_ECUDA;
    if (kv.second.err && cudaFree(kv.second.err) != cudaSuccess) rc = NB_ECUDA;
  }
  g_arenas.clear();
  cudaSetDevice(cur);
  if (rc != NB_OK) fail(rc, "freeing scratch failed");
  return rc;
}

const char *nb_strerror(nb_status status) {
  switch (status) {
    case NB_OK: return "success";
    case NB_EINVAL: return "invalid argument";
    case NB_ECUDA: return "CUDA runtime error";
    case NB_ENONFINITE: return "non-finite acceleration or velocity";
    case NB_ETIMEOUT: return "device-side wait timed out";
    case NB_ENOMEM: return "out of device memory";
    case NB_ENOTSUP: return "not supported";
  }
  return "unknown status";
}

const char *nb_last_error(void) { return g_last_error.c_str(); }

const char *nb_version(void) { return "nb-gb300 0.1 (sm_103a)"; }

uint64_t nb_launch_count(void) { return g_launches.load(); }

nb_status nb_timing_enable(int64_t capacity) {
  if (capacity < 0) return fail(NB_EINVAL, "capacity must be >= 0");
  std::lock_guard<std::mutex> lk(g_tmu);
  for (cudaEvent_t e : g_ev) cudaEventDestroy(e);
  g_ev.clear();
  g_ev_cap = g_ev_used = 0;
  for (int64_t k = 0; k < 2 * capacity; ++k) {
    cudaEvent_t e;
    NB_CUDA_TRY(cudaEventCreate(&e));
    g_ev.push_back(e);
  }
  g_ev_cap = capacity;
  return NB_OK;
}

nb_status nb_timing_read(int64_t *launches, double *total_ms) {
  if (!launches || !total_ms) return fail(NB_EINVAL, "NULL output");
  std::lock_guard<std::mutex> lk(g_tmu);
  double tot = 0.0;
  for (int64_t k = 0; k < g_ev_used; ++k) {
    float ms = 0.0f;
    NB_CUDA_TRY(cudaEventSynchronize(g_ev[2 * k + 1]));
    NB_CUDA_TRY(cudaEventElapsedTime(&ms, g_ev[2 * k], g_ev[2 * k + 1]));
    tot += ms;
  }
  *launches = g_ev_used;
  *total_ms = tot;
  g_ev_used = 0;
  return NB_OK;
}

}  // extern "C"
