/*
 * nb.h -- C ABI of libnb.so, a GB300 (sm_103a) library for the direct
 * N-body problem of laser-cooled trapped ions, after Pedregosa-Gutierrez &
 * Dempsey, "Direct N-Body problem optimisation using the AVX-512
 * instruction set" (arXiv 2106.11143).
 *
 * Conventions for every entry point
 * ---------------------------------
 *  - Units are SI.  Arrays are structure-of-arrays (SoA), float64, one value
 *    per ion, contiguous, 8-byte aligned, and live in DEVICE memory of the
 *    current CUDA device unless the argument says "host".  The caller owns
 *    every array it passes; the library never frees or keeps caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous with respect to the host on that
 *    stream unless stated otherwise.
 *  - Scratch memory (pair partial sums, the second position buffer, block
 *    partials, a device error word) belongs to the library.  It is
 *    allocated with cudaMalloc on first use, per (device, stream), grown on
 *    demand, reused by later calls on the same stream, and freed by
 *    nb_release().  Calls on the same stream are ordered; calls on
 *    different streams use different scratch.
 *  - Host threads: the entry points may be called from several host
 *    threads (the scratch registry and the tuning table are locked inside
 *    the library), but calls that share a stream must come from one thread
 *    at a time: any call may regrow that stream's scratch, after
 *    synchronising the stream, while another thread is still enqueuing work
 *    that uses the old buffer.  nb_release() must not overlap any other call.
 *  - Every call validates its arguments on the host first and returns
 *    NB_EINVAL without enqueuing any work if they are wrong.  Numerical
 *    failures on the device (a non-finite acceleration or velocity) are
 *    recorded in the stream's device error word and reported by the next
 *    nb_sync_status() on that stream; the state is then undefined.
 *  - n == 0 is valid and does nothing.
 *  - Results are deterministic: identical inputs and launch configuration
 *    give bitwise-identical outputs (fixed, atomic-free summation order).
 */
#ifndef NB_H
#define NB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NB_OK = 0,
  NB_EINVAL = 1,      /* invalid argument (null pointer, bad size, bad enum) */
  NB_ECUDA = 2,       /* a CUDA runtime call failed; see nb_last_error() */
  NB_ENONFINITE = 3,  /* a non-finite acceleration or velocity was produced */
  NB_ETIMEOUT = 4,    /* a bounded device-side wait gave up */
  NB_ENOMEM = 5,      /* scratch allocation failed */
  NB_ENOTSUP = 6      /* a valid request the library does not support */
} nb_status;

/* Arithmetic of the pair interaction (the O(N^2) inner loop).
 *  NB_FP64       -- FP64 displacement and FP64 accumulation of the forces.
 *                   In between, r^2, 1/sqrt(r^2) and r^-3 run on the FP32
 *                   pipe: the displacement is split into exponent-scaled
 *                   FP32 (hi, lo) pairs, r^2 is a double-float, the FP32
 *                   hardware reciprocal square root (MUFU) is refined by a
 *                   Newton residual formed in compensated FP32 (Sec. IV:
 *                   approximate 1/sqrt refined by Newton-Raphson), and one
 *                   FP64 add widens r^-3.  This is FP64-class, not IEEE FP64
 *                   per pair: r^-3 carries a relative error of up to 1.1e-13
 *                   (about 500 ulp; measured over displacements from 1 nm to
 *                   1 km and every exponent) where an IEEE FP64 evaluation
 *                   would be within a few ulp.  Forces meet the 1e-12
 *                   conditioned-error contract (measured 3.4e-14 at
 *                   N = 1e5).  NB_FP64_RSQ_NR2 is the plain FP64 Newton form.
 *  NB_MIXED      -- pair displacements in FP64, cast to FP32; r^2, rsqrt,
 *                   r^-3 and the products in FP32; per-tile FP32 partial
 *                   sums added into FP64 accumulators with compensation.
 *  NB_MIXED_SPLIT -- as NB_MIXED, but each position is carried as an FP32
 *                   (hi, lo) pair built from the FP64 value once per call,
 *                   and the displacement is (hi_i - hi_j) + (lo_i - lo_j)
 *                   in FP32: the FP64 difference, formed from the 48 bits
 *                   the pair keeps, then rounded once to FP32 (hi_i - hi_j
 *                   is exact for close pairs, the lo terms add the low
 *                   bits).  Same accuracy class as NB_MIXED while the
 *                   coordinates are not much larger than the separations:
 *                   the displacement error is about 2^-48 |r| beyond the
 *                   FP32 rounding (relative 2^-48 |r| / |r_i - r_j|, 1e-6 at
 *                   |r| / |r_i - r_j| ~ 3e8).  No FP64 instruction in the
 *                   pair loop.
 *  NB_DF64       -- FP64-class accuracy from FP32 arithmetic: FP64
 *                   displacement split into an FP32 (hi, lo) pair; r^2,
 *                   r^-3 and the force products as double-floats (FP32
 *                   pairs with exact products and TwoSum); per-tile
 *                   double-float sums added in FP64.  Per-pair relative
 *                   error about 2^-44.  Needs |r_i - r_j| >= 2.3e-13 and
 *                   r^2 within the FP32 normal range (SI ion-trap scales).
 * The 1/sqrt ladder of the paper (Sec. IV-VI), FP64 pair arithmetic with
 * r^-3 = y^3 and y from:
 *  NB_FP64_SQRTDIV -- 1.0 / sqrt(r^2) (the classical loop, "SQRT+DIV")
 *  NB_FP64_RSQ     -- the FP32 hardware seed alone (relative error ~2^-22;
 *                     the GPU counterpart of RSQRT14)
 *  NB_FP64_RSQ_NR1 -- seed + one Newton-Raphson step y (3 - r^2 y^2)/2
 *  NB_FP64_RSQ_NR2 -- seed + two Newton-Raphson steps
 * and on the FP32 path of NB_MIXED_SPLIT:
 *  NB_MIXED_SPLIT_RSQ -- NB_MIXED_SPLIT with r^-3 the cube of the bare FP32
 *                     seed (no correction; the GPU counterpart of RSQRT14
 *                     alone on the FP32 path): relative error of r^-3 about
 *                     3.7e-7 from the seed (3 x 2^-22.9) plus FP32 rounding,
 *                     inside the 1e-6 mixed-precision contract; three fewer
 *                     FP32 instructions per pair.
 * Positions, velocities, the integrator and energies are FP64 in all modes. */
typedef enum {
  NB_FP64 = 0,
  NB_MIXED = 1,
  NB_MIXED_SPLIT = 2,
  NB_DF64 = 3,
  NB_FP64_SQRTDIV = 4,
  NB_FP64_RSQ = 5,
  NB_FP64_RSQ_NR1 = 6,
  NB_FP64_RSQ_NR2 = 7,
  NB_MIXED_SPLIT_RSQ = 8
} nb_precision;

/* Confinement (Eq. 1 of the paper).
 *  NB_TRAP_HARMONIC -- static pseudopotential: a_k = -omega_k(t)^2 x_k.
 *  NB_TRAP_RF       -- linear Paul trap with Mathieu a = 0 and q = q_mathieu:
 *                      a_x = -(q Omega^2/2) cos(Omega t + phase) x,
 *                      a_y = +(q Omega^2/2) cos(Omega t + phase) y,
 *                      a_z = -omega_z(t)^2 z  (omega_z = omega[2]).       */
typedef enum { NB_TRAP_HARMONIC = 0, NB_TRAP_RF = 1 } nb_trap;

typedef struct nb_params {
  double k_coulomb;     /* 1/(4 pi eps0) */
  double mass;          /* kg, one species (Sec. II) */
  double charge;        /* C, charge of every ion when nb_system.q is NULL */
  double soft2;         /* softening eps^2 added to r^2 (m^2); 0 = none */
  int32_t trap;         /* nb_trap */
  int32_t precision;    /* nb_precision */
  double omega[3];      /* rad/s at t = 0 */
  double omega_rate[3]; /* rad/s^2: omega_k(t) = omega[k] + omega_rate[k] t */
  double q_mathieu;     /* RF Mathieu q */
  double omega_rf;      /* RF angular frequency Omega (rad/s) */
  double rf_phase;      /* rad */
  double gamma;         /* friction coefficient Gamma (kg/s), Eq. 1 */
  double dt;            /* time step (s) */
  double t0;            /* time of step 0: t = t0 + step * dt */
  double noise_T;       /* Langevin temperature (K); 0 = no noise */
  uint64_t seed;        /* Philox4x32-10 key for the Langevin noise */
  uint32_t instance;    /* ensemble member index (noise counter word) */
  uint32_t reserved;    /* must be 0 */
} nb_params;

typedef struct nb_system {
  int64_t n;            /* number of ions */
  double *x, *y, *z;    /* positions (m), device */
  double *vx, *vy, *vz; /* velocities (m/s), device */
  double *ax, *ay, *az; /* acceleration (m/s^2), device: the Verlet state */
  const double *q;      /* per-ion charge (C), device, or NULL = params.charge */
  int64_t step;         /* step counter; time t = t0 + step * dt */
  const double *m;      /* per-ion mass (kg), device, or NULL = params.mass.
                           With several species (Sec. II: 1-1, 2-2 and 1-2
                           interactions in one all-pairs sum), the trap's field
                           is that of params (charge, mass): ion i's trap
                           acceleration is scaled by (q_i/m_i)/(charge/mass),
                           its friction is -(gamma/m_i) v_i and its Langevin
                           kick uses m_i.  Not supported by nb_step_batched and
                           nb_traj_* (NB_ENOTSUP). */
} nb_system;

/* nb_forces flags */
#define NB_ACC_COULOMB 0 /* write the Coulomb acceleration only */
#define NB_ACC_TOTAL 1   /* Coulomb + trap(t) - (gamma/m) v: the Verlet state */

/* Acceleration of every ion (Eq. 1; the Sec. III pair loop):
 *   a_i = k_C q_i / m * sum_{j != i} q_j (r_i - r_j) / (|r_i - r_j|^2 + soft2)^{3/2}
 * plus, with NB_ACC_TOTAL, the trap term at t = t0 + step*dt and the friction
 * -(gamma/m) v.  Writes sys->ax/ay/az.  The pair arithmetic follows
 * params->precision.  If phi is non-NULL (device, n doubles) it receives the
 * potential sum_{j != i} q_j / sqrt(r_ij^2 + soft2) (FP64; no k_C factor).
 * Two distinct ions at the same position with soft2 == 0 contribute nothing
 * to each other (the self-pair rule applied to r == 0).                   */
nb_status nb_forces(const nb_params *params, const nb_system *sys, double *phi,
                    int flags, void *stream);

/* nsteps velocity-Verlet steps (Sec. II):
 *   r+ = r + v dt + a dt^2/2;  a+ = a(r+, t+dt);  v+ = v + (a + a+) dt/2.
 * The friction part of a+ depends on v+; the velocity update is solved for it
 * exactly: v+ = (v + (a + a+_cons) dt/2) / (1 + gamma dt/(2m)), and the stored
 * a+ = a+_cons - (gamma/m) v+.  With noise_T > 0 a Langevin kick
 * sqrt(2 gamma kB T dt)/m * xi is added to v+, xi ~ N(0,1) per component from
 * Philox4x32-10 with key `seed` and counter {ion, step, step >> 32, instance}
 * (step of the new state), via Box-Muller.
 * On entry sys->a must hold the total acceleration at the current state (call
 * nb_forces with NB_ACC_TOTAL once after setting positions/velocities).
 * Updates x, v, a in place and advances sys->step by nsteps.  Per step one
 * pair-force launch and one epilogue launch (which also performs the next
 * drift), plus the FP32 position split for NB_MIXED_SPLIT; one drift launch
 * per call; no host synchronisation.
 * Small systems: up to n = 48 ions (NB_DF64), 16 (NB_FP64_SQRTDIV) or 32
 * (the other precisions) -- nb_set_tuning kind 7
 * changes the bounds, up to 512 ions and 227 KB of shared memory -- the call
 * runs in one thread block: one launch per min(16384, max(64, 2^28/n^2))
 * steps, positions in shared memory, the one-sided plan's pair items and
 * chunk sums, and the same kick and drift, so the results are bitwise those
 * of the multi-kernel steps.
 * Step windows: for larger n up to 4096 and nsteps >= 32 (nb_set_tuning kind 6
 * changes both), the middle steps of the call run as replays of one CUDA
 * graph of 8 steps, captured on a private stream at the first such call for
 * a given set of kernel arguments (system arrays, parameters, plan) and kept
 * for reuse (up to four per stream, the least recently used replaced by a
 * new capture); the epilogues then read the
 * step index from two counters in the stream's scratch.  The replays run
 * the same kernels on the same data in the same order on `stream`, so the
 * results are bitwise those of plain launches.  They are not used while `stream` is
 * itself being captured or while nb_timing_enable has event pairs left. */
nb_status nb_step(const nb_params *params, nb_system *sys, int64_t nsteps,
                  void *stream);

/* ---- i-range sharding (Sec. VI.C's static ownership of target ions) ----
 * One rank (one GPU) owns the ions [i0, i1) of the system; every rank holds
 * all n positions.  A velocity-Verlet step of nb_step is split around the
 * one exchange it needs:
 *   nb_step_range_drift   r_i += v_i dt + a_i dt^2/2 for the owned ions;
 *   (the caller exchanges the owned positions so every rank has all n,
 *    e.g. one all-gather of 3 (i1 - i0) doubles per rank)
 *   nb_step_range_kick    a+_i from all n positions at t + dt and the kick
 *                         of the owned ions, exactly as nb_step's epilogue
 *                         (friction, trap, Langevin draws keyed by the
 *                         global ion index); advances sys->step by one.
 * The pair sums come from the one-sided kernel with the chunks of the full
 * one-sided plan, so the ranks' results, put together, are bitwise those
 * of a single call with the symmetric kernel disabled (nb_set_tuning kind
 * 4, R = 0).  Only the owned entries of x (drift) and of v and a (kick) are
 * written.  0 <= i0 <= i1 <= n, else NB_EINVAL; i0 == i1 does nothing (the
 * kick still advances the step counter).  nb_forces_range writes the
 * acceleration of the owned ions only, as nb_forces (flags) would.       */
nb_status nb_forces_range(const nb_params *params, const nb_system *sys, int64_t i0, int64_t i1,
                          int flags, void *stream);
nb_status nb_step_range_drift(const nb_params *params, nb_system *sys, int64_t i0, int64_t i1,
                              void *stream);
nb_status nb_step_range_kick(const nb_params *params, nb_system *sys, int64_t i0, int64_t i1,
                             void *stream);

/* Energies at the current state, written to HOST memory out[4] =
 * {kinetic, trap, Coulomb, total} in joules:
 *   kinetic = (m/2) sum |v|^2,
 *   trap    = the potential of the trap term of Eq. 1 at t (harmonic:
 *             (m/2) sum omega_k^2 x_k^2; RF: (m/2) sum (c (x^2 - y^2) +
 *             omega_z^2 z^2), c = (q Omega^2/2) cos(Omega t + phase)),
 *   Coulomb = (k_C/2) sum_i q_i sum_{j != i} q_j / sqrt(r_ij^2 + soft2).
 * FP64 differences and sums regardless of params->precision; the pair term
 * 1/sqrt(r^2 + soft2) is formed as in NB_FP64 (FP32-pipe double-float,
 * widened to FP64).  Synchronises the stream before returning.            */
nb_status nb_energy(const nb_params *params, const nb_system *sys,
                    double out[4], void *stream);

/* Vector-Jacobian product of the position dependence of the acceleration:
 *   g_i = k_C q_i/m sum_{j != i} q_j [ dl/s^3 - 3 d (d . dl) / s^5 ],
 *   d = r_i - r_j, dl = lam_i - lam_j, s^2 = |d|^2 + soft2,
 * plus, with NB_ACC_TOTAL, the trap's diagonal term at the current time.
 * The Jacobian is symmetric, so this is also the Jacobian-vector product.
 * lam* and g* are device SoA arrays of n doubles.  FP64 differences d and
 * dl.  Each pair's term (with its r^-3, r^-5 and d . dl) is formed in
 * double-float on the FP32 pipe, in units of the pair's own exponents
 * (relative error about 2^-44 of the term), and an ion's terms are summed in
 * double-float with one exponent per sum, the largest unit met so far, and
 * widened into an FP64 sum every 32 partners.  Weights q_j keep 48 bits;
 * a subnormal weight counts as 0.  One arithmetic for every
 * params->precision (NB_FP64 and NB_DF64 give the same bits).             */
nb_status nb_forces_vjp(const nb_params *params, const nb_system *sys,
                        const double *lx, const double *ly, const double *lz,
                        double *gx, double *gy, double *gz, int flags,
                        void *stream);

/* Ensemble of independent systems (a7: e.g. Kibble-Zurek quench
 * realisations, Sec. I): n_inst instances packed back to back in the SoA
 * arrays of `packed`; instance k owns ions [offsets[k], offsets[k+1])
 * (`offsets` in HOST memory, n_inst + 1 entries, offsets[0] = 0,
 * offsets[n_inst] = packed->n).  Every instance takes nsteps velocity-Verlet
 * steps exactly as nb_step defines them, with the shared params; instance k
 * draws its Langevin noise with instance word params->instance + k and ion
 * index local to the instance, so it reproduces a standalone nb_step run of
 * that instance.  One persistent kernel launch for all steps (NB_FP64 or
 * NB_DF64 pair arithmetic, otherwise NB_ENOTSUP); each instance lives in one thread block's shared
 * memory, so n_inst <= 1024 and every instance <= 6144 ions (NB_EINVAL
 * otherwise).  Instances are packed onto the SMs by the longest-processing-
 * time rule on n^2 (nb_plan_batched).  The launch copies nothing from the
 * host, so it can be captured in a CUDA graph after one uncaptured call has
 * set up the stream's error word; a replay repeats the captured step window
 * (the step counter, hence time and noise counter, is part of the launch).
 * Advances packed->step by nsteps.                                         */
nb_status nb_step_batched(const nb_params *params, int32_t n_inst, const int64_t *offsets,
                          nb_system *packed, int64_t nsteps, void *stream);

/* The ensemble with parameters of its own for every instance (a7; e.g. a
 * sweep of quench rates, trap ramps or cooling, one realisation per entry):
 * as nb_step_batched, except that instance k runs with per_inst[k] (HOST
 * array of n_inst nb_params) and draws its noise with instance word
 * per_inst[k].instance itself, so it reproduces a standalone nb_step run of
 * that instance with per_inst[k].  Every entry must pass nb_step's checks
 * and all entries must have the same precision (NB_FP64 or NB_DF64;
 * NB_EINVAL otherwise).  The step counter (packed->step) is shared: instance
 * k's time is per_inst[k].t0 + step * per_inst[k].dt.
 * The library keeps a device copy of the table per (device, stream) and
 * copies it again only when the contents differ from the stream's previous
 * call.  That copy is ordered on the stream after its earlier work (which
 * may still read the old table), and the call returns once the host array
 * has been read, so the caller may reuse it at once.  A graph capture records the launch, which reads the
 * stream's table when replayed: capture only after an uncaptured call with
 * the same per_inst (a capture with other contents fails with NB_EINVAL,
 * and a later uncaptured call with other contents changes what earlier
 * captures replay).  Freed by nb_release.                                  */
nb_status nb_step_batched_each(const nb_params *per_inst, int32_t n_inst, const int64_t *offsets,
                               nb_system *packed, int64_t nsteps, void *stream);

/* Host-only: the instance-to-block schedule nb_step_batched uses for n_bins
 * blocks.  order[n_inst] lists the instances grouped by block; block b runs
 * order[bin_start[b] .. bin_start[b+1]-1].  max_load / mean_load (nullable)
 * receive the largest and the mean per-block cost (sum of n^2).  No GPU.   */
nb_status nb_plan_batched(int32_t n_inst, const int64_t *offsets, int32_t n_bins,
                          uint16_t *order, uint16_t *bin_start, double *max_load,
                          double *mean_load);

/* Host-only: the launch plan a call at n ions would use, for kind 0 (the
 * force kernel of nb_forces / nb_step in `precision`), 1 (the potential
 * kernel) or 2 (the VJP kernel, fp64 and df64 alike; for kinds 1 and 2
 * `precision` is validated but does not change the plan), with the current tuning overrides:
 * out[0] threads per block (one-sided) or 256 / 128 (symmetric), out[1] ions
 * per thread R, out[2] partners per j-chunk, out[3] i-tiles (one-sided) or
 * blocks nbk (symmetric), out[4] partial slots n_jc (j-chunks; 1 for the
 * symmetric kernel, which adds into one slot in a fixed round order), out[5]
 * 1 for the symmetric kernel, out[6] its ions per block / 32, out[7] 1 if
 * nb_step would run the single-block path (kind 0).  Without a usable GPU
 * it plans for 152 SMs.  No device work.                                  */
nb_status nb_plan_info(int32_t kind, int32_t precision, int64_t n, int64_t out[8]);

/* Host-only: the work schedule of the half-pair kernels for nbk blocks
 * (1 <= nbk <= 60000): item t (0 <= t < nbk (nbk + 1) / 2) is the block pair
 * (P[t], Q[t]), P <= Q, in round round[t].  Each round touches every block
 * exactly once (a round-robin tournament; a block's own pairs, P == Q, take
 * its one free round), items are numbered round by round, and every item
 * adds its sums into the output after the previous round's items of the same
 * blocks, which fixes the order of each ion's sum (the paper's Sec. VI.C
 * static ownership, made deterministic for a GPU).  Arrays in HOST memory.
 * No GPU.                                                                 */
nb_status nb_sym_schedule(int32_t nbk, int32_t *P, int32_t *Q, int32_t *round);

/* Launch-shape override (used by the autotuner, paper_2106_11143_gb300/
 * tune.py).  For kind 0 (force), 1 (potential), 2 (VJP) pair kernels in
 * `precision` and n in [n_lo, n_hi]: `block` threads per block (32, 64, 128
 * or 256), `R` ions per thread (1, 2, 4; force kernel only) and about
 * `blocks_per_sm` (i-tile, j-chunk) blocks per SM.  The potential and VJP
 * plans are shared by every precision and read only the NB_FP64 entries
 * (kinds 1, 2 and 5): an override there also shapes the NB_DF64 VJP.  For kind 3 (the ensemble
 * kernel): `block` threads per block (multiple of 32, <= 512), and R = 0 to
 * keep its one-sided force phase (by default ensembles whose instances all
 * have at most 4096 ions use the half-pair phase).  For kind 4
 * (the symmetric half-pair force kernel of the four force precisions): `block` ions
 * per block pair unit (32, 64, 128, 256, 512, 1024) and R = 1 to use it or 0
 * to disable it for that n range (by default it is used from n = 500 in
 * NB_MIXED_SPLIT, 1000 in NB_MIXED, 1500 in NB_FP64 and 2000 in NB_DF64).
 * For kind 5
 * (the symmetric VJP kernel of NB_FP64 and NB_DF64; pass NB_FP64): `block` ions per block
 * pair unit (128 or 256) and R = 1 / 0 to use / disable it (by default it is
 * used from n = 2500).  For kind 6 (step windows of nb_step): R = 1 to
 * use them or 0 not to, for calls of at least `block` steps (by default
 * they are used for n <= 4096 and nsteps >= 32).  For kind 7 (single-block
 * steps of small systems in nb_step): R = 1 to use them or 0 not to, for n
 * in [n_lo, n_hi] (`block` >= 1, not used; the kernel's own limits still
 * apply).  For kind 8 (the epilogues of nb_forces, nb_step and
 * nb_forces_vjp, every precision; pass NB_FP64): R = 1 for eight threads per
 * ion (the default), 0 for one.  The latest
 * matching entry wins; block == 0 removes every override.  Results stay
 * deterministic for a fixed shape; different shapes may differ in the last
 * bits (summation order), except kind 3, which is shape-independent.     */
nb_status nb_set_tuning(int32_t kind, int32_t precision, int64_t n_lo, int64_t n_hi,
                        int32_t block, int32_t R, int32_t blocks_per_sm);

/* ---- Trajectory loss and its gradient (a9) ------------------------------
 * Loss of a velocity-Verlet trajectory (Sec. II) of nsteps steps from
 * (x_0, v_0), a_0 = A(x_0):
 *   L = E_coulomb(x_T) + E_trap(x_T) + sum_i |x_T,i - target_i|^2
 * (energies as in nb_energy; the squared distance in m^2, added as plain
 * numbers), and its exact gradient with respect to x_0, v_0 and the three
 * trap frequencies by the discrete adjoint (reverse sweep) of the Verlet
 * map.  Supported: static harmonic trap, gamma = 0, noise_T = 0, and the
 * NB_FP64 or NB_DF64 arithmetic for the forward and its recompute (as
 * nb_forces in that precision; NB_ENOTSUP otherwise); the Jacobian products
 * are those of nb_forces_vjp.  The forward stores the state (x, v, a)
 * at steps 0, every, 2*every, ... in `ckpt`; the backward recomputes each
 * segment from its checkpoint (bitwise identical to the forward) and sweeps
 * it in reverse, so the result does not depend on `every`. */

/* Doubles needed for the checkpoint buffer: ceil(nsteps/every) * 9 * n
 * (9 * n when nsteps == 0); -1 on invalid arguments. */
int64_t nb_traj_ckpt_doubles(int64_t n, int64_t nsteps, int64_t every);

/* Forward: sys holds x_0, v_0 on entry (its a is overwritten with A(x_0));
 * on return it holds x_T, v_T, a_T and step += nsteps.  ckpt (device,
 * nb_traj_ckpt_doubles) receives the checkpoints; target: device, 3n doubles
 * (x block, y block, z block); loss: device, one double.  Asynchronous.    */
nb_status nb_traj_forward(const nb_params *params, nb_system *sys, int64_t nsteps,
                          int64_t every, double *ckpt, const double *target, double *loss,
                          void *stream);

/* Backward: from the checkpoints of nb_traj_forward (same params, nsteps,
 * every; sys supplies n and q only), writes gscale * dL/dx_0 and
 * gscale * dL/dv_0 (device, 3n doubles each, SoA blocks) and
 * gscale * dL/domega (device, 3 doubles).  gscale: device pointer to one
 * double (the incoming gradient of a caller's chain rule) or NULL for 1.
 * Asynchronous; uses library scratch of about (every + 20) * 3n doubles.   */
nb_status nb_traj_backward(const nb_params *params, const nb_system *sys, int64_t nsteps,
                           int64_t every, const double *ckpt, const double *target,
                           const double *gscale, double *gx0, double *gv0, double *gomega,
                           void *stream);

/* nb_energy without any device allocation.  The paper has no counterpart:
 * this serves callers that cannot call cudaMalloc -- cudaMalloc may
 * synchronise the device, which a latency-bound loop cannot afford, and under
 * a host framework that owns device memory through its own pool it can fail
 * or take memory budgeted elsewhere.  Same inputs, outputs, argument checks
 * and arithmetic as nb_energy (out[4] in HOST memory; synchronises the
 * stream).  Its scratch is one fixed 8 MiB device array inside the library,
 * held on every GPU that loads the library until the process exits; n above
 * what it can hold is rejected with NB_EINVAL and a message in
 * nb_last_error().  With the default plan on a 152-SM GB300 the limit is
 * about n = 1,000,000; a potential-kernel tuning override (nb_set_tuning
 * kind 1) or a GPU with more SMs can lower it.
 * All calls share that array: calls that may overlap on the GPU (other
 * streams, unordered host threads) race and must be serialised.  The first
 * call on each device looks up the array's device address with that device
 * current; make that first call before any stream capture.                 */
nb_status nb_energy_noalloc(const nb_params *params, const nb_system *sys,
                            double out[4], void *stream);

/* ---- Arithmetic probes (steps a1-a3 of one pair, Sec. III-IV) ---------- */

/* out[i] = the r^-3 that precision mode `precision` (an nb_precision value)
 * forms for one pair with FP64 displacement (dx[i], dy[i], dz[i]) and
 * softening soft2 >= 0: r^2 = dx^2 + dy^2 + dz^2 + soft2, then the mode's
 * 1/sqrt and cube -- the same device functions as the pair kernels, before the
 * charge weight.  NB_MIXED and NB_MIXED_SPLIT share their FP32 bulk; here
 * both start from the displacement rounded to FP32 (the split mode's own
 * displacement comes from FP32 position pairs instead).  NB_DF64 returns
 * its double-float result summed into one double.  r^2 == 0 gives 0 in the
 * FP64 modes and a finite value (times the zero displacement in a pair) in
 * the FP32 ones.  All arrays are device memory of n doubles, caller-owned;
 * asynchronous on `stream`.  NB_EINVAL for n < 0, a NULL array with n > 0,
 * soft2 < 0 or NaN, or an unknown precision.                                */
nb_status nb_rinv3_probe(int precision, int64_t n, const double *dx, const double *dy,
                         const double *dz, double soft2, double *out, void *stream);

/* y[i] = the FP32 hardware reciprocal-square-root seed of x[i]
 * (rsqrt.approx.ftz.f32, Sec. IV's counterpart of RSQRT14), for the seed's
 * error bound.  Device arrays of n floats, caller-owned; asynchronous.      */
nb_status nb_rsqrt_seed_probe(int64_t n, const float *x, float *y, void *stream);

/* Throughput of one instruction kind on every SM of the current device: the
 * measured denominators of the ALU rooflines (Sec. VI reports the method's
 * speed as a fraction of the FMA peak; this is that peak on the GPU).
 * kind: 0 FP64 FMA, 1 FP64 add, 2 FP64 multiply, 3 FP32 FMA, 4 FP32 add,
 * 5 FP32 reciprocal square root (MUFU).  Two blocks of 512 threads per SM
 * run independent dependence chains of the instruction in three shapes (4
 * chains with their own operands, 4 and 8 chains sharing operands; the work
 * of 4 * 8 * iters instructions per thread in each; 2 <= iters <= 2^24) and
 * the fastest counts: register-bank conflicts make the attainable rate
 * depend on the shape.  out (HOST, 3 doubles): out[0] lanes retired per
 * clock per SM (median over SMs, from the SM cycle counter), out[1] the SM
 * clock in MHz over that launch (cycles / event time), out[2] the shape
 * (0, 1, 2 as listed).  Allocates a few KB of device memory for the clock
 * records and synchronises the stream.                                    */
nb_status nb_pipe_probe(int32_t kind, int64_t iters, double out[3], void *stream);

/* Synchronises `stream`, then returns and clears its device error word:
 * NB_OK, NB_ENONFINITE or NB_ETIMEOUT (or NB_ECUDA if the stream failed). */
nb_status nb_sync_status(void *stream);

/* Probe of the bounded wait behind the half-pair kernels' round-ordered
 * output (one item waits until the items of the previous round that touched
 * its blocks have committed): one device thread publishes `committed` rounds
 * for a block, with a release store, then waits with acquire loads until the
 * block has committed `round`, as an item does.  *ok (host) receives 1 if
 * the wait succeeded.  A wait for a round nobody commits (round > committed)
 * spins until its limit (one to a few seconds), sets the stream's device
 * error word, so that nb_sync_status returns NB_ETIMEOUT, and ends normally:
 * the failure path of every bounded wait, without a GPU fault.  Uses the
 * stream's scratch; synchronises the stream.  NB_EINVAL for a NULL ok or a
 * negative argument.                                                        */
nb_status nb_sym_wait_probe(int32_t committed, int32_t round, int32_t *ok, void *stream);

/* Frees all library scratch on every device (after synchronising them). */
nb_status nb_release(void);

/* Static description of a status code. */
const char *nb_strerror(nb_status status);

/* Detail of the most recent failure on the calling thread ("" if none). */
const char *nb_last_error(void);

/* Library version string. */
const char *nb_version(void);

/* ---- Instrumentation (benchmarks and tests) ---------------------------- */

/* Number of CUDA kernels this library has launched in this process. */
uint64_t nb_launch_count(void);

/* Kernel timing: with capacity > 0, every O(N^2) pair-kernel launch of the
 * calling process is bracketed by two CUDA events recorded on the stream it
 * is launched on, for up to `capacity` launches (events are created here, on
 * the current device).  capacity == 0 disables timing and frees the events. */
nb_status nb_timing_enable(int64_t capacity);

/* Waits for the recorded events, returns the number of timed pair-kernel
 * launches and their summed device duration in milliseconds, and restarts
 * the count.  Launches beyond the capacity are not timed.                  */
nb_status nb_timing_read(int64_t *launches, double *total_ms);

#ifdef __cplusplus
}
#endif

#endif /* NB_H */
