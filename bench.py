"""Benchmark: G pair-interactions/s of velocity-Verlet steps at N = 1e5.

Workload: the large-cloud configuration -- 1e5 singly charged ions of 40 u,
uniform in a 200 x 200 x 1000 um ellipsoid held by the harmonic
pseudopotential for which that spheroid is a cold-fluid equilibrium, 10 mK
velocities, dt = 1 ns (seeded, synthetic).  A step is one full
velocity-Verlet step through the C ABI (nb_step: drift, the O(N^2) pair
kernel, the kick/trap/friction epilogue).  value = N^2 pair interactions per
step x steps x ranks / the max over ranks of the device time of the K timed
steps (CUDA events on the launching stream; L2 flushed by a 256 MB write
between timed steps, outside the timed events).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P]
  python bench.py --impl reference   # the FP64 CPU oracle on the host cores

--gpus N > 1 runs one independent replica per rank (the path is one
all-pairs problem per GPU here; no collective on the data path).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "G pair-interactions/s & % FMA peak, FP64 vs mixed (rel err ≤1e-6) at N=1e5"
UNIT = "G pair-interactions/s"
# Flop convention A: 20 flops per pair evaluation (3 sub, 3 mul + 2 add for
# r^2, 1 softening add, sqrt, divide, 2 mul for the cube, 3 mul + 3 add).
FLOPS_PER_PAIR = 20
# Convention B for the fp64 path: the FP64 flops the half-pair kernel executes
# per evaluation, 2 x 6 DFMA (the force into both ions) + 4 DADD (the
# displacement and the widening of r^-3); everything else runs on the FP32 pipe.
FP64_FLOPS_PER_EVAL_SYM = 2 * 6 + 4
SM_COUNT = 152
# The pipe whose rate bounds each path's pair kernel, and the probe kind that
# measures it (nb_pipe_probe; 2 flops per FMA lane).
PATH_PIPE = {"fp64": "dfma", "df64": "ffma", "mixed": "ffma", "mixed_split": "ffma", "mixed_split_rsq": "ffma"}
DTYPE = {"fp64": "f64", "df64": "f32x2+f64", "mixed": "f32+f64", "mixed_split": "f32+f64", "mixed_split_rsq": "f32+f64"}
ACCURACY_GATE = {"fp64": 1e-12, "df64": 1e-12, "mixed": 1e-6, "mixed_split": 1e-6, "mixed_split_rsq": 1e-6}
PATHS = ("fp64", "df64", "mixed", "mixed_split", "mixed_split_rsq")
PROFILES = os.path.join(ROOT, "profiles")
# Kernel sources a recorded DRAM-traffic figure is valid for.
KERNEL_SOURCES = ("nb_sym.cu", "nb_symsched.cuh", "nb_pair.cu", "nb_common.cuh", "nb_pairterm.cuh")
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed_split",
                    choices=["fp64", "df64", "mixed", "mixed_split", "mixed_split_rsq"])
    ap.add_argument("--ions", "--n", dest="n", type=int, default=100000,
                    help="ions (default: the 1e5 workload); spelled --ions under torchrun, whose "
                         "parser takes --n for an abbreviation of its own options")
    ap.add_argument("--no-paths", action="store_true", help="skip the secondary precisions")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--precisions", default="fp64,df64,mixed,mixed_split",
                    help="--profile-forces: the precisions, in launch order")
    ap.add_argument("--kz-instances", type=int, default=512,
                    help="instances of the kz / kz_sweep ensemble (512 as configured; fewer for a profile)")
    ap.add_argument("--workload", default="large", choices=["large", "kz", "kz_sweep"],
                    help="large: the N=1e5 headline; kz: the 512-instance ensemble (extra line); "
                         "kz_sweep: the same ensemble with a quench rate per instance")
    ap.add_argument("--profile-forces", action="store_true",
                    help="profiling case: two nb_forces calls per precision at --n, no timing")
    ap.add_argument("--one-sided", action="store_true",
                    help="with --profile-forces: the one-sided force kernel at any n")
    ap.add_argument("--profile-vjp", action="store_true",
                    help="profiling case: two nb_forces_vjp calls at --n, no timing")
    ap.add_argument("--profile-small", action="store_true",
                    help="profiling case: small-n steps (single-block at n = 16, windows at n = 1000)")
    ap.add_argument("--peaks", action="store_true",
                    help="only the measured pipe rates of this GPU (nb_pipe_probe), one JSON line")
    ap.add_argument("--step-sweep", default=None, metavar="SIZES",
                    help="step rate per N (comma-separated sizes, e.g. 10,100,1000,10000,100000) by "
                         "launch path, one JSON line per N and precision")
    ap.add_argument("--cpu-sweep", action="store_true",
                    help="the oracle's force evaluation per N on one core and on all host cores, "
                         "beside the GPU force evaluation (one JSON line per N)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", "nb_clocks_%d_%d.csv" % (os.getpid(), index))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sms) if sms else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sms)}


# ---------------------------------------------------------------------------
def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if args.impl == "ours":
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    elif args.impl == "ours":
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, world, device="cuda"):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def pair_rate(world, pairs_per_step, steps, ms):
    """Whole-job G pair-interactions/s: every rank advances its own problem of
    pairs_per_step pairs by `steps` steps; ms is the max over ranks."""
    return world * pairs_per_step * steps / (ms / 1e3) / 1e9


def cpu_baseline(w, target_s=12.0, gpu_acc=None):
    """The FP64 oracle (as it stands) on the host cores: one force evaluation
    restricted to a bounded sample of target ions [0, S) against all N.  The
    same sample's oracle forces are the reference for each path's accuracy:
    gpu_acc maps a precision to the Coulomb accelerations (3, N) that nb_forces
    gave for the same positions; per path the largest conditioned error (the
    gate's measure, |da_i| / sum_j |a_ij|), the largest, 99th-percentile and
    median plain relative error |da_i| / |a_i| and the global ||da|| / ||a||
    over the sample."""
    import oracle
    p = oracle.make_params(**w["phys"])
    n = w["n"]
    s0 = 256
    t = time.perf_counter()
    oracle.coulomb(p, *w["pos"], i0=0, i1=s0)
    dt0 = time.perf_counter() - t
    s = int(min(n, max(s0, s0 * target_s / max(dt0, 1e-6))))
    t = time.perf_counter()
    ax, ay, az, _, absf = oracle.coulomb(p, *w["pos"], i0=0, i1=s, want_absf=True)
    dt = time.perf_counter() - t
    out = {"value": s * n / dt / 1e9, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
           "sample": "one FP64 force evaluation of ions [0, %d) against all %d ions (%.3g pairs, %.1f s)"
                     % (s, n, s * n, dt)}
    if gpu_acc:
        ref = np.stack([ax, ay, az])
        mag = np.sqrt(np.sum(ref ** 2, axis=0))
        acc = {}
        for prec, g in gpu_acc.items():
            d = np.sqrt(np.sum((g[:, :s] - ref) ** 2, axis=0))
            rel = d / mag
            acc[prec] = {"max_conditioned": float("%.3g" % np.max(d / absf)), "gate": ACCURACY_GATE[prec],
                         "max_rel": float("%.3g" % np.max(rel)),
                         "p99_rel": float("%.3g" % np.percentile(rel, 99)),
                         "median_rel": float("%.3g" % np.median(rel)),
                         "global_rel": float("%.3g" % (np.sqrt(np.sum(d * d)) / np.sqrt(np.sum(mag * mag)))),
                         "ions_rel_above_gate": int(np.sum(rel > ACCURACY_GATE[prec]))}
        out["accuracy_vs_oracle"] = {"ions": s, "paths": acc}
    return out


# ---------------------------------------------------------------------------
def run_path(nb, w, precision, steps, warmup, world, flush, clocks=None):
    """Time `steps` single-step nb_step calls; returns device ms per step, the
    mean pair-kernel duration, and the launch count of the timed region."""
    import torch
    lib = nb.lib()
    par = nb.Params.from_phys(w["phys"], precision=precision)
    sysm = nb.System(w["pos"], w["vel"])
    nb.forces(par, sysm, total=True)
    for _ in range(warmup):
        nb.step(par, sysm, 1)
    nb.sync_status()
    st = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    _check(lib.nb_timing_enable(steps), lib)
    launches0 = lib.nb_launch_count()
    barrier(world)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    t_wall = time.perf_counter()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(st)
        nb.step(par, sysm, 1)
        ev[k][1].record(st)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    barrier(world)
    clk = clocks.stop() if clocks else None
    launches = lib.nb_launch_count() - launches0
    nl, tot = _timing_read(lib)
    _check(lib.nb_timing_enable(0), lib)
    nb.sync_status()
    dev_ms = sum(a.elapsed_time(b) for a, b in ev)
    return {"ms": dev_ms, "ms_per_step": dev_ms / steps, "kernel_ms": tot / max(nl, 1),
            "kernel_launches": nl, "launches": int(launches), "wall_s": t_wall, "clocks": clk,
            "sys": sysm, "par": par}


def _check(rc, lib):
    if rc != 0:
        raise RuntimeError("libnb: " + lib.nb_last_error().decode())


def _timing_read(lib):
    import ctypes as C
    n = C.c_int64()
    ms = C.c_double()
    _check(lib.nb_timing_read(C.byref(n), C.byref(ms)), lib)
    return n.value, ms.value


def run_e2e(nb, w, precision, steps, world, flush):
    """Same metric through the public API with host buffers: every step copies
    the Verlet state (x, v, a: System.state, one packed device tensor) from
    pinned host memory to the device in one copy, runs nb_step, and reads the
    state back into pinned host memory in one copy."""
    import torch
    n = w["n"]
    par = nb.Params.from_phys(w["phys"], precision=precision)
    sysm = nb.System(w["pos"], w["vel"])
    nb.forces(par, sysm, total=True)
    host = sysm.state.cpu().pin_memory()
    st = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier(world)
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(st)
        sysm.state.copy_(host, non_blocking=True)
        nb.step(par, sysm, 1)
        host.copy_(sysm.state, non_blocking=True)
        ev[k][1].record(st)
    torch.cuda.synchronize()
    barrier(world)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ms = allreduce_max(ms, world)
    nbytes = host.numel() * host.element_size()
    return {"value": pair_rate(world, n * n, steps, ms), "unit": UNIT,
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "copies_per_step": {"h2d": 1, "d2h": 1}}


def measure_peaks(nb, kinds=("dfma", "dadd", "ffma", "fadd", "mufu_rsq")):
    """Measured pipe rates of this GPU (nb_pipe_probe): lanes retired per clock
    per SM for each instruction kind, after one warm-up launch."""
    out = {}
    for k in kinds:
        nb.pipe_probe(k, iters=16)
        r = nb.pipe_probe(k)
        out[k] = {"lanes_per_clk_per_sm": round(r["lanes_per_clk_per_sm"], 3), "sm_mhz": round(r["sm_mhz"], 1),
                  "shape": r["shape"]}
    return out


def evaluations(nb, precision, n):
    """Pair evaluations one force launch performs, and the kernel's name.
    One-sided kernel: every ordered pair, N^2 (the self pair contributes 0).
    Half-pair kernel (blocks of BI = 32 G ions): every pair of ions in
    different blocks once, serving both, plus each block's own pairs
    one-sided: (N^2 + sum_b n_b^2) / 2."""
    p = nb.plan_info("force", precision, n)
    if not p["symmetric"]:
        return n * n, "k_pair_force<%s>" % precision
    bi = 32 * p["G"]
    full, rem = divmod(n, bi)
    return (n * n + full * bi * bi + rem * rem) // 2, "k_pair_sym<%s>" % precision


def kernel_source_sha():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2106_11143_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def recorded_counters(precision, n):
    """ncu counters of the pair kernel per launch, from the summaries under
    profiles/: a line `traffic: precision=P n=N bytes=B [inst=I] source=S`
    records one capture of this bench's command: B the DRAM bytes (read +
    write), I the warp instructions executed (smsp__inst_executed.sum), S
    the kernel sources' hash when it was taken.  ({}, None) when there is no
    capture for this case or the kernel has changed since."""
    import glob
    want = kernel_source_sha()
    out, src = {}, None
    for path in sorted(glob.glob(os.path.join(PROFILES, "*.md"))):
        for line in open(path):
            line = line.strip()
            if not line.startswith("traffic: "):
                continue
            kv = dict(t.split("=", 1) for t in line.split()[1:])
            if kv.get("precision") == precision and int(kv.get("n", -1)) == n and kv.get("source") == want:
                for k in ("bytes", "inst", "fp64_inst"):  # the first summary naming a counter wins
                    if k in kv and k not in out:
                        out[k] = int(kv[k])
                        src = src or os.path.basename(path)
    return out, src


OPMIX_KINDS = ("dadd", "dfma", "dmul", "fadd", "ffma", "fmul", "fadd2", "ffma2", "fmul2")


def recorded_opmix(precision):
    """Lane-instructions per pair evaluation of the pair kernel in this
    precision, by kind (FP64 "dadd", "dfma", "dmul"; FP32 "fadd", "ffma",
    "fmul" and the packed "fadd2", "ffma2", "fmul2"), from an `opmix:` line
    of the summaries under profiles/ (SASS op counters of one ncu capture,
    which take three passes, so they come from a case smaller than the
    bench's with the same kernel configuration); {} when unrecorded or the
    kernel sources have changed since."""
    import glob
    want = kernel_source_sha()
    for path in sorted(glob.glob(os.path.join(PROFILES, "*.md"))):
        for line in open(path):
            line = line.strip()
            if not line.startswith("opmix: "):
                continue
            kv = dict(t.split("=", 1) for t in line.split()[1:])
            if kv.get("precision") == precision and kv.get("source") == want:
                return {k: float(kv[k]) for k in OPMIX_KINDS if k in kv}
    return {}


def recorded_traffic(precision, n):
    """DRAM bytes (read + write) per launch of the pair kernel and the
    summary they come from (recorded_counters); (None, None) if unrecorded."""
    c, src = recorded_counters(precision, n)
    return c.get("bytes"), src


def roofline(nb, path, n, kernel_ms, peaks, sm_mhz):
    """Roofline of the pair kernel: convention-A flops (20 per evaluation) on
    the evaluations the kernel performs, over its measured duration, against
    the measured rate of the pipe that bounds it at the SM clock sampled
    during the timed steps."""
    evals, kname = evaluations(nb, path, n)
    pipe = PATH_PIPE[path]
    lanes = peaks[pipe]["lanes_per_clk_per_sm"]
    mhz = sm_mhz or peaks[pipe]["sm_mhz"]
    peak = 2 * lanes * SM_COUNT * mhz * 1e6 / 1e12
    achieved = FLOPS_PER_PAIR * evals / (kernel_ms / 1e3) / 1e12
    counters, src = recorded_counters(path, n)
    traffic = counters.get("bytes")
    r = {"bound": "alu", "pipe": "FP64 FMA" if pipe == "dfma" else "FP32 FMA",
         "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
         "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": kname,
         "evaluations_per_launch": evals, "flops_per_evaluation": FLOPS_PER_PAIR,
         "peak_source": "measured: nb_pipe_probe %s %.3f lanes/clk/SM x 2 flops x %d SMs x %.0f MHz "
                        "(%s)" % (pipe.upper(), lanes, SM_COUNT, mhz,
                                  "median SM clock during the timed steps" if sm_mhz else "probe clock"),
         "convention": "A: 20 flops per pair evaluation performed",
         "n2_equivalent": {"tflops": round(FLOPS_PER_PAIR * n * n / (kernel_ms / 1e3) / 1e12, 3),
                           "note": "20 flops x N^2 interactions; a half-pair evaluation serves two "
                                   "interactions, so this is not a pipe fraction"}}
    if traffic is not None:
        r["traffic_source"] = "profiles/" + src
    if "inst" in counters:
        # instruction issue: 4 warp instructions per clock per SM (one per
        # scheduler), the unit that binds a kernel whose evaluation needs more
        # issue slots than its convention-A flops suggest
        ipeak = 4 * SM_COUNT * mhz * 1e6 / 1e9
        iach = counters["inst"] / (kernel_ms / 1e3) / 1e9
        r["issue"] = {"achieved": round(iach, 2), "peak": round(ipeak, 2), "unit": "G warp-instructions/s",
                      "frac": round(iach / ipeak, 4),
                      "warp_instructions_per_32_evaluations": round(counters["inst"] / (evals / 32.0), 2),
                      "source": "smsp__inst_executed.sum per launch from profiles/ over the live kernel time; "
                                "peak 4 per clock per SM x %d SMs x %.0f MHz" % (SM_COUNT, mhz)}
    if "fp64_inst" in counters and "dfma" in peaks:
        # the FP64 pipe, for the paths whose FP64 adds bind them (2 lanes per
        # clock per SM: a warp instruction occupies it for 16 clocks)
        lanes64 = peaks["dfma"]["lanes_per_clk_per_sm"]
        fpeak = lanes64 * SM_COUNT * mhz * 1e6 / 1e12
        fach = counters["fp64_inst"] * 32 / (kernel_ms / 1e3) / 1e12
        r["fp64_pipe"] = {"achieved": round(fach, 4), "peak": round(fpeak, 4), "unit": "T lane-instructions/s",
                          "frac": round(fach / fpeak, 4),
                          "fp64_instructions_per_evaluation": round(counters["fp64_inst"] * 32 / evals, 3),
                          "source": "smsp__inst_executed_pipe_fp64.sum per launch from profiles/ over the live "
                                    "kernel time; peak the measured FP64 FMA rate %.3f lanes/clk/SM x %d SMs x "
                                    "%.0f MHz" % (lanes64, SM_COUNT, mhz)}
        # the pipe's attainable rate for this kernel's own mix of FP64 adds,
        # FMAs and multiplies, each at its measured rate (an add retires at
        # about 0.84 of an FMA's rate on this GPU)
        mix = recorded_opmix(path)
        kinds = [k for k in ("dadd", "dfma", "dmul") if mix.get(k, 0.0) > 0.0]
        if kinds and all(k in peaks for k in kinds):
            tot = sum(mix[k] for k in kinds)
            lanes_mix = tot / sum(mix[k] / peaks[k]["lanes_per_clk_per_sm"] for k in kinds)
            mpeak = lanes_mix * SM_COUNT * mhz * 1e6 / 1e12
            r["fp64_pipe"]["mix"] = {k: mix[k] for k in kinds}
            r["fp64_pipe"]["mix_ceiling"] = round(mpeak, 4)
            r["fp64_pipe"]["frac_of_mix_ceiling"] = round(fach / mpeak, 4)
            r["fp64_pipe"]["mix_note"] = ("ceiling = the kernel's FP64 lane-instructions per evaluation by kind "
                                          "(opmix, profiles/) at the measured rate of each kind: %.3f lanes/clk/SM"
                                          % lanes_mix)
    mix = recorded_opmix(path)
    if pipe == "ffma" and all(k in mix for k in ("fadd", "ffma", "fmul", "fadd2", "ffma2", "fmul2")):
        # the FMA pipe by the work it does: each FP32 add, multiply or FMA
        # one lane-cycle, each packed .f32x2 one two lane-cycles (it holds
        # the pipe for two cycles), against the measured FFMA rate
        lane_ops = mix["fadd"] + mix["ffma"] + mix["fmul"] + 2 * (mix["fadd2"] + mix["ffma2"] + mix["fmul2"])
        cpeak = lanes * SM_COUNT * mhz * 1e6 / 1e12
        cach = lane_ops * evals / (kernel_ms / 1e3) / 1e12
        r["fma_pipe"] = {"achieved": round(cach, 3), "peak": round(cpeak, 3), "unit": "T lane-cycles/s",
                         "frac": round(cach / cpeak, 4),
                         "lane_cycles_per_evaluation": round(lane_ops, 3),
                         "source": "FP32 op mix per evaluation (opmix, profiles/) x evaluations over the live "
                                   "kernel time; peak the measured FFMA rate %.3f lanes/clk/SM x %d SMs x "
                                   "%.0f MHz" % (lanes, SM_COUNT, mhz)}
        # convention B on the FP32 pipe: the flops it executes (an FMA two, an
        # add or multiply one, a packed instruction twice that) over the FP32
        # FMA peak
        flops = (2 * mix["ffma"] + mix["fadd"] + mix["fmul"]
                 + 2 * (2 * mix["ffma2"] + mix["fadd2"] + mix["fmul2"]))
        bach = flops * evals / (kernel_ms / 1e3) / 1e12
        r["conv_B"] = {"achieved": round(bach, 3), "frac": round(bach / peak, 4),
                       "flops_per_evaluation": round(flops, 3),
                       "note": "executed FP32 flops from the recorded op mix (2 per FFMA, 1 per FADD/FMUL, "
                               "twice that per packed .f32x2 instruction) over the FP32 FMA peak"}
    units = [("FP64 FMA" if pipe == "dfma" else "FP32 FMA", r["frac"])]
    if "issue" in r:
        units.append(("issue", r["issue"]["frac"]))
    if "fp64_pipe" in r:
        units.append(("FP64 pipe", r["fp64_pipe"]["frac"]))
    if "fma_pipe" in r:
        units.append(("FMA pipe", r["fma_pipe"]["frac"]))
    if len(units) > 1:
        r["binding"] = max(units, key=lambda u: u[1])[0]
    if path == "fp64" and kname.startswith("k_pair_sym"):
        b = FP64_FLOPS_PER_EVAL_SYM * evals / (kernel_ms / 1e3) / 1e12
        r["conv_B"] = {"achieved": round(b, 3), "frac": round(b / peak, 4),
                       "note": "executed FP64 flops, 2 x 6 DFMA + 4 DADD per evaluation, over the FP64 FMA peak"}
    return r


def gpu_forces(nb, w, precision):
    """Coulomb accelerations (3, N) of the workload's initial positions
    through nb_forces in one precision (for the accuracy leg)."""
    par = nb.Params.from_phys(w["phys"], precision=precision)
    sysm = nb.System(w["pos"])
    nb.forces(par, sysm)
    nb.sync_status()
    return sysm.acc().cpu().numpy()


def main_ours(args):
    import torch
    world, rank, local = dist_setup(args)
    import paper_2106_11143_gb300 as nb
    from paper_2106_11143_gb300 import workloads as W
    w = W.cloud_large(n=args.n)
    n = w["n"]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    peaks = measure_peaks(nb, ("dfma", "dadd", "ffma"))
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    head = run_path(nb, w, args.precision, args.steps, args.warmup, world, flush, clocks)
    ms = allreduce_max(head["ms"], world)
    value = pair_rate(world, n * n, args.steps, ms)
    e2e = run_e2e(nb, w, args.precision, min(args.steps, 20), world, flush)
    sm_mhz = (head["clocks"] or {}).get("sm_mhz")
    paths = {}
    if not args.no_paths:
        for pth in PATHS:
            r = head if pth == args.precision else run_path(nb, w, pth, max(2, min(args.steps, 5)), 1,
                                                            world, flush)
            paths[pth] = {"value": round(n * n / (r["ms_per_step"] / 1e3) / 1e9, 3), "unit": UNIT,
                          "ms_per_step": round(r["ms_per_step"], 4),
                          "kernel_ms": round(r["kernel_ms"], 4),
                          "roofline": roofline(nb, pth, n, r["kernel_ms"], peaks, sm_mhz)}
        paths["speedup_mixed_over_fp64"] = round(paths["fp64"]["ms_per_step"] / paths["mixed"]["ms_per_step"], 3)
        paths["speedup_mixed_split_over_fp64"] = round(
            paths["fp64"]["ms_per_step"] / paths["mixed_split"]["ms_per_step"], 3)
        paths["speedup_df64_over_fp64"] = round(paths["fp64"]["ms_per_step"] / paths["df64"]["ms_per_step"], 3)
        paths["speedup_mixed_split_rsq_over_fp64"] = round(
            paths["fp64"]["ms_per_step"] / paths["mixed_split_rsq"]["ms_per_step"], 3)
        paths["note"] = ("mixed is the literal form (FP64 displacement, then cast); mixed_split forms the "
                         "displacement from FP32 (hi, lo) position pairs (reading C19); mixed_split_rsq is "
                         "mixed_split with the bare FP32 seed for r^-3 (no Newton step); accuracy of each "
                         "against the oracle is under cpu_baseline.accuracy_vs_oracle")
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu:
        precs = PATHS if not args.no_paths else (args.precision,)
        cpu = cpu_baseline(w, gpu_acc={pr: gpu_forces(nb, w, pr) for pr in precs})
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
        "config": {"workload": w["name"] + ": 1e5 ions (40 u, +e) uniform in a 200x200x1000 um ellipsoid, "
                   "cold-fluid harmonic trap, 10 mK, dt=1 ns; one velocity-Verlet step per timed step",
                   "n": n, "precision": args.precision, "pairs_per_step": n * n,
                   "l2": "flushed between timed steps (256 MB write outside the timed events)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline(nb, args.precision, n, head["kernel_ms"], peaks, sm_mhz),
        "peaks": peaks,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": head["launches"],
        "clocks": head["clocks"],
        "paths": paths,
    }
    print(json.dumps(out))


def main_peaks(args):
    """One JSON line: the measured rate of each instruction kind on this GPU
    (nb_pipe_probe) and the resulting peaks at the probe's own clock."""
    import torch
    torch.cuda.set_device(0)
    import paper_2106_11143_gb300 as nb
    pk = measure_peaks(nb)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    tf = {k: round((2 if k in ("dfma", "ffma") else 1) * v["lanes_per_clk_per_sm"] * sms * v["sm_mhz"] * 1e6 / 1e12, 4)
          for k, v in pk.items()}
    print(json.dumps({"peaks": pk, "sms": sms, "tflops_or_tops_at_probe_clock": tf,
                      "note": "lanes retired per clock per SM, median over SMs; FMA counts 2 flops"}))


def main_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2106_11143_gb300 import workloads as W
    w = W.cloud_large(n=args.n)
    n = w["n"]
    p = oracle.make_params(**w["phys"])
    # one step = one oracle force evaluation for a bounded sample of target ions
    s0 = 128
    t = time.perf_counter()
    oracle.coulomb(p, *w["pos"], i0=0, i1=s0)
    dt0 = time.perf_counter() - t
    s = int(min(n, max(s0, s0 * 4.0 / max(dt0, 1e-6))))
    for k in range(args.warmup):
        oracle.coulomb(p, *w["pos"], i0=0, i1=min(s, 2048))
    t = time.perf_counter()
    for k in range(args.steps):
        i0 = (k * s) % n
        oracle.coulomb(p, *w["pos"], i0=i0, i1=min(n, i0 + s))
    dt = time.perf_counter() - t
    value = args.steps * s * n / dt / 1e9
    sample = "per step: FP64 oracle forces of %d target ions against all %d ions (%.3g pairs)" % (s, n, s * n)
    print(json.dumps({
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": w["name"], "n": n, "precision": "fp64 oracle (Neumaier-compensated)"},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": oracle.get_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def kz_roofline(nb, prec, pairs, steps, ms, clk):
    """The ensemble kernel's rate against the measured pipe peak.  Its
    half-pair phase evaluates each pair of an instance once (about half of
    sum N_k^2 per step); the figure counts 20 flops per pair interaction, so
    it is an N^2-equivalent rate, not a pipe fraction."""
    pipe = PATH_PIPE[prec]
    pk = measure_peaks(nb, (pipe,))[pipe]
    mhz = (clk or {}).get("sm_mhz") or pk["sm_mhz"]
    peak = 2 * pk["lanes_per_clk_per_sm"] * SM_COUNT * mhz * 1e6 / 1e12
    a = FLOPS_PER_PAIR * pairs * steps / (ms / 1e3) / 1e12
    return {"bound": "alu", "pipe": "FP64 FMA" if pipe == "dfma" else "FP32 FMA", "achieved": round(a, 4),
            "peak": round(peak, 3), "unit": "TFLOP/s", "n2_equivalent_frac": round(a / peak, 4),
            "frac": None, "note": "20 flops per N^2 interaction; the half-pair phase performs about half "
                                  "as many evaluations, so no pipe fraction is claimed"}


def main_kz(args):
    """Extra line: the Kibble-Zurek ensemble (512 instances, N_k uniform in
    32..4096, FP64) advanced by K steps in ONE persistent launch of
    nb_step_batched (kz_sweep: nb_step_batched_each, one quench rate per
    instance); value = sum_k N_k^2 x K / device time."""
    import torch
    torch.cuda.set_device(0)
    import paper_2106_11143_gb300 as nb
    from paper_2106_11143_gb300 import workloads as W
    each = args.workload == "kz_sweep"
    k = args.kz_instances
    w = W.kz_quench_sweep(n_inst=k) if each else W.kz_ensemble(n_inst=k)
    off = w["offsets"]
    pairs = float(np.sum(np.diff(off).astype(np.float64) ** 2))
    prec = args.precision if args.precision in ("fp64", "df64") else "fp64"
    if each:
        par = [nb.Params.from_phys(ph, precision=prec) for ph in w["phys"]]
        run = lambda n: nb.step_batched_each(par, sysm, off, n)
    else:
        par = nb.Params.from_phys(w["phys"], precision=prec)
        run = lambda n: nb.step_batched(par, sysm, off, n)
    sysm = nb.System(w["pos"], w["vel"])
    nb.init_batched(par, sysm, off)
    run(args.warmup)
    nb.sync_status()
    lib = nb.lib()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    flush.zero_()
    st = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device())
    l0 = lib.nb_launch_count()
    torch.cuda.synchronize()
    clocks.start()
    a.record(st)
    run(args.steps)
    b.record(st)
    torch.cuda.synchronize()
    clk = clocks.stop()
    nb.sync_status()
    ms = a.elapsed_time(b)
    sizes = np.diff(off)
    order, start, mx, mean = nb.plan_batched(off, min(len(sizes), torch.cuda.get_device_properties(0).multi_processor_count))
    print(json.dumps({
        "metric": "G pair-interactions/s, Kibble-Zurek ensemble (extra line, not the headline)",
        "value": round(pairs * args.steps / (ms / 1e3) / 1e9, 3), "unit": UNIT,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
        "dtype": DTYPE[prec], "precision": prec, "data": "synthetic",
        "config": {"workload": w["name"], "instances": int(len(sizes)), "ions": int(off[-1]),
                   "pairs_per_step": pairs, "launches": int(lib.nb_launch_count() - l0),
                   "lpt_max_over_mean_load": round(mx / mean, 4)},
        "roofline": kz_roofline(nb, prec, pairs, args.steps, ms, clk),
        "clocks": clk}))


def profile_forces(args):
    """Case for ncu: a warm-up pass then a measured pass of nb_forces in each
    precision of --precisions (default fp64, df64, mixed, mixed_split: pair-kernel
    launches 1-4 warm up, 5-8 are the ones to capture)."""
    import torch
    torch.cuda.set_device(0)
    import paper_2106_11143_gb300 as nb
    from paper_2106_11143_gb300 import workloads as W
    w = W.cloud_large(n=args.n)
    sysm = nb.System(w["pos"], w["vel"])
    if args.one_sided:  # the one-sided kernel, as the ladder modes use it at every n
        for prec in ("fp64", "df64", "mixed", "mixed_split"):
            nb.set_tuning("symmetric", prec, 0, 1 << 40, 128, R=0)
    for _ in range(2):
        for prec in args.precisions.split(","):
            nb.forces(nb.Params.from_phys(w["phys"], precision=prec), sysm)
    nb.sync_status()
    print("profile case done: n=%d" % w["n"])


def profile_vjp(args):
    """Small case for ncu: two nb_forces_vjp calls (the adjoint's pair kernel)
    in fp64, then two in df64, at --n on the large-cloud distribution with
    seeded cotangents."""
    import torch
    torch.cuda.set_device(0)
    import paper_2106_11143_gb300 as nb
    from paper_2106_11143_gb300 import workloads as W
    w = W.cloud_large(n=args.n)
    sysm = nb.System(w["pos"], w["vel"])
    lam = np.random.default_rng(1).standard_normal((3, w["n"]))
    for prec in ("fp64", "df64"):
        par = nb.Params.from_phys(w["phys"], precision=prec)
        for _ in range(2):
            nb.forces_vjp(par, sysm, lam)
    nb.sync_status()
    print("profile case done: n=%d" % w["n"])


def profile_small(args):
    """Small case for ncu: fp64 steps of the small-n paths in a static trap.
    First 200 steps at n = 16 (one launch of the single-block kernel), then
    40 steps at n = 1000 (drift, 7 plain steps, 4 replays of the 8-step
    window, the last step: pair kernel and eight-lane epilogue per step)."""
    import math
    import torch
    torch.cuda.set_device(0)
    import paper_2106_11143_gb300 as nb
    from paper_2106_11143_gb300 import workloads as W
    phys = W.phys(omega=(2 * math.pi * 1e6, 2 * math.pi * 1e6, 2 * math.pi * 200e3))
    par = nb.Params.from_phys(phys)
    for n, k in ((16, 200), (1000, 40)):
        c = 4e-6 * (n / (4.0 / 3.0 * math.pi * 25.0)) ** (1.0 / 3.0)
        pos, vel = W.random_cloud(n, seed=21, semi_axes=(c, c, 5 * c))
        s = nb.System(pos, vel)
        nb.forces(par, s, total=True)
        nb.step(par, s, k)
    nb.sync_status()
    print("profile case done")


def cpu_sweep(sizes=(10, 100, 1000, 10000, 100000), target_s=2.0):
    """One force evaluation per N: the FP64 oracle (as it stands) on one host
    core and on all of them, and the GPU (nb_forces, fp64 and mixed_split;
    CUDA events around repeated calls from Python, so small N includes the
    call overhead).  At large N the oracle times ions [0, S) against all N,
    S sized for about target_s seconds, and the rate is scaled to all N."""
    import math
    import torch
    import oracle
    import paper_2106_11143_gb300 as nb
    from paper_2106_11143_gb300 import workloads as W
    nb.lib()
    cores = oracle.get_threads()
    for n in sizes:
        c = 4e-6 * (n / (4.0 / 3.0 * math.pi * 25.0)) ** (1.0 / 3.0)  # about 4 um spacing
        pos, _ = W.random_cloud(n, seed=21, semi_axes=(c, c, 5 * c))
        phys = W.phys(omega=(2 * math.pi * 1e6, 2 * math.pi * 1e6, 2 * math.pi * 200e3))
        p = oracle.make_params(**phys)
        row = {"n": n, "pairs": n * n}
        for k in (1, cores):
            oracle.set_threads(k)
            s, reps, dt = min(n, 64), 1, 0.0
            while True:  # grow the sample (ions, then repetitions) to about target_s
                t = time.perf_counter()
                for _ in range(reps):
                    oracle.coulomb(p, *pos, i0=0, i1=s)
                dt = time.perf_counter() - t
                if dt >= target_s or (s == n and reps >= 1 << 20):
                    break
                grow = max(2.0, min(16.0, target_s / max(dt, 1e-6)))
                if s < n:
                    s = int(min(n, s * grow))
                else:
                    reps = int(reps * grow)
            row["oracle_%dcore_ms" % k] = round(dt / reps * 1e3 * n / s, 6)
            row["oracle_%dcore_sample" % k] = "%d of %d ions x %d" % (s, n, reps)
        oracle.set_threads(cores)
        for prec in ("fp64", "mixed_split"):
            par = nb.Params.from_phys(phys, precision=prec)
            sysm = nb.System(pos)
            for _ in range(3):
                nb.forces(par, sysm)
            torch.cuda.synchronize()
            reps = 2000 if n <= 10000 else 20
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                nb.forces(par, sysm)
            b.record()
            torch.cuda.synchronize()
            row["gpu_%s_ms" % prec] = round(a.elapsed_time(b) / reps, 6)
        nb.sync_status()
        row["cores"] = cores
        row["gpu_fp64_over_oracle_allcores"] = round(row["oracle_%dcore_ms" % cores] / row["gpu_fp64_ms"], 1)
        print(json.dumps(row), flush=True)


# ---------------------------------------------------------------------------
# Step-rate sweep over the paper's 10^1 - 10^5 ion range (Sec. I, Sec. VI):
# for each N and precision the device time of K velocity-Verlet steps through
# nb_step, as ms per step, steps per second and G pair-interactions per second
# (N^2 per step).  At small N a step is a few short kernels, so launch latency
# dominates and the numbers depend on how the steps are issued:
#   ms_per_step          one nb_step call of K steps, the library default
#                        (single-block steps for the smallest N, else the
#                        multi-kernel steps, with replays of a captured 8-step
#                        window for N <= 4096)
#   windows_ms_per_step  the multi-kernel steps with windows (N <= 4096)
#   plain_ms_per_step    the multi-kernel steps without windows
#   per_call_ms_per_step K nb_step calls of one step from Python
#   graph_ms_per_step    K replays of one caller-captured graph of one step
# Inputs: uniform seeded clouds of about 4 um spacing in a static harmonic trap.
SWEEP_PRECISIONS = ["fp64", "df64", "mixed", "mixed_split"]


def _sweep_steps(n):
    return 2000 if n <= 1000 else (200 if n <= 10000 else 10)


def _timed(fn, k):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / k


def time_call(par, sysm, k, precision, small=None, windows=None):
    """One nb_step call of k steps, after one untimed call of the same length;
    small / windows = True or False force the single-block steps or the step
    windows on or off, None keeps the library's default."""
    from paper_2106_11143_gb300 import api
    import torch
    api.set_tuning("force", "fp64", 0, 0, 0)
    if small is not None:
        api.set_tuning("small_steps", precision, 0, 1 << 40, 1, R=int(small))
    if windows is not None:
        api.set_tuning("step_windows", precision, 0, 1 << 40, 1, R=int(windows))
    try:
        api.step(par, sysm, k)
        torch.cuda.synchronize()
        return _timed(lambda: api.step(par, sysm, k), k)
    finally:
        api.set_tuning("force", "fp64", 0, 0, 0)


def time_per_call(par, sysm, k):
    from paper_2106_11143_gb300 import api
    import torch
    api.step(par, sysm, 2)
    torch.cuda.synchronize()

    def run():
        for _ in range(k):
            api.step(par, sysm, 1)
    return _timed(run, k)


def time_graph(par, sysm, k, pos, vel):
    from paper_2106_11143_gb300 import api
    import torch
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        api.step(par, api.System(pos, vel), 1, stream=s)  # this stream's scratch
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        api.step(par, sysm, 1)
    g.replay()
    torch.cuda.synchronize()

    def run():
        for _ in range(k):
            g.replay()
    return _timed(run, k)


def step_sweep(sizes=(10, 100, 1000, 10000, 100000), precisions=SWEEP_PRECISIONS, graphs=True):
    import math
    from paper_2106_11143_gb300 import api
    from paper_2106_11143_gb300 import workloads as W
    out = []
    for n in sizes:
        # about 4 um mean spacing at every N, so the clouds have similar dynamics
        c = 4e-6 * (n / (4.0 / 3.0 * math.pi * 25.0)) ** (1.0 / 3.0)
        pos, vel = W.random_cloud(n, seed=21, semi_axes=(c, c, 5 * c))
        phys = W.phys(omega=(2 * math.pi * 1e6, 2 * math.pi * 1e6, 2 * math.pi * 200e3))
        k = _sweep_steps(n)
        for prec in precisions:
            par = api.Params.from_phys(phys, precision=prec)
            sysm = api.System(pos, vel)
            api.forces(par, sysm, total=True)
            ms = time_call(par, sysm, k, prec)
            row = {"n": n, "precision": prec, "steps": k, "ms_per_step": round(ms, 5),
                   "steps_per_s": round(1e3 / ms, 1), "G_pairs_per_s": round(n * n / ms / 1e6, 4)}
            if n <= 4096:
                row.update(windows_ms_per_step=round(time_call(par, sysm, k, prec, small=False, windows=True), 5))
            if n <= 10000:
                pms = time_call(par, sysm, k, prec, small=False, windows=False)
                row.update(plain_ms_per_step=round(pms, 5), per_call_ms_per_step=round(time_per_call(par, sysm, k), 5))
            if graphs and n <= 10000:
                gms = time_graph(par, sysm, k, pos, vel)
                row.update(graph_ms_per_step=round(gms, 5), graph_steps_per_s=round(1e3 / gms, 1),
                           graph_G_pairs_per_s=round(n * n / gms / 1e6, 4))
            out.append(row)
    return out



if __name__ == "__main__":
    a = parse()
    if a.step_sweep:
        import torch
        torch.cuda.set_device(0)
        for row in step_sweep(tuple(int(v) for v in a.step_sweep.split(","))):
            print(json.dumps(row))
    elif a.peaks:
        main_peaks(a)
    elif a.cpu_sweep:
        cpu_sweep()
    elif a.profile_small:
        profile_small(a)
    elif a.profile_vjp:
        profile_vjp(a)
    elif a.profile_forces:
        profile_forces(a)
    elif a.workload in ("kz", "kz_sweep") and a.impl == "ours":
        main_kz(a)
    elif a.impl == "reference":
        main_reference(a)
    else:
        main_ours(a)
