"""Autotuner for the launch shapes of the pair kernels and the ensemble kernel.

For each (kernel, precision, n bucket) it times candidate shapes -- threads
per block, ions per thread (R) and target (i-tile, j-chunk) blocks per SM for
the one-sided force kernel; ions per block pair, or the one-sided kernel
instead, for the symmetric force kernel --
with the library's own CUDA-event timing of the pair-kernel launches
(nb_timing_*), keeps the fastest, and installs it with nb_set_tuning.  The
ensemble kernel is tuned over threads per block on a Kibble-Zurek-shaped
ensemble.  Results go to a JSON cache keyed by the device name, so a later
process can apply them without re-timing (load()).

    python -m paper_2106_11143_gb300.tune --out tune_cache.json [--quick]

A shape changes only the order of the floating-point summation, so tuned and
untuned results agree to rounding (the ensemble kernel is bitwise shape
independent).
"""
import argparse
import ctypes as C
import json
import os
import time

import torch

from . import api
from . import workloads as W

# n buckets of the one-sided force kernel (the default below n = 500-2000,
# by precision, and for the ladder modes): (lo, hi, representative n)
BUCKETS = [(1, 1500, 1024), (1501, 4095, 3000)]
FORCE_SHAPES = [(b, r, bps) for b in (64, 128, 256) for r in (1, 2, 4) for bps in (4, 8, 16, 32)]
SMALL_SHAPES = [(b, 1, bps) for b in (32, 64, 128) for bps in (8, 16, 32, 64)]


def _time_forces(par, sysm, reps):
    L = api.lib()
    api._check(L.nb_timing_enable(reps), "nb_timing_enable")
    for _ in range(reps):
        api.forces(par, sysm)
    n = C.c_int64()
    ms = C.c_double()
    api._check(L.nb_timing_read(C.byref(n), C.byref(ms)), "nb_timing_read")
    api._check(L.nb_timing_enable(0), "nb_timing_enable")
    return ms.value / max(n.value, 1)


def tune_pair(precision, quick=False, log=print):
    """Best (block, R, blocks_per_sm) per n bucket for the one-sided force
    kernel (the symmetric kernel is switched off while timing)."""
    out = []
    for lo, hi, n in BUCKETS:
        if quick and n < 3000:
            continue
        pos, vel = W.random_cloud(n, seed=1, semi_axes=(200e-6, 200e-6, 1000e-6))
        sysm = api.System(pos, vel)
        par = api.Params.from_phys(W.phys(), precision=precision)
        shapes = SMALL_SHAPES if n < 3001 else FORCE_SHAPES
        if quick:
            shapes = [s for s in shapes if s[2] in (8, 16)]
        reps = 3 if (precision == "fp64" and n >= 100000) else 10
        best = None
        for (b, r, bps) in shapes:
            if not precision.startswith("mixed_split") and r > 1:
                continue
            api.set_tuning("symmetric", precision, lo, hi, 256, R=0)
            api.set_tuning("force", precision, lo, hi, b, r, bps)
            _time_forces(par, sysm, 1)  # warm-up with this shape
            t = _time_forces(par, sysm, reps)
            if best is None or t < best[0]:
                best = (t, b, r, bps)
        api.set_tuning("force", precision, 0, 0, 0)  # clear
        t, b, r, bps = best
        log("force %-11s n=%-7d best block=%d R=%d blocks/SM=%d  %.4f ms" % (precision, n, b, r, bps, t))
        out.append(dict(kind="force", precision=precision, n_lo=lo, n_hi=hi, block=b, R=r,
                        blocks_per_sm=bps, ms=t))
    return out


SYM_BUCKETS = [(500, 1499, 1000), (1500, 2499, 2000), (2500, 4095, 3000), (4096, 10000, 8192),
               (10001, 40000, 16384), (40001, 1 << 31, 100000)]
SYM_BLOCKS = (32, 64, 128, 256, 512, 1024)


def _time_step(par, sysm, reps):
    """Device time of one velocity-Verlet step (pair kernel and epilogue), ms."""
    api.step(par, sysm, 1)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    api.step(par, sysm, reps)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def tune_symmetric(precision, quick=False, log=print):
    """Best ions per block pair of the symmetric force kernel, or the one-sided
    kernel (R = 0), per n bucket, timed as whole steps so that the epilogue's
    reads of the per-partner-block partials count."""
    out = []
    for lo, hi, n in SYM_BUCKETS:
        if quick and n < 100000:
            continue
        pos, vel = W.random_cloud(n, seed=1, semi_axes=(200e-6, 200e-6, 1000e-6))
        sysm = api.System(pos, vel)
        par = api.Params.from_phys(W.phys(), precision=precision)
        api.forces(par, sysm, total=True)
        reps = 2 if (n >= 100000 and precision == "fp64") else 10
        best = None
        for block, use in [(b, 1) for b in SYM_BLOCKS] + [(256, 0)]:
            api.set_tuning("symmetric", precision, lo, hi, block, R=use)
            t = _time_step(par, sysm, reps)
            if best is None or t < best[0]:
                best = (t, block, use)
        api.set_tuning("symmetric", precision, 0, 0, 0)
        t, block, use = best
        log("symmetric %-11s n=%-7d best %s  %.4f ms/step" % (precision, n, ("block=%d" % block) if use else "one-sided", t))
        out.append(dict(kind="symmetric", precision=precision, n_lo=lo, n_hi=hi, block=block, R=use,
                        blocks_per_sm=1, ms=t))
    return out


def tune_ensemble(quick=False, log=print):
    w = W.kz_ensemble()
    off = w["offsets"]
    par = api.Params.from_phys(w["phys"])
    best = None
    for threads in ((256, 512) if quick else (128, 256, 384, 512)):
        api.set_tuning("ensemble", "fp64", 0, 1 << 40, threads)
        sysm = api.System(w["pos"], w["vel"])
        api.init_batched(par, sysm, off)
        api.step_batched(par, sysm, off, 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        api.step_batched(par, sysm, off, 2)
        torch.cuda.synchronize()
        t = (time.perf_counter() - t0) / 2 * 1e3
        if best is None or t < best[0]:
            best = (t, threads)
    api.set_tuning("ensemble", "fp64", 0, 0, 0)
    log("ensemble best threads=%d  %.2f ms/step" % (best[1], best[0]))
    return [dict(kind="ensemble", precision="fp64", n_lo=0, n_hi=1 << 40, block=best[1], R=1,
                 blocks_per_sm=1, ms=best[0])]


def apply(entries):
    for e in entries:
        api.set_tuning(e["kind"], e["precision"], e["n_lo"], e["n_hi"], e["block"], e["R"],
                       e["blocks_per_sm"])


def load(path):
    """Apply a cache written by this module if it was made on this device."""
    if not os.path.exists(path):
        return False
    d = json.load(open(path))
    if d.get("device") != torch.cuda.get_device_name():
        return False
    apply(d["entries"])
    return True


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="tune_cache.json")
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--precisions", default="fp64,df64,mixed,mixed_split")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    entries = []
    for prec in a.precisions.split(","):
        entries += tune_pair(prec, quick=a.quick)
        entries += tune_symmetric(prec, quick=a.quick)
    entries += tune_ensemble(quick=a.quick)
    json.dump({"device": torch.cuda.get_device_name(), "entries": entries}, open(a.out, "w"), indent=1)
    print("wrote", a.out)


if __name__ == "__main__":
    main()
