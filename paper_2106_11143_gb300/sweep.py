"""Step-rate sweep over the paper's 10^1 - 10^5 ion range (Sec. I, Sec. VI).

For each N and precision: the device time of K velocity-Verlet steps through
nb_step (CUDA events on the launching stream), reported as ms per step, steps
per second and G pair-interactions per second (N^2 per step).  At small N a
step is a few short kernels, so launch latency dominates, and the numbers
depend on how the steps are issued:

  ms_per_step          one nb_step call of K steps, the library default:
                       single-block steps for the smallest N (one launch
                       for the call), else the multi-kernel steps, whose
                       middle steps are replays of a captured 8-step window
                       for N <= 4096
  windows_ms_per_step  the multi-kernel steps with windows (N <= 4096)
  plain_ms_per_step    the multi-kernel steps without windows (one launch
                       per kernel, issued from the library's host loop)
  per_call_ms_per_step K nb_step calls of one step from Python
  graph_ms_per_step    K replays of one caller-captured graph of one step

Inputs: uniform seeded clouds in a static harmonic trap (a caller's graph
repeats the captured step counter, so the trap is static and there is no
noise).

    python -m paper_2106_11143_gb300.sweep [--sizes 10,100,1000,10000,100000]
"""
import argparse
import json
import math

import torch

from . import api
from . import workloads as W

PRECISIONS = ["fp64", "df64", "mixed", "mixed_split"]


def _steps(n):
    return 2000 if n <= 1000 else (200 if n <= 10000 else 10)


def _timed(fn, k):
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
    api.step(par, sysm, 2)
    torch.cuda.synchronize()

    def run():
        for _ in range(k):
            api.step(par, sysm, 1)
    return _timed(run, k)


def time_graph(par, sysm, k, pos, vel):
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


def sweep(sizes=(10, 100, 1000, 10000, 100000), precisions=PRECISIONS, graphs=True):
    out = []
    for n in sizes:
        # about 4 um mean spacing at every N, so the clouds have similar dynamics
        c = 4e-6 * (n / (4.0 / 3.0 * math.pi * 25.0)) ** (1.0 / 3.0)
        pos, vel = W.random_cloud(n, seed=21, semi_axes=(c, c, 5 * c))
        phys = W.phys(omega=(2 * math.pi * 1e6, 2 * math.pi * 1e6, 2 * math.pi * 200e3))
        k = _steps(n)
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", default="10,100,1000,10000,100000")
    ap.add_argument("--precisions", default=",".join(PRECISIONS))
    a = ap.parse_args()
    torch.cuda.set_device(0)
    rows = sweep(tuple(int(s) for s in a.sizes.split(",")), a.precisions.split(","))
    for r in rows:
        print(json.dumps(r))


if __name__ == "__main__":
    main()
