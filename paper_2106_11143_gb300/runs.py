"""The five workloads end to end, each exactly as configured, with their
device times (CUDA events) and the quantities a user of each would look at.

  cloud-harmonic-N1024   FP64 forces at step 0, then 100 velocity-Verlet steps
  cloud-rf-N16384        1000 steps of the RF trap with friction, FP64
  cloud-large-N100000    50 steps in mixed precision (split) beside FP64: the
                         speed-up and the final-state difference between them
  kz-ensemble            the 512-instance ensemble, FP64, one persistent launch
                         per chunk of steps (a prefix by default; --kz-steps 20000
                         is the full run).  Most of its chains are far denser than
                         a linear chain in this trap can be, so the first steps
                         throw ions out radially (the FP64 oracle does the same);
                         the friction damps that over the full run.
  adjoint-cloud-N4096    trajectory loss and its gradient with respect to the
                         initial positions and the three trap frequencies
                         (checkpoints every 100 steps), with the forward in
                         fp64 and in df64

    python -m paper_2106_11143_gb300.runs [--kz-steps 200]
"""
import argparse
import json

import numpy as np
import torch

from . import api
from . import workloads as W


def _events():
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_steps(w, precision, nsteps, chunk=None):
    """Forces at step 0, then nsteps steps; returns (system, device ms)."""
    par = api.Params.from_phys(w["phys"], precision=precision)
    s = api.System(w["pos"], w["vel"])
    a, b = _events()
    a.record()
    api.forces(par, s, total=True)
    done = 0
    while done < nsteps:
        k = min(chunk or nsteps, nsteps - done)
        api.step(par, s, k)
        done += k
    b.record()
    torch.cuda.synchronize()
    api.sync_status()
    return s, a.elapsed_time(b)


def cloud_run(w, precision, nsteps):
    run_steps(w, precision, min(nsteps, 40))  # untimed: loads the kernels (lazy module loading)
    s, ms = run_steps(w, precision, nsteps)
    n = w["n"]
    e = api.energy(api.Params.from_phys(w["phys"], precision=precision), s)
    return {"workload": w["name"], "precision": precision, "n": n, "steps": nsteps,
            "device_ms": round(ms, 3), "ms_per_step": round(ms / nsteps, 4),
            "G_pairs_per_s": round(n * n * nsteps / ms / 1e6, 2), "final_energy_J": [float(v) for v in e]}


def large_cloud(nsteps=50):
    w = W.cloud_large()
    out = []
    fin = {}
    for prec in ("fp64", "mixed_split"):
        s, ms = run_steps(w, prec, nsteps)
        fin[prec] = s.pos().cpu().numpy()
        n = w["n"]
        out.append({"workload": w["name"], "precision": prec, "n": n, "steps": nsteps,
                    "device_ms": round(ms, 2), "ms_per_step": round(ms / nsteps, 3),
                    "G_pairs_per_s": round(n * n * nsteps / ms / 1e6, 2)})
    scale = np.max(np.abs(fin["fp64"]))
    out[1]["speedup_over_fp64"] = round(out[0]["device_ms"] / out[1]["device_ms"], 2)
    out[1]["max_position_difference_vs_fp64_rel"] = float(np.max(np.abs(fin["mixed_split"] - fin["fp64"])) / scale)
    return out


def kz(nsteps=200, chunk=200):
    w = W.kz_ensemble()
    off = w["offsets"]
    pairs = float(np.sum(np.diff(off).astype(np.float64) ** 2))
    par = api.Params.from_phys(w["phys"])
    s = api.System(w["pos"], w["vel"])
    api.init_batched(par, s, off)
    a, b = _events()
    a.record()
    done = 0
    while done < nsteps:
        k = min(chunk, nsteps - done)
        api.step_batched(par, s, off, k)
        done += k
    b.record()
    torch.cuda.synchronize()
    api.sync_status()
    ms = a.elapsed_time(b)
    x = s.pos().cpu().numpy()
    return {"workload": w["name"], "precision": "fp64", "instances": len(off) - 1, "ions": int(off[-1]),
            "steps": nsteps, "device_s": round(ms / 1e3, 3), "G_pairs_per_s": round(pairs * nsteps / ms / 1e6, 2),
            "max_radial_um": round(float(np.max(np.hypot(x[0], x[1]))) * 1e6, 3)}


def adjoint(precision="fp64"):
    """The adjoint workload with the forward, its recompute and the Jacobian
    products in `precision` (fp64 or df64)."""
    from .autograd import trajectory_loss
    w = W.adjoint_cloud()
    par = api.Params.from_phys(w["phys"], precision=precision)
    x0 = torch.tensor(w["pos"], device="cuda", requires_grad=True)
    v0 = torch.tensor(w["vel"], device="cuda", requires_grad=True)
    om = torch.tensor(w["phys"]["omega"], dtype=torch.float64, device="cuda", requires_grad=True)
    tg = torch.tensor(w["target"], device="cuda")
    a, b = _events()
    c = torch.cuda.Event(enable_timing=True)
    a.record()
    loss = trajectory_loss(x0, v0, om, par, w["steps"], 100, tg)
    b.record()
    loss.backward()
    c.record()
    torch.cuda.synchronize()
    return {"workload": w["name"], "precision": precision, "n": w["n"], "steps": w["steps"], "checkpoint_every": 100,
            "forward_s": round(a.elapsed_time(b) / 1e3, 3), "backward_s": round(b.elapsed_time(c) / 1e3, 3),
            "loss": float(loss.item()), "grad_omega": [float(g) for g in om.grad.cpu()],
            "grad_x0_max_abs": float(x0.grad.abs().max().item())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kz-steps", type=int, default=200)
    args = ap.parse_args()
    torch.cuda.set_device(0)
    rows = [cloud_run(W.cloud_harmonic_1024(), "fp64", 100),
            cloud_run(W.cloud_rf_16384(), "fp64", 1000)]
    rows += large_cloud()
    rows.append(kz(args.kz_steps))
    rows.append(adjoint())
    rows.append(adjoint("df64"))
    for r in rows:
        print(json.dumps(r))


if __name__ == "__main__":
    main()
