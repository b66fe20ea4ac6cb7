"""The 1/sqrt precision ladder of the paper (Sec. IV-VI) on GB300.

Methods (nb_precision): SQRT+DIV (``sqrtdiv``), the bare hardware seed
(``rsq``, the counterpart of RSQRT14), the seed with one or two
Newton-Raphson steps (``rsq_nr1``, ``rsq_nr2``), and this library's default
``fp64`` (seed + compensated third-order correction) and ``df64``.

speed():  time per force evaluation for each method and N, and the paper's
          speed-up measure relative to SQRT+DIV, 100 (t_SQRT+DIV / t - 1)
          (Sec. VI.B, read with the sign that makes a faster method positive).
chain():  the N = 16 ion-chain comparison of Sec. V: the same trajectory with
          each method; the mean relative difference of the ions' distances
          from the trap centre against SQRT+DIV after the run.

    python -m paper_2106_11143_gb300.ladder [--steps 5000]
"""
import argparse
import json
import math

import numpy as np
import torch

from . import api
from . import workloads as W

METHODS = ["sqrtdiv", "rsq", "rsq_nr1", "rsq_nr2", "fp64", "df64"]


def _time(par, sysm, reps):
    import ctypes as C
    L = api.lib()
    api._check(L.nb_timing_enable(reps), "nb_timing_enable")
    for _ in range(reps):
        api.forces(par, sysm)
    n = C.c_int64()
    ms = C.c_double()
    api._check(L.nb_timing_read(C.byref(n), C.byref(ms)), "nb_timing_read")
    api._check(L.nb_timing_enable(0), "nb_timing_enable")
    return ms.value / max(n.value, 1)


def speed(sizes=(1000, 10000, 100000), methods=METHODS, reps=3):
    out = {}
    for n in sizes:
        pos, vel = W.random_cloud(n, seed=5, semi_axes=(200e-6, 200e-6, 1000e-6))
        sysm = api.System(pos, vel)
        row = {}
        for m in methods:
            par = api.Params.from_phys(W.phys(), precision=m)
            _time(par, sysm, 1)
            t = _time(par, sysm, reps if n >= 100000 else reps * 10)
            row[m] = {"ms": round(t, 5), "G_pairs_per_s": round(n * n / (t / 1e3) / 1e9, 3)}
        base = row["sqrtdiv"]["ms"]
        for m in methods:
            row[m]["speedup_vs_sqrtdiv_pct"] = round(100.0 * (base / row[m]["ms"] - 1.0), 1)
        out[str(n)] = row
    return out


def chain_params(dt=5e-9):
    """Sec. V chain: Omega/2pi = 2 MHz, r0 = 2.5 mm, V_RF = 20 V, omega/2pi =
    1.581 kHz, Gamma = 1e-19 kg/s, Ca+ (40 u).  The RF amplitude is converted
    to the Mathieu q with the prefactor of Eq. 1 and angular Omega:
    q = 4 Q V_RF / (m r0^2 Omega^2)."""
    om = W.TWO_PI * 2e6
    q = 4 * W.E_CHARGE * 20.0 / (W.MASS_40U * (2.5e-3) ** 2 * om ** 2)
    return W.phys(trap="rf", q_mathieu=q, omega_rf=om, omega=(0.0, 0.0, W.TWO_PI * 1.581e3),
                  gamma=1e-19, dt=dt)


def chain(methods=METHODS, steps=5000, n=16, seed=6):
    phys = chain_params()
    rng = np.random.default_rng(seed)
    pos = np.zeros((3, n))
    pos[2] = W.chain_positions(n, phys["omega"][2])
    pos[:2] = 1e-7 * rng.standard_normal((2, n))
    vel = W.thermal_velocities(n, 1e-3, W.MASS_40U, rng)
    final = {}
    for m in methods:
        par = api.Params.from_phys(phys, precision=m)
        s = api.System(pos, vel)
        api.forces(par, s, total=True)
        api.step(par, s, steps)
        api.sync_status()
        final[m] = s.pos().cpu().numpy()
    d0 = np.linalg.norm(final["sqrtdiv"], axis=0)
    res = {"q_mathieu": phys["q_mathieu"], "steps": steps, "dt": phys["dt"], "n": n}
    for m in methods:
        d = np.linalg.norm(final[m], axis=0)
        res[m] = float(np.mean(np.abs((d - d0) / d0)))
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--sizes", default="1000,10000,100000")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    sizes = tuple(int(s) for s in a.sizes.split(","))
    print(json.dumps({"speed": speed(sizes), "chain_dbar": chain(steps=a.steps)}))


if __name__ == "__main__":
    main()
