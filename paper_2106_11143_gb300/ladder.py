"""The 1/sqrt precision ladder of the paper (Sec. IV-VI) on GB300.

Methods (nb_precision): SQRT+DIV (``sqrtdiv``), the bare hardware seed
(``rsq``, the counterpart of RSQRT14), the seed with one or two
Newton-Raphson steps (``rsq_nr1``, ``rsq_nr2``), and this library's default
``fp64`` (seed + compensated third-order correction) and ``df64``.

speed():   time per force evaluation for each method and N, and the paper's
           speed-up measure relative to SQRT+DIV, 100 (t_SQRT+DIV / t - 1)
           (Sec. VI.B, read with the sign that makes a faster method positive).
           Every method runs on the same one-sided kernel, so the comparison
           isolates the 1/sqrt method; the symmetric (half-pair) kernel of the
           fp64 and df64 paths is timed beside them as fp64_sym and df64_sym.
chain():   the N = 16 ion-chain comparison of Sec. V: the same trajectory with
           each method; the mean relative difference of the ions' distances
           from the trap centre against SQRT+DIV after the run.
pancake(): the N = 128 radial-plane (2D) crystal of Sec. V, compared the same
           way from a common crystal (a disc start cooled with SQRT+DIV).  The printed drive (V_RF = 352 V with the chain's Omega and r0)
           puts the Mathieu q near 3.4, outside the stability region, and a
           1.581 kHz axial frequency cannot flatten a crystal into the radial
           plane; this keeps the experiment's form with the chain's RF drive
           (q = 0.196, radial secular frequency about 2 pi 138 kHz), an axial
           frequency of 2 pi 700 kHz (a single radial plane for 128 ions) and
           the stated Gamma = 1e-21 kg/s.

    python -m paper_2106_11143_gb300.ladder [--steps 5000] [--pancake-steps 880000] [--speed-only]
"""
import argparse
import json

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


SYMMETRIC = ("fp64", "df64")


def speed(sizes=(1000, 10000, 100000), methods=METHODS, reps=3):
    out = {}
    for n in sizes:
        pos, vel = W.random_cloud(n, seed=5, semi_axes=(200e-6, 200e-6, 1000e-6))
        sysm = api.System(pos, vel)
        row = {}
        runs = [(m, m, False) for m in methods]
        runs += [(m + "_sym", m, True) for m in SYMMETRIC if m in methods and n >= 4096]
        for name, m, sym in runs:
            par = api.Params.from_phys(W.phys(), precision=m)
            try:
                if not sym and m in SYMMETRIC:  # the one-sided kernel, as for the other methods
                    api.set_tuning("symmetric", m, 1, 1 << 40, 256, R=0)
                _time(par, sysm, 1)
                t = _time(par, sysm, reps if n >= 100000 else reps * 10)
            finally:
                api.set_tuning("symmetric", m, 0, 0, 0)
            row[name] = {"ms": round(t, 5), "G_pairs_per_s": round(n * n / (t / 1e3) / 1e9, 3)}
        base = row["sqrtdiv"]["ms"]
        for name in row:
            row[name]["speedup_vs_sqrtdiv_pct"] = round(100.0 * (base / row[name]["ms"] - 1.0), 1)
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


def _compare(phys, pos, vel, methods, steps, step0=0):
    """Run the same start with each method; d-bar of Sec. V against SQRT+DIV:
    the mean over ions of |d - d0| / d0, d the distance from the trap centre."""
    final = {}
    for m in methods:
        par = api.Params.from_phys(phys, precision=m)
        s = api.System(pos, vel, step=step0)
        api.forces(par, s, total=True)
        api.step(par, s, steps)
        api.sync_status()
        final[m] = s.pos().cpu().numpy()
    d0 = np.linalg.norm(final["sqrtdiv"], axis=0)
    res = {"q_mathieu": phys["q_mathieu"], "steps": steps, "dt": phys["dt"], "n": pos.shape[1]}
    for m in methods:
        d = np.linalg.norm(final[m], axis=0)
        res[m] = float(np.mean(np.abs((d - d0) / d0)))
    return res, final


def chain(methods=METHODS, steps=5000, n=16, seed=6):
    phys = chain_params()
    rng = np.random.default_rng(seed)
    pos = np.zeros((3, n))
    pos[2] = W.chain_positions(n, phys["omega"][2])
    pos[:2] = 1e-7 * rng.standard_normal((2, n))
    vel = W.thermal_velocities(n, 1e-3, W.MASS_40U, rng)
    return _compare(phys, pos, vel, methods, steps)[0]


def pancake_params(dt=5e-9):
    """The chain's RF drive with a strong axial confinement (see the module
    docstring for the reading of the printed parameters)."""
    p = chain_params(dt)
    p.update(omega=(0.0, 0.0, W.TWO_PI * 700e3), gamma=1e-21)
    return p


def pancake(methods=METHODS, steps=880000, n=128, seed=7, quench_steps=20000, relax_steps=100000):
    """E2: N = 128 ions started on a disc in the radial plane (radius 80 um,
    0.5 um axial jitter, 1 mK) are cooled into a crystal with SQRT+DIV:
    quench_steps with 100x the stated friction, then relax_steps with the
    stated Gamma, after which the RF-driven crystal is regular (1.6e-5 K).
    Every method then runs `steps` steps from that common state with the
    stated Gamma (1e6 steps in all by default, as in the paper).  The
    comparison is of crystals, as in the chain case: from the random start,
    or during the switch from the quench friction to the stated one, the
    motion is chaotic and d-bar is O(0.1) even between methods that differ
    only in FP64 rounding.  Returns d-bar per method and the flatness of the
    final SQRT+DIV crystal, max |z| / max radius."""
    phys = pancake_params()
    rng = np.random.default_rng(seed)
    rad = 80e-6 * np.sqrt(rng.uniform(size=n))
    ang = W.TWO_PI * rng.uniform(size=n)
    pos = np.stack([rad * np.cos(ang), rad * np.sin(ang), 0.5e-6 * rng.standard_normal(n)])
    vel = W.thermal_velocities(n, 1e-3, W.MASS_40U, rng)
    s = api.System(pos, vel)
    for g, k in ((100.0 * phys["gamma"], quench_steps), (phys["gamma"], relax_steps)):
        par = api.Params.from_phys(dict(phys, gamma=g), precision="sqrtdiv")
        api.forces(par, s, total=True)
        api.step(par, s, k)
    api.sync_status()
    pos, vel = s.pos().cpu().numpy(), s.vel().cpu().numpy()
    res, final = _compare(phys, pos, vel, methods, steps, step0=s.step)
    res["quench_steps"], res["relax_steps"] = quench_steps, relax_steps
    f = final["sqrtdiv"]
    res["flatness"] = float(np.max(np.abs(f[2])) / np.max(np.hypot(f[0], f[1])))
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--pancake-steps", type=int, default=880000)
    ap.add_argument("--sizes", default="1000,10000,100000")
    ap.add_argument("--speed-only", action="store_true", help="only the force-evaluation timings")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    sizes = tuple(int(s) for s in a.sizes.split(","))
    if a.speed_only:
        print(json.dumps({"speed": speed(sizes)}))
        return
    print(json.dumps({"speed": speed(sizes), "chain_dbar": chain(steps=a.steps),
                      "pancake_dbar": pancake(steps=a.pancake_steps)}))


if __name__ == "__main__":
    main()
