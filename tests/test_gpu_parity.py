"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Error measure for forces: the conditioned error per ion
    e_i = |a_i^gpu - a_i^oracle| / sum_{j != i} |a_ij|,
(the oracle also returns the sum of the pair-term magnitudes), gated at
1e-12 for the FP64 path and 1e-6 for the mixed paths.  The plain relative
error |da|/|a| is ill-conditioned for ions whose pair forces cancel.
"""
import math

import numpy as np
import pytest
import torch

from paper_2106_11143_gb300 import workloads as W

import floors

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "df64": 1e-12, "mixed": 1e-6, "mixed_split": 1e-6, "mixed_split_rsq": 1e-6}
ALL = ["fp64", "df64", "mixed", "mixed_split", "mixed_split_rsq"]


@pytest.fixture(scope="module")
def nb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_11143_gb300 as nbm
    nbm.lib()
    return nbm


def oparams(orc, phys):
    return orc.make_params(**phys)


def cond_err(gpu, ref, absf):
    d = np.sqrt(np.sum((np.asarray(gpu) - np.asarray(ref)) ** 2, axis=0))
    return float(np.max(d / absf))


def gpu_forces(nb, phys, pos, q=None, precision="fp64", total=False, vel=None, step=0):
    sysm = nb.System(pos, vel, q=q, step=step)
    par = nb.Params.from_phys(phys, precision=precision)
    nb.forces(par, sysm, total=total)
    nb.sync_status()
    return sysm.acc().cpu().numpy()


SIZES = [1, 2, 3, 31, 32, 33, 63, 64, 65, 127, 129, 255, 257, 1000, 1024, 2049, 4097, 8191, 9000]


@pytest.mark.parametrize("precision", ALL)
def test_forces_ragged_sizes(nb, orc, precision):
    phys = W.phys()
    worst = 0.0
    for k, n in enumerate(SIZES):
        pos, _ = W.random_cloud(n, seed=100 + k)
        g = gpu_forces(nb, phys, pos, precision=precision)
        if n == 1:
            assert np.all(g == 0)
            continue
        ax, ay, az, _, absf = orc.coulomb(oparams(orc, phys), *pos, want_absf=True)
        e = cond_err(g, np.stack([ax, ay, az]), absf)
        worst = max(worst, e)
        assert e <= TOL[precision], (n, e)
    print("max conditioned error %s: %.3g" % (precision, worst))


@pytest.mark.parametrize("precision", ALL)
def test_forces_charges_and_softening(nb, orc, precision):
    rng = np.random.default_rng(7)
    n = 3001
    pos, _ = W.random_cloud(n, seed=7)
    q = W.E_CHARGE * rng.choice([-1.0, 1.0, 2.0], size=n)
    for soft2 in (0.0, (0.2e-6) ** 2):
        phys = W.phys(soft2=soft2)
        g = gpu_forces(nb, phys, pos, q=q, precision=precision)
        ax, ay, az, _, absf = orc.coulomb(oparams(orc, phys), *pos, q=q, want_absf=True)
        e = cond_err(g, np.stack([ax, ay, az]), absf)
        assert e <= TOL[precision], (soft2, e)


def test_forces_total_rf_trap_friction(nb, orc):
    w = W.cloud_rf_16384(n=2000)
    phys = dict(w["phys"])
    step = 37
    g = gpu_forces(nb, phys, w["pos"], vel=w["vel"], total=True, step=step)
    t = phys["t0"] + step * phys["dt"]
    ref = np.stack(orc.accel(oparams(orc, phys), t, *w["pos"], *w["vel"]))
    _, _, _, _, absf = orc.coulomb(oparams(orc, phys), *w["pos"], want_absf=True)
    scale = absf + np.sqrt(np.sum(ref ** 2, axis=0))
    assert cond_err(g, ref, scale) <= 1e-12


def test_potential_and_energy(nb, orc):
    for trap in ("harmonic", "rf"):
        w = W.cloud_harmonic_1024(n=1500) if trap == "harmonic" else W.cloud_rf_16384(n=1500)
        phys = w["phys"]
        sysm = nb.System(w["pos"], w["vel"], step=11)
        par = nb.Params.from_phys(phys)
        phi = nb.forces(par, sysm, want_phi=True).cpu().numpy()
        _, _, _, phi_ref, _ = orc.coulomb(oparams(orc, phys), *w["pos"], want_phi=True)
        assert np.max(np.abs(phi - phi_ref) / phi_ref) <= 1e-12
        e = nb.energy(par, sysm)
        e_ref = orc.energy(oparams(orc, phys), 11, *w["pos"], *w["vel"])
        for k in range(3):
            assert abs(e[k] - e_ref[k]) <= 1e-12 * abs(e_ref[k]), (trap, k, e[k], e_ref[k])


def test_energy_with_softening_and_charges(nb, orc):
    rng = np.random.default_rng(3)
    n = 700
    pos, vel = W.random_cloud(n, seed=31)
    q = W.E_CHARGE * rng.choice([1.0, 2.0], size=n)
    phys = W.phys(soft2=(0.3e-6) ** 2, omega=(1e6, 2e6, 3e5))
    sysm = nb.System(pos, vel, q=q)
    e = nb.energy(nb.Params.from_phys(phys), sysm)
    e_ref = orc.energy(oparams(orc, phys), 0, *pos, *vel, q=q)
    assert np.all(np.abs(e - e_ref) <= 1e-12 * np.abs(e_ref))


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_vjp(nb, orc, precision):
    rng = np.random.default_rng(5)
    n = 1500
    pos, _ = W.random_cloud(n, seed=5)
    q = W.E_CHARGE * rng.choice([1.0, 2.0], size=n)
    lam = rng.standard_normal((3, n))
    phys = W.phys(omega=(6e6, 5e6, 1.2e6))
    for total in (False, True):
        sysm = nb.System(pos, q=q)
        g = nb.forces_vjp(nb.Params.from_phys(phys, precision=precision), sysm, lam, total=total).cpu().numpy()
        ref = np.stack(orc.forces_vjp(oparams(orc, phys), 0.0, *pos, *lam, q=q, include_trap=total))
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(g - ref)) <= 1e-11 * scale


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_vjp_symmetric_kernel(nb, orc, precision):
    """The half-pair VJP kernel (on from n = 2500), forced on at small and
    ragged sizes with both block sizes, with charges and softening, against the
    oracle; and against the one-sided VJP kernel at n = 4100."""
    rng = np.random.default_rng(6)
    Pm = lambda phys: nb.Params.from_phys(phys, precision=precision)
    try:
        for k, (n, block) in enumerate([(2, 128), (129, 128), (1000, 128), (1500, 256), (4100, 128)]):
            nb.set_tuning("symmetric_vjp", "fp64", 1, 1 << 40, block, R=1)
            pos, _ = W.random_cloud(n, seed=400 + k)
            q = W.E_CHARGE * rng.choice([-1.0, 1.0, 2.0], size=n) if k % 2 else None
            lam = rng.standard_normal((3, n))
            phys = W.phys(omega=(6e6, 5e6, 1.2e6), soft2=(0.1e-6) ** 2 if k == 2 else 0.0)
            g = nb.forces_vjp(Pm(phys), nb.System(pos, q=q), lam, total=True).cpu().numpy()
            ref = np.stack(orc.forces_vjp(oparams(orc, phys), 0.0, *pos, *lam, q=q, include_trap=True))
            assert np.max(np.abs(g - ref)) <= 1e-11 * np.max(np.abs(ref)), (n, block)
            g2 = nb.forces_vjp(Pm(phys), nb.System(pos, q=q), lam, total=True).cpu().numpy()
            assert np.array_equal(g, g2)
        nb.set_tuning("symmetric_vjp", "fp64", 1, 1 << 40, 128, R=0)
        one = nb.forces_vjp(Pm(phys), nb.System(pos, q=q), lam, total=True).cpu().numpy()
    finally:
        nb.set_tuning("force", "fp64", 0, 0, 0)
    assert not np.array_equal(one, g)  # genuinely the other kernel
    assert np.max(np.abs(one - g)) <= 1e-11 * np.max(np.abs(g))


def _vjp_term_bound(pos, lam, q, k_c, mass):
    """Per ion, a bound on the sum of its VJP term magnitudes:
    |k_C q_i / m| sum_j |q_j| 4 |lam_i - lam_j| / r_ij^3 (|T| <= 4 |dl| r^-3)."""
    n = pos.shape[1]
    out = np.empty(n)
    for i0 in range(0, n, 512):
        i1 = min(n, i0 + 512)
        d = pos[:, i0:i1, None] - pos[:, None, :]
        r = np.sqrt(np.sum(d * d, axis=0))
        dl = np.sqrt(np.sum((lam[:, i0:i1, None] - lam[:, None, :]) ** 2, axis=0))
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.where(r > 0, 4.0 * np.abs(q)[None, :] * dl / r ** 3, 0.0)
        out[i0:i1] = np.abs(k_c * q[i0:i1] / mass) * np.sum(t, axis=1)
    return out


@pytest.mark.parametrize("n", [1500, 6000])
def test_vjp_extreme_units(nb, orc, n):
    """The VJP forms each pair's term in that pair's own units and sums the
    terms in block-floating double-float.  Stress the units: a cloud 1 cm off
    the origin (a position scale far above the spacing), cotangents spread
    over 20 decades, a pair 10 nm apart, charges; the one-sided (n = 1500) and
    the half-pair (n = 6000) kernels.  Gate per ion: the error against the
    oracle within 1e-12 of a bound on the sum of the ion's term magnitudes.
    NB_FP64 and NB_DF64 share the VJP arithmetic, so they agree bit for bit."""
    rng = np.random.default_rng(n)
    pos, _ = W.random_cloud(n, seed=n)
    pos = pos + np.array([[1e-2], [0.0], [-3e-3]])
    pos[:, 1] = pos[:, 0] + np.array([1e-8, 0.0, 0.0])
    q = W.E_CHARGE * rng.choice([1.0, 2.0], size=n)
    lam = rng.standard_normal((3, n)) * 10.0 ** rng.uniform(-10, 10, size=n)
    phys = W.phys(omega=(6e6, 5e6, 1.2e6))
    ref = np.stack(orc.forces_vjp(oparams(orc, phys), 0.0, *pos, *lam, q=q))
    bound = _vjp_term_bound(pos, lam, q, W.K_COULOMB, W.MASS_40U)
    out = {}
    for prec in ("fp64", "df64"):
        out[prec] = nb.forces_vjp(nb.Params.from_phys(phys, precision=prec), nb.System(pos, q=q),
                                  lam).cpu().numpy()
        err = np.max(np.sqrt(np.sum((out[prec] - ref) ** 2, axis=0)) / bound)
        print("%s n=%d: max conditioned error %.3g" % (prec, n, err))
        assert err <= 1e-12, prec
    assert np.array_equal(out["fp64"], out["df64"])


@pytest.mark.parametrize("n", [1500, 3000])
def test_vjp_no_unit_cap(nb, orc, n):
    """A pair far closer than the cloud's extent is exact, since every pair
    is scaled by its own exponents: a pair 0.1 nm apart in a cloud 1 cm off
    the origin (2^-27 of the position scale), one-sided and half-pair
    kernels."""
    rng = np.random.default_rng(n + 3)
    pos, _ = W.random_cloud(n, seed=n + 3)
    pos = pos + np.array([[1e-2], [0.0], [-3e-3]])
    pos[:, 1] = pos[:, 0] + np.array([0.0, 1e-10, 0.0])
    lam = rng.standard_normal((3, n))
    phys = W.phys(omega=(6e6, 5e6, 1.2e6))
    q = np.full(n, W.E_CHARGE)
    ref = np.stack(orc.forces_vjp(oparams(orc, phys), 0.0, *pos, *lam))
    bound = _vjp_term_bound(pos, lam, q, W.K_COULOMB, W.MASS_40U)
    g = nb.forces_vjp(nb.Params.from_phys(phys), nb.System(pos), lam).cpu().numpy()
    err = np.max(np.sqrt(np.sum((g - ref) ** 2, axis=0)) / bound)
    print("n=%d: conditioned error %.3g" % (n, err))
    assert err <= 1e-12


@pytest.mark.parametrize("n", [1500, 3000])
def test_vjp_block_floating_sums(nb, orc, n):
    """The VJP sums each 32-partner tile in double-float with one
    exponent per accumulator, rescaled when a term of a larger unit arrives.
    Stress the rescaling: weights (charges) spread over 80 decades with both
    signs, cotangents over 20 decades, a pair 10 nm apart and two ions with
    equal cotangents (a vanishing term besides the self pairs); the one-sided
    (n = 1500) and the half-pair (n = 3000) kernels.  Gate per ion: 1e-12 of
    the bound on the sum of the ion's term magnitudes."""
    rng = np.random.default_rng(n + 7)
    pos, _ = W.random_cloud(n, seed=n + 7)
    pos[:, 1] = pos[:, 0] + np.array([1e-8, 0.0, 0.0])
    q = W.E_CHARGE * rng.choice([-1.0, 1.0], size=n) * 10.0 ** rng.uniform(-40, 40, size=n)
    lam = rng.standard_normal((3, n)) * 10.0 ** rng.uniform(-10, 10, size=n)
    lam[:, 5] = lam[:, 4]
    phys = W.phys(omega=(6e6, 5e6, 1.2e6))
    ref = np.stack(orc.forces_vjp(oparams(orc, phys), 0.0, *pos, *lam, q=q))
    bound = _vjp_term_bound(pos, lam, q, W.K_COULOMB, W.MASS_40U)
    g = nb.forces_vjp(nb.Params.from_phys(phys), nb.System(pos, q=q), lam).cpu().numpy()
    assert np.all(np.isfinite(g))
    err = np.max(np.sqrt(np.sum((g - ref) ** 2, axis=0)) / bound)
    print("fp64 n=%d: max conditioned error %.3g" % (n, err))
    assert err <= 1e-12


def _oracle_traj(orc, phys, pos, vel, nsteps, reverse=False, q=None, eps=0.0):
    p = oparams(orc, phys)
    pos = np.asarray(pos) * (1.0 + eps)
    ax, ay, az = orc.accel(p, phys["t0"], *pos, *vel, q=q, reverse=reverse)
    st = dict(x=pos[0], y=pos[1], z=pos[2], vx=vel[0], vy=vel[1], vz=vel[2],
              ax=ax, ay=ay, az=az, step=0)
    return orc.run(p, st, nsteps, q=q, reverse=reverse)


def _self_divergence(orc, phys, pos, vel, nsteps, ref):
    """How far two correct FP64 computations of the same trajectory drift
    apart: the oracle against itself with the j order reversed and with the
    initial positions moved by one ulp (2^-52 relative).  The compensated
    oracle sums are order-independent, so the second term dominates."""
    rev = _oracle_traj(orc, phys, pos, vel, nsteps, reverse=True)
    ulp = _oracle_traj(orc, phys, pos, vel, nsteps, eps=2.0 ** -52)
    a = _traj_errs_np(ref, rev)
    b = _traj_errs_np(ref, ulp)
    return max(a[0], b[0]), max(a[1], b[1])


def _gpu_traj(nb, phys, pos, vel, nsteps, precision="fp64", chunks=1, q=None):
    sysm = nb.System(pos, vel, q=q)
    par = nb.Params.from_phys(phys, precision=precision)
    nb.forces(par, sysm, total=True)
    for c in range(chunks):
        nb.step(par, sysm, nsteps // chunks)
    nb.sync_status()
    return sysm


def _assert_traj_per_ion(orc, phys, pos0, sysm, ref, nsteps, tol_p, tol_v):
    """Per ion: |x_gpu - x_oracle| <= tol_p + the force contract's position
    floor of that ion, and the same for velocities (floors.contract_floor)."""
    gp = sysm.pos().cpu().numpy()
    gv = sysm.vel().cpu().numpy()
    rp = np.stack([ref["x"], ref["y"], ref["z"]])
    rv = np.stack([ref["vx"], ref["vy"], ref["vz"]])
    fp, fv = floors.contract_floor(orc, oparams(orc, phys), [pos0, rp], nsteps, phys["dt"], vels=[rv])
    ep, ev = floors.per_ion(gp - rp), floors.per_ion(gv - rv)
    assert np.all(ep <= tol_p + fp), (int(np.argmax(ep - fp)), float(np.max(ep - tol_p - fp)))
    assert np.all(ev <= tol_v + fv), (int(np.argmax(ev - fv)), float(np.max(ev - tol_v - fv)))


def _traj_errs(sysm, ref):
    gp = sysm.pos().cpu().numpy()
    gv = sysm.vel().cpu().numpy()
    rp = np.stack([ref["x"], ref["y"], ref["z"]])
    rv = np.stack([ref["vx"], ref["vy"], ref["vz"]])
    return np.max(np.abs(gp - rp)), np.max(np.abs(gv - rv))


@pytest.mark.parametrize("which,precision", [("harmonic", "fp64"), ("rf", "fp64"), ("harmonic", "df64")])
def test_trajectory_parity(nb, orc, which, precision):
    """Trajectories: GPU vs oracle within 10x the oracle's own divergence (see
    _self_divergence), with a floor of 1e-14 of the cloud size / thermal speed."""
    if which == "harmonic":
        w = W.cloud_harmonic_1024()
        nsteps = 100
    else:
        w = W.cloud_rf_16384(n=2048)
        nsteps = 200
    phys = w["phys"]
    ref = _oracle_traj(orc, phys, w["pos"], w["vel"], nsteps)
    sysm = _gpu_traj(nb, phys, w["pos"], w["vel"], nsteps, precision=precision, chunks=2)
    assert sysm.step == nsteps
    dp_self, dv_self = _self_divergence(orc, phys, w["pos"], w["vel"], nsteps, ref)
    dp, dv = _traj_errs(sysm, ref)
    L = np.max(np.abs(w["pos"]))
    V = math.sqrt(W.K_B * 10e-3 / W.MASS_40U)
    print("%s: gpu dp=%.3g dv=%.3g | oracle self dp=%.3g dv=%.3g" % (which, dp, dv, dp_self, dv_self))
    # 10x the oracle's own one-ulp sensitivity, plus, per ion, the drift the
    # force contract allows (floors.contract_floor)
    _assert_traj_per_ion(orc, phys, w["pos"], sysm, ref, nsteps, max(10 * dp_self, 1e-14 * L),
                         max(10 * dv_self, 1e-14 * V))


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_trajectory_full_size_rf(nb, orc, precision):
    """The RF workload at its full N = 16384, where nb_step runs the symmetric
    kernel (as the bench does from n = 16384): 20 steps of the time-dependent
    trap with friction against the oracle, same tolerance as above."""
    w = W.cloud_rf_16384()
    phys, nsteps = w["phys"], 20
    ref = _oracle_traj(orc, phys, w["pos"], w["vel"], nsteps)
    sysm = _gpu_traj(nb, phys, w["pos"], w["vel"], nsteps, precision=precision, chunks=2)
    dp_self, dv_self = _self_divergence(orc, phys, w["pos"], w["vel"], nsteps, ref)
    dp, dv = _traj_errs(sysm, ref)
    L = np.max(np.abs(w["pos"]))
    V = math.sqrt(W.K_B * 10e-3 / W.MASS_40U)
    print("rf N=16384 %s: gpu dp=%.3g dv=%.3g | oracle self dp=%.3g dv=%.3g" % (precision, dp, dv, dp_self, dv_self))
    _assert_traj_per_ion(orc, phys, w["pos"], sysm, ref, nsteps, max(10 * dp_self, 1e-14 * L),
                         max(10 * dv_self, 1e-14 * V))


def _traj_errs_np(a, b):
    ap = np.stack([a["x"], a["y"], a["z"]]); bp = np.stack([b["x"], b["y"], b["z"]])
    av = np.stack([a["vx"], a["vy"], a["vz"]]); bv = np.stack([b["vx"], b["vy"], b["vz"]])
    return np.max(np.abs(ap - bp)), np.max(np.abs(av - bv))


def test_trajectory_langevin_noise(nb, orc):
    """Langevin kicks drawn from the same Philox stream on both sides."""
    w = W.kz_ensemble(n_inst=1, n_min=300, n_max=300, steps=20000)
    phys = dict(w["phys"])
    pos, vel = w["pos"], w["vel"]
    nsteps = 300
    ref = _oracle_traj(orc, phys, pos, vel, nsteps)
    sysm = _gpu_traj(nb, phys, pos, vel, nsteps, chunks=3)
    dp_self, dv_self = _self_divergence(orc, phys, pos, vel, nsteps, ref)
    dp, dv = _traj_errs(sysm, ref)
    V = math.sqrt(W.K_B * 0.5e-3 / W.MASS_40U)
    print("langevin: gpu dp=%.3g dv=%.3g | self dp=%.3g dv=%.3g" % (dp, dv, dp_self, dv_self))
    # the kick is ~0.04 V per step: a wrong noise stream would differ by ~V
    assert dv <= 10 * dv_self + 1e-14 * V
    assert dp <= 10 * dp_self + 1e-14 * V * phys["dt"] * nsteps


def test_step_determinism_and_resume(nb):
    """Bitwise: two identical runs agree; 2 x 25 steps == 50 steps."""
    w = W.cloud_harmonic_1024(n=3000)
    a = _gpu_traj(nb, w["phys"], w["pos"], w["vel"], 50, chunks=1)
    b = _gpu_traj(nb, w["phys"], w["pos"], w["vel"], 50, chunks=1)
    c = _gpu_traj(nb, w["phys"], w["pos"], w["vel"], 50, chunks=2)
    for t in ("x", "vx", "az"):
        assert torch.equal(getattr(a, t), getattr(b, t))
        assert torch.equal(getattr(a, t), getattr(c, t))


def test_checkpoint_resume_bitwise(nb, tmp_path):
    """A run checkpointed to a file after 15 steps (System.state_dict through
    torch.save, and save_checkpoint's framework-free file with the params) and
    resumed in a fresh System continues bit for bit as the uninterrupted run:
    RF trap (time from the step counter), friction and Langevin noise (the
    Philox counter includes the step)."""
    w = W.cloud_rf_16384(n=2000)
    phys = dict(w["phys"], noise_T=0.5e-3)
    par = nb.Params.from_phys(phys)
    a = nb.System(w["pos"], w["vel"])
    nb.forces(par, a, total=True)
    nb.step(par, a, 30)
    b = nb.System(w["pos"], w["vel"])
    nb.forces(par, b, total=True)
    nb.step(par, b, 15)
    nb.sync_status()
    torch.save(b.state_dict(), tmp_path / "ckpt.pt")
    nb.save_checkpoint(tmp_path / "ckpt.nbck", b, par)
    c = nb.System.from_state(torch.load(tmp_path / "ckpt.pt"))
    d, dpar = nb.load_checkpoint(tmp_path / "ckpt.nbck")  # the framework-free file, with its params
    assert c.step == 15 and d.step == 15 and dpar == par
    nb.step(par, c, 15)
    nb.step(dpar, d, 15)
    nb.sync_status()
    for t in ("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az"):
        assert torch.equal(getattr(a, t), getattr(c, t)), t
        assert torch.equal(getattr(a, t), getattr(d, t)), t


@pytest.mark.parametrize("precision", ALL)
def test_full_size_sampled(nb, orc, precision):
    """N = 1e5 (the large-cloud workload, launch configuration of the bench):
    all forces on the GPU, a sample of 192 ions (spread over tiles and the
    ragged tail) by the oracle one by one."""
    w = W.cloud_large()
    phys = w["phys"]
    g = gpu_forces(nb, phys, w["pos"], precision=precision)
    n = w["n"]
    idx = np.unique(np.concatenate([np.arange(0, 64), np.arange(n - 64, n),
                                    np.random.default_rng(1).integers(0, n, 64)]))
    p = oparams(orc, phys)
    errs = []
    for i in idx:
        ax, ay, az, _, absf = orc.coulomb(p, *w["pos"], i0=int(i), i1=int(i) + 1, want_absf=True)
        d = math.sqrt((g[0, i] - ax[0]) ** 2 + (g[1, i] - ay[0]) ** 2 + (g[2, i] - az[0]) ** 2)
        errs.append(d / absf[0])
    print("N=1e5 %s: max conditioned error %.3g" % (precision, max(errs)))
    assert max(errs) <= TOL[precision]
    # Newton's third law over all ions (uniform mass: sum a_i = 0)
    tot = np.abs(g).sum(axis=1)
    assert np.all(np.abs(g.sum(axis=1)) <= (1e-12 if precision in ("fp64", "df64") else 1e-6) * tot)


@pytest.mark.parametrize("precision,n", [("fp64", 262151), ("mixed_split", 262151), ("mixed_split", 2000003)])
def test_large_n_sampled(nb, orc, precision, n):
    """Ragged N = 262151 and N = 2000003: the symmetric kernel, which needs no
    partial-sum buffer (it adds into the 3N output in round order), far past
    where per-partner-block partials would have filled device memory;
    sampled ions against the oracle."""
    pos, _ = W.random_cloud(n, seed=8, semi_axes=(300e-6, 300e-6, 1500e-6))
    phys = W.phys()
    g = gpu_forces(nb, phys, pos, precision=precision)
    rng = np.random.default_rng(2)
    idx = np.unique(np.concatenate([np.arange(0, 8), np.arange(n - 8, n), rng.integers(0, n, 32)]))
    p = oparams(orc, phys)
    errs = []
    for i in idx:
        ax, ay, az, _, absf = orc.coulomb(p, *pos, i0=int(i), i1=int(i) + 1, want_absf=True)
        d = math.sqrt((g[0, i] - ax[0]) ** 2 + (g[1, i] - ay[0]) ** 2 + (g[2, i] - az[0]) ** 2)
        errs.append(d / absf[0])
    print("N=%d %s: max conditioned error %.3g" % (n, precision, max(errs)))
    assert max(errs) <= TOL[precision]


def test_argument_errors(nb):
    par = nb.Params.from_phys(W.phys())
    sysm = nb.System(np.zeros((3, 4)) + np.arange(4.0) * 1e-6)
    bad = nb.Params.from_phys(W.phys(), mass=-1.0)
    with pytest.raises(nb.NBError) as ei:
        nb.forces(bad, sysm)
    assert ei.value.status == 1
    with pytest.raises(nb.NBError):
        nb.step(par, sysm, -1)
    empty = nb.System(np.zeros((3, 0)))
    nb.forces(par, empty)
    nb.step(par, empty, 5)
    assert empty.step == 5
    assert np.all(nb.energy(par, empty) == 0)


def test_nonfinite_detected(nb):
    pos = np.zeros((3, 8)) + np.arange(8.0) * 1e-6
    pos[0, 3] = np.nan
    sysm = nb.System(pos)
    nb.forces(nb.Params.from_phys(W.phys()), sysm)
    with pytest.raises(nb.NBError) as ei:
        nb.sync_status()
    assert ei.value.status == 3
    nb.sync_status()  # cleared


@pytest.mark.parametrize("precision", ALL)
def test_symmetric_kernel_small_and_ragged(nb, orc, precision):
    """The half-pair kernel (Newton's third law), forced on at small n with
    every block size, including ragged last blocks, charges and softening."""
    rng = np.random.default_rng(17)
    try:
        for k, (n, block) in enumerate([(2, 256), (257, 256), (1000, 256), (2049, 512), (4100, 1024),
                                        (6000, 512), (33, 32), (700, 32), (95, 64), (1501, 64)]):
            nb.set_tuning("symmetric", precision, 1, 1 << 40, block, R=1)
            pos, _ = W.random_cloud(n, seed=300 + k)
            q = W.E_CHARGE * rng.choice([-1.0, 1.0, 2.0], size=n) if k % 2 else None
            soft2 = (0.1e-6) ** 2 if k == 3 else 0.0
            phys = W.phys(soft2=soft2)
            g = gpu_forces(nb, phys, pos, q=q, precision=precision)
            ax, ay, az, _, absf = orc.coulomb(oparams(orc, phys), *pos, q=q, want_absf=True)
            e = cond_err(g, np.stack([ax, ay, az]), absf)
            assert e <= TOL[precision], (n, block, e)
            g2 = gpu_forces(nb, phys, pos, q=q, precision=precision)
            assert np.array_equal(g, g2)
    finally:
        nb.set_tuning("force", "fp64", 0, 0, 0)


def test_symmetric_matches_one_sided_at_scale(nb):
    """At N = 20000 (symmetric by default) the half-pair and the one-sided
    kernels agree to FP64 rounding (conditioned by the largest force)."""
    pos, _ = W.random_cloud(20000, seed=41, semi_axes=(200e-6, 200e-6, 1000e-6))
    phys = W.phys()
    a = gpu_forces(nb, phys, pos, precision="fp64")
    try:
        nb.set_tuning("symmetric", "fp64", 1, 1 << 40, 256, R=0)
        b = gpu_forces(nb, phys, pos, precision="fp64")
    finally:
        nb.set_tuning("force", "fp64", 0, 0, 0)
    assert not np.array_equal(a, b)  # genuinely different summation orders
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


@pytest.mark.parametrize("precision", ["fp64", "mixed_split"])
@pytest.mark.parametrize("n", [1000, 20000])
def test_step_cuda_graph_capture(nb, precision, n):
    """One nb_step captured in a CUDA graph (after a first call has set up the
    stream's scratch) and replayed three times equals three eager steps,
    bitwise, through the one-sided and the symmetric kernel.  A replay repeats
    the captured step counter, so the trap is static and there is no noise."""
    pos, vel = W.random_cloud(n, seed=77, semi_axes=(200e-6, 200e-6, 1000e-6))
    phys = W.phys(omega=(2 * math.pi * 300e3, 2 * math.pi * 300e3, 2 * math.pi * 100e3))
    par = nb.Params.from_phys(phys, precision=precision)
    eager = nb.System(pos, vel)
    nb.forces(par, eager, total=True)
    for _ in range(3):
        nb.step(par, eager, 1)
    sysm = nb.System(pos, vel)
    nb.forces(par, sysm, total=True)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        nb.step(par, nb.System(pos, vel), 1, stream=s)  # sets up this stream's scratch
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        nb.step(par, sysm, 1)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    nb.sync_status()
    for t in ("x", "vz", "ay"):
        assert torch.equal(getattr(eager, t), getattr(sysm, t)), t


def test_concurrent_host_threads_own_streams(nb):
    """Two host threads, each stepping its own system on its own stream (the
    library's scratch registry is shared and locked), give bitwise the
    results of running them one after the other."""
    import threading
    ws = [W.cloud_harmonic_1024(n=5000), W.cloud_rf_16384(n=20000)]
    par = [nb.Params.from_phys(ws[0]["phys"]), nb.Params.from_phys(ws[1]["phys"], precision="mixed_split")]

    def run(k, stream, out):
        with torch.cuda.stream(stream):
            s = nb.System(ws[k]["pos"], ws[k]["vel"])
            nb.forces(par[k], s, total=True, stream=stream)
            for _ in range(4):
                nb.step(par[k], s, 5, stream=stream)
            stream.synchronize()
            out[k] = s

    serial = {}
    for k in range(2):
        run(k, torch.cuda.Stream(), serial)
    conc = {}
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    th = [threading.Thread(target=run, args=(k, streams[k], conc)) for k in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    torch.cuda.synchronize()
    for k in range(2):
        nb.sync_status(streams[k])
        for t in ("x", "vy", "az"):
            assert torch.equal(getattr(serial[k], t), getattr(conc[k], t)), (k, t)


@pytest.mark.parametrize("n", [300, 3000])
@pytest.mark.parametrize("precision", ["fp64", "df64", "mixed", "mixed_split"])
def test_coincident_ions_contribute_nothing(nb, orc, precision, n):
    """Reading C1: two distinct ions A and B at the same position (no
    softening) exert no force on each other; every other pair is as usual.
    That equals the system with B merged into A (charge q_A + q_B), which the
    oracle can evaluate: each other ion's acceleration is the merged system's,
    and A's and B's are the merged ion's scaled by q_A / (q_A + q_B) and
    q_B / (q_A + q_B).  The VJP likewise, with lam_B = lam_A.  One-sided
    (n = 300) and half-pair (n = 3000) kernels; A and B at ragged places."""
    rng = np.random.default_rng(n + 11)
    pos, _ = W.random_cloud(n, seed=n + 11)
    q = W.E_CHARGE * rng.choice([1.0, 2.0], size=n)
    a, b = 5, n - 7
    pos[:, b] = pos[:, a]
    lam = rng.standard_normal((3, n))
    lam[:, b] = lam[:, a]
    keep = np.array([i for i in range(n) if i != b])
    qm = q[keep].copy()
    ia = int(np.where(keep == a)[0][0])
    qm[ia] = q[a] + q[b]
    phys = W.phys(omega=(6e6, 5e6, 1.2e6))
    p = oparams(orc, phys)
    ax, ay, az, _, absf = orc.coulomb(p, *pos[:, keep], q=qm, want_absf=True)
    merged = np.stack([ax, ay, az])
    ref = np.empty((3, n))
    ref[:, keep] = merged
    ref[:, a] = merged[:, ia] * (q[a] / qm[ia])
    ref[:, b] = merged[:, ia] * (q[b] / qm[ia])
    cond = np.empty(n)
    cond[keep] = absf
    cond[a] = absf[ia] * q[a] / qm[ia]
    cond[b] = absf[ia] * q[b] / qm[ia]
    par = nb.Params.from_phys(phys, precision=precision)
    s = nb.System(pos, q=q)
    nb.forces(par, s)
    nb.sync_status()
    got = s.acc().cpu().numpy()
    assert np.all(np.isfinite(got))
    err = np.max(np.sqrt(np.sum((got - ref) ** 2, axis=0)) / cond)
    gate = 1e-12 if precision in ("fp64", "df64") else 1e-6
    print("%s n=%d: conditioned error %.3g" % (precision, n, err))
    assert err <= gate
    if precision == "fp64":
        gv = nb.forces_vjp(par, nb.System(pos, q=q), lam).cpu().numpy()
        vm = np.stack(orc.forces_vjp(p, 0.0, *pos[:, keep], *lam[:, keep], q=qm))
        vref = np.empty((3, n))
        vref[:, keep] = vm
        vref[:, a] = vm[:, ia] * (q[a] / qm[ia])
        vref[:, b] = vm[:, ia] * (q[b] / qm[ia])
        assert np.all(np.isfinite(gv))
        assert np.max(np.abs(gv - vref)) <= 1e-11 * np.max(np.abs(vref))
