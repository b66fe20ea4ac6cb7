"""Two species (Sec. II: interactions 1-1, 2-2 and 1-2 in one all-pairs
sum): per-ion charge and mass through the C ABI against the oracle."""
import math

import numpy as np
import pytest
import torch

from paper_2106_11143_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_11143_gb300 as nbm
    nbm.lib()
    return nbm


def species_cloud(n, seed):
    rng = np.random.default_rng(seed)
    pos, vel = W.random_cloud(n, seed=seed)
    kind = rng.integers(0, 2, size=n)
    q = W.E_CHARGE * np.where(kind == 0, 1.0, 1.0)
    m = W.AMU * np.where(kind == 0, 40.0, 9.0)          # Ca+ and Be+
    q[rng.random(n) < 0.1] = 2 * W.E_CHARGE             # a few doubly charged ions
    return pos, vel, q, m


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("df64", 1e-12), ("mixed_split", 1e-6)])
def test_species_total_acceleration(nb, orc, precision, tol):
    pos, vel, q, m = species_cloud(1537, 4)
    for trap, phys in (("harmonic", W.phys(omega=(6e6, 5e6, 1.2e6), gamma=1e-20)),
                       ("rf", W.phys(trap="rf", q_mathieu=0.3, omega_rf=6.3e7, omega=(0, 0, 1.2e6),
                                     gamma=1e-20))):
        s = nb.System(pos, vel, q=q, m=m, step=7)
        nb.forces(nb.Params.from_phys(phys, precision=precision), s, total=True)
        nb.sync_status()
        g = s.acc().cpu().numpy()
        p = orc.make_params(**phys)
        t = 7 * phys["dt"]
        ref = np.stack(orc.accel(p, t, *pos, *vel, q=q, masses=m))
        _, _, _, _, absf = orc.coulomb(p, *pos, q=q, masses=m, want_absf=True)
        scale = absf + np.sqrt(np.sum(ref ** 2, axis=0))
        err = np.max(np.sqrt(np.sum((g - ref) ** 2, axis=0)) / scale)
        assert err <= tol, (trap, precision, err)


def test_species_energy_and_vjp(nb, orc):
    pos, vel, q, m = species_cloud(900, 5)
    phys = W.phys(omega=(6e6, 5e6, 1.2e6))
    par = nb.Params.from_phys(phys)
    s = nb.System(pos, vel, q=q, m=m)
    e = nb.energy(par, s)
    e_ref = orc.energy(orc.make_params(**phys), 0, *pos, *vel, q=q, masses=m)
    assert np.all(np.abs(e - e_ref) <= 1e-12 * np.abs(e_ref))
    lam = np.random.default_rng(1).standard_normal((3, 900))
    g = nb.forces_vjp(par, s, lam, total=True).cpu().numpy()
    ref = np.stack(orc.forces_vjp(orc.make_params(**phys), 0.0, *pos, *lam, q=q, include_trap=True, masses=m))
    assert np.max(np.abs(g - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_species_trajectory(nb, orc):
    pos, vel, q, m = species_cloud(600, 6)
    phys = W.phys(omega=(2 * math.pi * 1e6, 2 * math.pi * 1e6, 2 * math.pi * 200e3), gamma=3e-21, dt=2e-9)
    par = nb.Params.from_phys(phys)
    s = nb.System(pos, vel, q=q, m=m)
    nb.forces(par, s, total=True)
    nb.step(par, s, 80)
    nb.sync_status()
    p = orc.make_params(**phys)

    def oracle(eps):
        x = pos * (1 + eps)
        ax, ay, az = orc.accel(p, 0.0, *x, *vel, q=q, masses=m)
        st = dict(x=x[0], y=x[1], z=x[2], vx=vel[0], vy=vel[1], vz=vel[2], ax=ax, ay=ay, az=az, step=0)
        return orc.run(p, st, 80, q=q, masses=m)
    ref, ulp = oracle(0.0), oracle(2.0 ** -52)
    gv = s.vel().cpu().numpy()
    rv = np.stack([ref["vx"], ref["vy"], ref["vz"]])
    uv = np.stack([ulp["vx"], ulp["vy"], ulp["vz"]])
    dv, sv = np.max(np.abs(gv - rv)), np.max(np.abs(uv - rv))
    print("species trajectory: gpu dv %.3g, self %.3g" % (dv, sv))
    assert dv <= 10 * sv + 1e-14 * np.max(np.abs(rv))


def test_species_rejected_where_unsupported(nb):
    pos, vel, q, m = species_cloud(40, 7)
    s = nb.System(pos, vel, q=q, m=m)
    par = nb.Params.from_phys(W.phys(omega=(6e6, 5e6, 1.2e6)))
    with pytest.raises(nb.NBError) as ei:
        nb.step_batched(par, s, np.array([0, 40]), 1)
    assert ei.value.status == 6
