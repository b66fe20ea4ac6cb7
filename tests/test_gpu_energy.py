"""Energy conservation of the GPU velocity-Verlet path (no friction, static
harmonic trap, Sec. II): the total energy from nb_energy stays bounded and,
for the FP64-class force paths, its maximum error shrinks about 4x when dt
halves (second order), as the oracle's does on the same start (ratio 4.00)."""
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


def start():
    # sparse enough (nearest pair 1.65 um) that close encounters take >> dt
    rng = np.random.default_rng(31)
    pos = W.ellipsoid_uniform(512, (100e-6, 100e-6, 300e-6), rng)
    vel = W.thermal_velocities(512, 10e-3, W.MASS_40U, rng)
    return pos, vel


def max_energy_error(nb, precision, dt, T=4e-6, checks=20):
    pos, vel = start()
    phys = W.phys(omega=(2 * math.pi * 200e3, 2 * math.pi * 200e3, 2 * math.pi * 100e3), dt=dt)
    par = nb.Params.from_phys(phys, precision=precision)
    s = nb.System(pos, vel)
    nb.forces(par, s, total=True)
    e0 = nb.energy(par, s)[3]
    nsteps = int(round(T / dt))
    emax = 0.0
    for _ in range(checks):
        nb.step(par, s, nsteps // checks)
        e = nb.energy(par, s)[3]
        emax = max(emax, abs(e - e0) / abs(e0))
    nb.sync_status()
    return e0, emax


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_energy_error_second_order(nb, orc, precision):
    e0, e2 = max_energy_error(nb, precision, 2e-9)
    _, e1 = max_energy_error(nb, precision, 1e-9)
    pos, vel = start()
    p = orc.make_params(**W.phys(omega=(2 * math.pi * 200e3, 2 * math.pi * 200e3, 2 * math.pi * 100e3)))
    assert abs(e0 - orc.energy(p, 0, *pos, *vel)[3]) <= 1e-13 * abs(e0)
    print(precision, e2, e1, e2 / e1)
    assert e2 < 1e-6
    assert 3.5 < e2 / e1 < 4.5


def test_energy_bounded_mixed_split(nb):
    """The split path's FP32 pair terms (conditioned error ~2e-8) act as a small
    non-conservative force: the energy error stays at the Verlet level."""
    _, ef = max_energy_error(nb, "fp64", 1e-9)
    _, em = max_energy_error(nb, "mixed_split", 1e-9)
    print(ef, em)
    assert em < 2 * ef + 1e-7
