"""GPU results against closed forms and symmetries (no oracle values):

  - a ring of N ions: the force on every ion is radial with magnitude
    k_C e^2 / (4 R^2 m) sum_k 1/sin(pi k / N), and has no tangential part;
  - two ions in a harmonic trap at the equilibrium spacing
    d^3 = e^2 / (2 pi eps0 m w_z^2) feel no total force (Eq. 1);
  - a permutation of the ions permutes the forces.

Every precision, at sizes that take the one-sided and the symmetric kernels.
The tolerance is the precision's gate on the conditioned error (relative to
S = sum_j |a_ij|, C9), plus, for the ring, the rounding of the cos/sin input
positions, which reaches the net force as ~N^2 eps of its magnitude."""
import math

import numpy as np
import pytest
import torch

from paper_2106_11143_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GATE = {"fp64": 1e-12, "df64": 1e-12, "mixed": 1e-6, "mixed_split": 1e-6, "mixed_split_rsq": 1e-6}
ALL = list(GATE)


@pytest.fixture(scope="module")
def nb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_11143_gb300 as nbm
    nbm.lib()
    return nbm


def coulomb_acc(nb, pos, precision, **kw):
    s = nb.System(pos)
    nb.forces(nb.Params.from_phys(W.phys(**kw), precision=precision), s)
    nb.sync_status()
    return s.acc().cpu().numpy()


@pytest.mark.parametrize("precision", ALL)
def test_ring_radial_closed_form(nb, precision):
    R = 37e-6
    for n in (2, 64, 1000, 20000):
        pos = W.ring(n, R)
        a = coulomb_acc(nb, pos, precision)
        k = np.arange(1, n)
        unit = W.K_COULOMB * W.E_CHARGE ** 2 / (4 * R * R * W.MASS_40U)
        mag = unit * np.sum(1 / np.sin(np.pi * k / n))
        S = unit * np.sum(1 / np.sin(np.pi * k / n) ** 2)  # sum_j |a_ij|
        th = 2 * np.pi * np.arange(n) / n
        radial = a[0] * np.cos(th) + a[1] * np.sin(th)
        tang = -a[0] * np.sin(th) + a[1] * np.cos(th)
        tol = GATE[precision] * S + 2.2e-16 * n * n * mag
        print("%s n=%d: max radial err %.3g, max tangential %.3g, tol %.3g" %
              (precision, n, np.max(np.abs(radial - mag)), np.max(np.abs(tang)), tol))
        assert np.all(np.abs(radial - mag) <= tol)
        assert np.all(np.abs(tang) <= tol)
        assert np.all(np.abs(a[2]) <= GATE[precision] * S)


@pytest.mark.parametrize("precision", ALL)
def test_two_ion_equilibrium(nb, precision):
    wz = 2 * math.pi * 200e3
    d = (W.E_CHARGE ** 2 / (2 * math.pi * W.EPS0 * W.MASS_40U * wz ** 2)) ** (1.0 / 3.0)
    assert abs(d - 16.385e-6) < 1e-9  # the worked value for 40 u at 200 kHz
    pos = np.array([[0.0, 0.0], [0.0, 0.0], [-d / 2, d / 2]])
    s = nb.System(pos, np.zeros((3, 2)))
    par = nb.Params.from_phys(W.phys(omega=(2 * math.pi * 1e6, 2 * math.pi * 1e6, wz)), precision=precision)
    nb.forces(par, s, total=True)
    nb.sync_status()
    a = s.acc().cpu().numpy()
    scale = W.K_COULOMB * W.E_CHARGE ** 2 / (W.MASS_40U * d * d)
    assert np.all(np.abs(a) <= (GATE[precision] + 1e-14) * scale), a


@pytest.mark.parametrize("precision", ALL)
def test_permutation_permutes_forces(nb, orc, precision):
    rng = np.random.default_rng(9)
    for n in (3000, 20000):
        pos, _ = W.random_cloud(n, seed=500 + n)
        perm = rng.permutation(n)
        a = coulomb_acc(nb, pos, precision)
        ap = coulomb_acc(nb, pos[:, perm], precision)
        inv = np.empty(n, dtype=np.int64)
        inv[perm] = np.arange(n)
        back = ap[:, inv]
        # the scale S_i = sum_j |a_ij| of a few ions (the oracle's sum of
        # magnitudes); the two results differ by summation order only
        idx = rng.integers(0, n, 16)
        p = orc.make_params(**W.phys())
        S = np.array([orc.coulomb(p, *pos, i0=int(i), i1=int(i) + 1, want_absf=True)[4][0] for i in idx])
        d = np.sqrt(np.sum((a[:, idx] - back[:, idx]) ** 2, axis=0))
        assert np.all(d <= 2 * GATE[precision] * S), (n, np.max(d / S))


@pytest.mark.parametrize("precision", ALL)
def test_translation_invariance(nb, orc, precision):
    """Shifting every position by the same vector (1 cm and 10 cm off the
    origin) leaves the forces unchanged, through both the one-sided and the
    symmetric kernel.  Positions sit on a 2^-40 m grid and the shifts are
    grid multiples, so shifted positions and all their differences are exact
    in FP64: the modes that form the displacement in FP64 (fp64, df64, mixed)
    see bitwise the same displacements and must give bitwise the same forces;
    the split modes, which work from FP32 (hi, lo) positions, stay within
    their gate."""
    g = 2.0 ** -40
    for n in (3000, 20000):
        pos, _ = W.random_cloud(n, seed=600 + n)
        pos = np.round(pos / g) * g
        a = coulomb_acc(nb, pos, precision)
        split = precision.startswith("mixed_split")
        if split:
            idx = np.random.default_rng(n).integers(0, n, 16)
            p = orc.make_params(**W.phys())
            S = np.array([orc.coulomb(p, *pos, i0=int(i), i1=int(i) + 1, want_absf=True)[4][0] for i in idx])
        for shift in (1e-2, 1e-1):
            sh = np.round(np.array([[shift], [-0.5 * shift], [0.3 * shift]]) / g) * g
            moved = pos + sh
            assert np.array_equal(moved - sh, pos)  # exact
            b = coulomb_acc(nb, moved, precision)
            if split:
                d = np.sqrt(np.sum((a[:, idx] - b[:, idx]) ** 2, axis=0))
                assert np.all(d <= GATE[precision] * S), (n, shift, np.max(d / S))
            else:
                assert np.array_equal(a, b), (n, shift)
