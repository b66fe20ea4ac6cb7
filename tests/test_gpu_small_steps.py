"""Single-block steps of nb_step for small systems (one launch runs many steps
in one thread block).  The kernel evaluates the one-sided plan's work items
with the same pair terms, adds the chunk partials in chunk order and applies
the same kick and drift, so every ion must get bitwise the multi-kernel
path's result.  Tuning kind 7 turns the path on (R = 1) or off (R = 0).
Covered: all eight pair precisions, uniform and per-ion charges, two
species (per-ion masses), the RF trap, friction and Langevin noise, call
lengths of 1 and many steps, a call longer than one launch's step bound, and
sizes up to the kernel's 512-ion limit."""
import numpy as np
import pytest
import torch

from paper_2106_11143_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MODES = ["fp64", "df64", "mixed", "mixed_split", "sqrtdiv", "rsq", "rsq_nr1", "rsq_nr2", "mixed_split_rsq"]


@pytest.fixture(scope="module")
def nb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_11143_gb300 as nbm
    nbm.lib()
    yield nbm
    nbm.set_tuning("force", "fp64", 0, 0, 0)


def _system(nb, n, charges=False, species=False, seed=0):
    w = W.cloud_rf_16384(n=n, seed=seed + 11)
    rng = np.random.default_rng(seed)
    q = None
    m = None
    if charges:
        q = W.E_CHARGE * rng.choice([1.0, 2.0], size=n)
    if species:
        m = W.MASS_40U * rng.choice([1.0, 9.0 / 40.0], size=n)
    return w, q, m


def _run(nb, phys, precision, w, q, m, calls, small):
    nb.set_tuning("force", "fp64", 0, 0, 0)
    nb.set_tuning("small_steps", precision, 0, 1 << 40, 1, R=1 if small else 0)
    par = nb.Params.from_phys(phys, precision=precision)
    s = nb.System(w["pos"], w["vel"], q=q, m=m)
    nb.forces(par, s, total=True)
    lib = nb.lib()
    torch.cuda.synchronize()
    l0 = lib.nb_launch_count()
    for k in calls:
        nb.step(par, s, k)
    torch.cuda.synchronize()
    launches = lib.nb_launch_count() - l0
    nb.sync_status()
    nb.set_tuning("force", "fp64", 0, 0, 0)
    return s, launches


def _equal(a, b):
    for t in ("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az"):
        assert torch.equal(getattr(a, t), getattr(b, t)), t
    assert a.step == b.step


@pytest.mark.parametrize("precision", MODES)
@pytest.mark.parametrize("n", [1, 2, 7, 16, 33, 64, 100])
def test_small_steps_bitwise_equal_multi_kernel(nb, precision, n):
    w, _, _ = _system(nb, n)
    phys = dict(w["phys"], noise_T=0.5e-3)
    calls = [1, 5, 40]
    small, ls = _run(nb, phys, precision, w, None, None, calls, True)
    multi, _ = _run(nb, phys, precision, w, None, None, calls, False)
    _equal(small, multi)
    assert ls == len(calls)  # one launch per call


@pytest.mark.parametrize("precision", MODES)
def test_small_steps_charges_and_species(nb, precision):
    w, q, m = _system(nb, 48, charges=True, species=True, seed=3)
    phys = dict(w["phys"], noise_T=0.5e-3, soft2=1e-14)
    small, _ = _run(nb, phys, precision, w, q, m, [3, 30], True)
    multi, _ = _run(nb, phys, precision, w, q, m, [3, 30], False)
    _equal(small, multi)


@pytest.mark.parametrize("precision", ["fp64", "df64", "mixed", "mixed_split"])
@pytest.mark.parametrize("n", [128, 257, 400, 512])
def test_small_steps_up_to_the_block_limit(nb, precision, n):
    """Forced on at sizes above the defaults, where the plan has fewer,
    longer j-chunks of several tiles (and the split mode at n = 512 exceeds
    the shared-memory bound, so nb_step keeps the multi-kernel path)."""
    w, q, _ = _system(nb, n, charges=True, seed=n)
    phys = dict(w["phys"], noise_T=0.5e-3)
    small, _ = _run(nb, phys, precision, w, q, None, [20], True)
    multi, _ = _run(nb, phys, precision, w, q, None, [20], False)
    _equal(small, multi)


def test_small_steps_longer_than_one_launch(nb):
    """16400 steps: two launches of the single-block kernel (16384 + 16),
    continuing bit for bit across the launch boundary."""
    w, _, _ = _system(nb, 8, seed=5)
    phys = dict(w["phys"], noise_T=0.5e-3)
    small, ls = _run(nb, phys, "fp64", w, None, None, [16400], True)
    multi, _ = _run(nb, phys, "fp64", w, None, None, [16400], False)
    _equal(small, multi)
    assert ls == 2


def test_small_steps_default_sizes(nb):
    """Without overrides nb_step takes the single-block path at the default
    sizes (one launch per call) and the multi-kernel path above them."""
    w, _, _ = _system(nb, 16)
    par = nb.Params.from_phys(w["phys"])
    lib = nb.lib()
    nb.set_tuning("force", "fp64", 0, 0, 0)
    for n, launches in ((16, 1), (1000, None)):
        ww = W.cloud_rf_16384(n=n)
        s = nb.System(ww["pos"], ww["vel"])
        nb.forces(par, s, total=True)
        torch.cuda.synchronize()
        l0 = lib.nb_launch_count()
        nb.step(par, s, 50)
        torch.cuda.synchronize()
        got = lib.nb_launch_count() - l0
        nb.sync_status()
        if launches is None:
            assert got >= 2 * 50  # pair kernel and epilogue per step
        else:
            assert got == launches


def test_small_steps_nonfinite_detected(nb):
    pos = np.zeros((3, 8)) + np.arange(8.0) * 1e-6
    vel = np.zeros((3, 8))
    vel[1, 5] = np.nan
    par = nb.Params.from_phys(W.phys())
    s = nb.System(pos, vel)
    nb.set_tuning("small_steps", "fp64", 0, 1 << 40, 1, R=1)
    try:
        nb.forces(par, s)  # the Coulomb part only: finite, v is not read
        nb.sync_status()
        nb.step(par, s, 3)  # the kick carries the NaN into v and a
        with pytest.raises(nb.NBError) as ei:
            nb.sync_status()
        assert ei.value.status == 3
        nb.sync_status()  # cleared
    finally:
        nb.set_tuning("force", "fp64", 0, 0, 0)
