"""The i-range entry points on one GPU (nb_forces_range, nb_step_range_drift,
nb_step_range_kick) and the sharding driver with one rank.  Ranks are
emulated by calling the range entry points one range after another on a
single system: every range's drift, then (the exchange is a no-op when all
ranges share one array) every range's kick.  The ranges put together must
give the bits of the one-sided kernel's full-system calls, and the oracle's
values within the force gate."""
import copy
import math

import numpy as np
import pytest
import torch

from paper_2106_11143_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "df64": 1e-12, "mixed": 1e-6, "mixed_split": 1e-6, "mixed_split_rsq": 1e-6}


@pytest.fixture(scope="module")
def nb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_11143_gb300 as nbm
    nbm.lib()
    return nbm


@pytest.fixture
def one_sided(nb):
    """The symmetric kernel off (tuning kind 4, R = 0) for the duration."""
    for prec in ("fp64", "df64", "mixed", "mixed_split", "mixed_split_rsq"):
        nb.set_tuning("symmetric", prec, 0, 1 << 40, 128, R=0)
    yield
    nb.set_tuning("force", "fp64", 0, 0, 0)


@pytest.mark.parametrize("precision", ["fp64", "df64", "mixed", "mixed_split", "mixed_split_rsq"])
def test_forces_range_pieces_equal_full_call(nb, orc, one_sided, precision):
    n = 3001
    rng = np.random.default_rng(5)
    pos, vel = W.random_cloud(n, seed=5)
    q = W.E_CHARGE * rng.choice([1.0, 2.0], size=n)
    phys = W.phys(gamma=1e-20)
    par = nb.Params.from_phys(phys, precision=precision)
    full = nb.System(pos, vel, q=q, step=3)
    nb.forces(par, full, total=True)
    parts = nb.System(pos, vel, q=q, step=3)
    for a, b in ((0, 1), (1, 1000), (1000, 1000), (1000, 2999), (2999, n)):
        nb.forces_range(par, parts, a, b, total=True)
    nb.sync_status()
    assert torch.equal(parts.acc(), full.acc())
    # Coulomb part against the oracle
    coul = nb.System(pos, q=q)
    for a, b in ((0, 1500), (1500, n)):
        nb.forces_range(par, coul, a, b)
    nb.sync_status()
    ax, ay, az, _, absf = orc.coulomb(orc.make_params(**phys), *pos, q=q, want_absf=True)
    err = np.max(np.sqrt(np.sum((coul.acc().cpu().numpy() - np.stack([ax, ay, az])) ** 2, axis=0)) / absf)
    assert err <= TOL[precision], err


def test_forces_range_writes_only_its_ions(nb):
    n = 700
    pos, _ = W.random_cloud(n, seed=9)
    par = nb.Params.from_phys(W.phys())
    s = nb.System(pos)
    for t in (s.ax, s.ay, s.az):
        t.fill_(7.0)
    nb.forces_range(par, s, 100, 250)
    nb.sync_status()
    a = s.acc().cpu().numpy()
    assert np.all(a[:, :100] == 7.0) and np.all(a[:, 250:] == 7.0)
    assert np.all(a[:, 100:250] != 7.0)
    with pytest.raises(nb.NBError):
        nb.forces_range(par, s, 300, 200)
    with pytest.raises(nb.NBError):
        nb.forces_range(par, s, 0, n + 1)


def _emulated_ranks_step(nb, par, systems, ranges, nsteps):
    """Every rank's drift, then every rank's kick, per step; the ranks' System
    objects share the arrays (so the exchange is implicit) and each keeps its
    own step counter, as on separate GPUs."""
    for _ in range(nsteps):
        for s, (a, b) in zip(systems, ranges):
            nb.step_range_drift(par, s, a, b)
        for s, (a, b) in zip(systems, ranges):
            nb.step_range_kick(par, s, a, b)


@pytest.mark.parametrize("world,precision,trap", [(2, "fp64", "harmonic"), (3, "mixed_split", "rf"),
                                                  (4, "df64", "harmonic")])
def test_emulated_sharded_steps_bitwise(nb, one_sided, world, precision, trap):
    """Sharded steps (RF trap, friction and Langevin noise keyed by the global
    ion index) reproduce nb_step with the one-sided kernel bit for bit."""
    from paper_2106_11143_gb300.shard import partition
    n, nsteps = 2501, 12
    rng = np.random.default_rng(world)
    pos, vel = W.random_cloud(n, seed=world)
    q = W.E_CHARGE * rng.choice([1.0, 2.0], size=n)
    if trap == "rf":
        phys = W.phys(trap="rf", q_mathieu=0.3, omega_rf=2 * math.pi * 10e6,
                      omega=(0.0, 0.0, 2 * math.pi * 200e3), gamma=1e-20, noise_T=0.5e-3, seed=11, dt=2e-9)
    else:
        phys = W.phys(omega=(2 * math.pi * 1e6, 2 * math.pi * 1e6, 2 * math.pi * 200e3), gamma=1e-20,
                      noise_T=0.5e-3, seed=11)
    par = nb.Params.from_phys(phys, precision=precision)
    ref = nb.System(pos, vel, q=q)
    nb.forces(par, ref, total=True)
    nb.step(par, ref, nsteps)
    base = nb.System(pos, vel, q=q)
    ranges = partition(n, world)
    for a, b in ranges:
        nb.forces_range(par, base, a, b, total=True)
    systems = [copy.copy(base) for _ in range(world)]
    _emulated_ranks_step(nb, par, systems, ranges, nsteps)
    nb.sync_status()
    assert all(s.step == nsteps for s in systems)
    for t in ("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az"):
        assert torch.equal(getattr(base, t), getattr(ref, t)), t


def test_sharded_driver_single_rank(nb, one_sided):
    """ShardedSystem with one rank (torch.distributed not initialised) runs
    the range calls over the whole system: nb_step's bits."""
    from paper_2106_11143_gb300.shard import ShardedSystem
    w = W.cloud_harmonic_1024(n=1500)
    par = nb.Params.from_phys(w["phys"])
    ref = nb.System(w["pos"], w["vel"])
    nb.forces(par, ref, total=True)
    nb.step(par, ref, 20)
    s = nb.System(w["pos"], w["vel"])
    sh = ShardedSystem(par, s)
    assert (sh.world, sh.i0, sh.i1) == (1, 0, 1500)
    sh.init_forces()
    sh.step(20)
    sh.gather_state()
    nb.sync_status()
    assert s.step == 20
    for t in ("x", "vx", "ax"):
        assert torch.equal(getattr(s, t), getattr(ref, t)), t
