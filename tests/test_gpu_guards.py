"""Guard words around every caller-owned device array (the stand-in for a
sanitizer, which this pool does not offer): each array is the middle of a
larger tensor whose G leading and G trailing words hold a NaN-boxed pattern.
After each entry point, at ragged sizes that take every kernel path, the
guards must be bit for bit unchanged: no kernel writes (or, through a
result, reads into its output) outside [0, n)."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2106_11143_gb300 import workloads as W

pytestmark = pytest.mark.gpu

G = 64
PATTERN = 0x7FF8DEADBEEF0001  # as a double: a quiet NaN with a payload


@pytest.fixture(scope="module")
def nb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_11143_gb300 as nbm
    nbm.lib()
    yield nbm
    nbm.set_tuning("force", "fp64", 0, 0, 0)


def api():
    from paper_2106_11143_gb300 import api as a
    return a


class Guarded:
    """Device arrays of n doubles, each inside a tensor with G guard words on
    both sides."""

    def __init__(self):
        self.bufs = []

    def array(self, values):
        values = torch.as_tensor(np.asarray(values, dtype=np.float64)).reshape(-1)
        n = values.numel()
        big = torch.empty(n + 2 * G, dtype=torch.float64, device="cuda")
        big.view(torch.int64).fill_(PATTERN)
        big[G:G + n] = values.to("cuda")
        self.bufs.append(big)
        return big[G:G + n]

    def check(self, what):
        torch.cuda.synchronize()
        for k, big in enumerate(self.bufs):
            bits = big.view(torch.int64)
            n = big.numel() - 2 * G
            head = torch.all(bits[:G] == PATTERN).item()
            tail = torch.all(bits[G + n:] == PATTERN).item()
            assert head and tail, "%s: guard of array %d overwritten" % (what, k)


def guarded_system(nb, gd, pos, vel, q=None):
    s = nb.System(pos, vel, q=q)
    for k, arr in zip(("x", "y", "z"), pos):
        setattr(s, k, gd.array(arr))
    for k, arr in zip(("vx", "vy", "vz"), vel):
        setattr(s, k, gd.array(arr))
    for k in ("ax", "ay", "az"):
        setattr(s, k, gd.array(np.zeros(s.n)))
    if q is not None:
        s.q = gd.array(q)
    return s


SIZES = [1, 31, 33, 257, 3001, 5003]


@pytest.mark.parametrize("precision", ["fp64", "df64", "mixed", "mixed_split"])
@pytest.mark.parametrize("n", SIZES)
def test_guards_forces_step_energy(nb, precision, n):
    """nb_forces (with the potential), nb_step (single-block, windows,
    plain and symmetric paths by size), nb_energy and nb_energy_noalloc."""
    gd = Guarded()
    w = W.cloud_rf_16384(n=n, seed=n)
    q = W.E_CHARGE * np.random.default_rng(n).choice([1.0, 2.0], size=n) if n % 2 else None
    s = guarded_system(nb, gd, w["pos"], w["vel"], q=q)
    par = nb.Params.from_phys(dict(w["phys"], noise_T=0.5e-3), precision=precision)
    phi = gd.array(np.zeros(n))
    L = nb.lib()
    sc = s.to_c()
    api()._check(L.nb_forces(C.byref(par.to_c()), C.byref(sc), api()._ptr(phi), 1, api()._stream(None)),
              "nb_forces")
    nb.sync_status()
    gd.check("nb_forces")
    for k in (1, 40):
        nb.step(par, s, k)
        nb.sync_status()
        gd.check("nb_step(%d)" % k)
    nb.energy(par, s)
    gd.check("nb_energy")
    out = np.empty(4)
    sc = s.to_c()
    api()._check(L.nb_energy_noalloc(C.byref(par.to_c()), C.byref(sc), out.ctypes.data_as(api()._dp),
                                  api()._stream(None)), "nb_energy_noalloc")
    gd.check("nb_energy_noalloc")


@pytest.mark.parametrize("precision", ["fp64", "df64"])
@pytest.mark.parametrize("n", SIZES)
def test_guards_vjp(nb, precision, n):
    gd = Guarded()
    w = W.cloud_rf_16384(n=n, seed=n + 1)
    s = guarded_system(nb, gd, w["pos"], w["vel"])
    lam = np.random.default_rng(n).standard_normal((3, n))
    lx, ly, lz = (gd.array(lam[k]) for k in range(3))
    gx, gy, gz = (gd.array(np.zeros(n)) for _ in range(3))
    par = nb.Params.from_phys(w["phys"], precision=precision)
    sc = s.to_c()
    p = api()._ptr
    api()._check(nb.lib().nb_forces_vjp(C.byref(par.to_c()), C.byref(sc), p(lx), p(ly), p(lz), p(gx), p(gy),
                                     p(gz), 1, api()._stream(None)), "nb_forces_vjp")
    nb.sync_status()
    gd.check("nb_forces_vjp")
    assert torch.all(torch.isfinite(gx)).item()


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_guards_ensemble(nb, precision):
    """nb_step_batched over uneven instances, with the half-pair and the
    one-sided force phase."""
    gd = Guarded()
    sizes = [1, 31, 33, 257, 700, 4200]
    off = np.concatenate([[0], np.cumsum(sizes)])
    pos = np.concatenate([W.chain_positions(m, 2e6 * np.pi * 0.1)[None, :] * np.array([[0.0], [0.0], [1.0]])
                          + np.random.default_rng(m).normal(0, 1e-7, (3, m)) for m in sizes], axis=1)
    vel = np.zeros_like(pos)
    s = guarded_system(nb, gd, pos, vel)
    par = nb.Params.from_phys(W.phys(omega=(2e6 * np.pi, 2e6 * np.pi, 2e5 * np.pi), gamma=1e-20,
                                     noise_T=0.5e-3), precision=precision)
    nb.init_batched(par, s, off)
    nb.step_batched(par, s, off, 5)
    nb.sync_status()
    gd.check("nb_step_batched")
