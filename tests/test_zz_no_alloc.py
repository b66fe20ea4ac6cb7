"""nb_energy_noalloc: the energy entry point for callers that cannot call
cudaMalloc (it may synchronise the device, and a framework that owns device
memory through its own pool may not allow it).  It runs nb_energy's kernels
with nb_energy's plan, so it must agree with nb_energy bit for bit, on
consecutive calls that share its fixed scratch array, whatever an earlier
call left there; it must reject systems larger than that array, and bad
arguments, with NB_EINVAL and a message, before any launch."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2106_11143_gb300 import workloads as W


def _bind(api):
    L = api.lib()
    L.nb_energy_noalloc.argtypes = [C.POINTER(api.NbParams), C.POINTER(api.NbSystem),
                                    C.POINTER(C.c_double), C.c_void_p]
    L.nb_energy_noalloc.restype = C.c_int
    return L


@pytest.fixture(scope="module")
def nbl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_11143_gb300 import api
    return api, _bind(api)


def _noalloc(api, L, par, sysm):
    out = np.full(4, np.nan)
    s = sysm.to_c()
    rc = L.nb_energy_noalloc(C.byref(par.to_c()), C.byref(s),
                             out.ctypes.data_as(C.POINTER(C.c_double)),
                             C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, out


@pytest.mark.gpu
def test_noalloc_matches_energy_on_consecutive_calls(nbl):
    """Sizes in the order 1500, 4097, 300: the potential plan's partial count
    changes from call to call, so a call that read a slot the previous call
    left behind would not reproduce nb_energy's bits."""
    api, L = nbl
    cases = [W.cloud_harmonic_1024(n=1500), W.cloud_rf_16384(n=4097), W.cloud_harmonic_1024(n=300)]
    for w in cases:
        par = api.Params.from_phys(w["phys"])
        sysm = api.System(w["pos"], w["vel"], step=5)
        ref = api.energy(par, sysm)
        for _ in range(2):  # the second call reuses the scratch the first one left behind
            rc, out = _noalloc(api, L, par, sysm)
            assert rc == 0, L.nb_last_error()
            assert np.array_equal(out, ref), (out, ref)


@pytest.mark.gpu
def test_noalloc_with_charges_softening_and_zero_velocity(nbl):
    api, L = nbl
    rng = np.random.default_rng(2)
    pos, vel = W.random_cloud(777, seed=2)
    q = W.E_CHARGE * rng.choice([1.0, 2.0], size=777)
    par = api.Params.from_phys(W.phys(soft2=(0.2e-6) ** 2, omega=(1e6, 2e6, 3e5)))
    for v in (vel, np.zeros_like(vel)):
        sysm = api.System(pos, v, q=q)
        ref = api.energy(par, sysm)
        for _ in range(2):
            rc, out = _noalloc(api, L, par, sysm)
            assert rc == 0
            assert np.array_equal(out, ref)
    assert out[0] == 0.0 and out[2] > 0.0  # the zero-velocity case: no kinetic energy


@pytest.mark.gpu
def test_noalloc_near_capacity(nbl):
    """n = 900 000, close to the fixed array's limit (the potential plan
    then has one partial per ion): one call, bitwise equal to nb_energy."""
    api, L = nbl
    n = 900_000
    rng = np.random.default_rng(9)
    pos = W.ellipsoid_uniform(n, (400e-6, 400e-6, 2000e-6), rng)
    vel = W.thermal_velocities(n, 10e-3, W.MASS_40U, rng)
    par = api.Params.from_phys(W.phys())
    sysm = api.System(pos, vel)
    rc, out = _noalloc(api, L, par, sysm)
    assert rc == 0, L.nb_last_error()
    assert np.array_equal(out, api.energy(par, sysm))


@pytest.mark.gpu
def test_noalloc_rejects_oversize(nbl):
    api, L = nbl
    n = 1_100_000
    sysm = api.System(torch.zeros(3, n, dtype=torch.float64, device="cuda"))
    par = api.Params.from_phys(W.phys())
    rc, out = _noalloc(api, L, par, sysm)
    assert rc == 1
    assert b"scratch" in L.nb_last_error()
    # a valid call afterwards still works
    w = W.cloud_harmonic_1024(n=200)
    par = api.Params.from_phys(w["phys"])
    small = api.System(w["pos"], w["vel"])
    rc, out = _noalloc(api, L, par, small)
    assert rc == 0 and np.array_equal(out, api.energy(par, small))


def test_noalloc_rejects_bad_arguments_on_host():
    """Without a GPU: the host-side checks of nb_energy run first, so a
    misaligned array or a non-finite parameter returns NB_EINVAL with a
    message and nothing is launched (the fake device addresses are never
    dereferenced)."""
    from paper_2106_11143_gb300 import api
    L = _bind(api)
    base = 1 << 20
    s = api.NbSystem()
    s.n = 10
    for k, name in enumerate(("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az")):
        setattr(s, name, C.cast(C.c_void_p(base + 4096 * k), C.POINTER(C.c_double)))
    p = api.Params.from_phys(W.phys()).to_c()
    out = (C.c_double * 4)()
    s.x = C.cast(C.c_void_p(base + 4), C.POINTER(C.c_double))  # 4-byte offset
    assert L.nb_energy_noalloc(C.byref(p), C.byref(s), out, None) == 1
    assert b"aligned" in L.nb_last_error()
    s.x = C.cast(C.c_void_p(base), C.POINTER(C.c_double))
    p.mass = float("nan")
    assert L.nb_energy_noalloc(C.byref(p), C.byref(s), out, None) == 1
    assert b"mass" in L.nb_last_error()
    p = api.Params.from_phys(W.phys()).to_c()
    p.precision = 99
    assert L.nb_energy_noalloc(C.byref(p), C.byref(s), out, None) == 1
    assert b"precision" in L.nb_last_error()
    assert L.nb_energy_noalloc(C.byref(p), C.byref(s), None, None) == 1
