"""nb_energy_noalloc: the energy entry point for callers that cannot call
cudaMalloc (it may synchronise the device, and a framework that owns device
memory through its own pool may not allow it).  It must agree with nb_energy,
on consecutive calls that share its fixed scratch array, and must reject
systems larger than that array with NB_EINVAL and a message."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2106_11143_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nbl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_11143_gb300 import api
    L = api.lib()
    L.nb_energy_noalloc.argtypes = [C.POINTER(api.NbParams), C.POINTER(api.NbSystem),
                                    C.POINTER(C.c_double), C.c_void_p]
    L.nb_energy_noalloc.restype = C.c_int
    return api, L


def _noalloc(api, L, par, sysm):
    out = np.full(4, np.nan)
    s = sysm.to_c()
    rc = L.nb_energy_noalloc(C.byref(par.to_c()), C.byref(s),
                             out.ctypes.data_as(C.POINTER(C.c_double)),
                             C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, out


def test_noalloc_matches_energy_on_consecutive_calls(nbl):
    api, L = nbl
    cases = [W.cloud_harmonic_1024(n=1500), W.cloud_rf_16384(n=4097), W.cloud_harmonic_1024(n=300)]
    for w in cases:
        par = api.Params.from_phys(w["phys"])
        sysm = api.System(w["pos"], w["vel"], step=5)
        ref = api.energy(par, sysm)
        for _ in range(2):  # the second call reuses the scratch the first one left behind
            rc, out = _noalloc(api, L, par, sysm)
            assert rc == 0, L.nb_last_error()
            assert np.all(np.abs(out - ref) <= 1e-12 * np.abs(ref)), (out, ref)


def test_noalloc_with_charges_and_softening(nbl):
    api, L = nbl
    rng = np.random.default_rng(2)
    pos, vel = W.random_cloud(777, seed=2)
    q = W.E_CHARGE * rng.choice([1.0, 2.0], size=777)
    par = api.Params.from_phys(W.phys(soft2=(0.2e-6) ** 2, omega=(1e6, 2e6, 3e5)))
    sysm = api.System(pos, vel, q=q)
    ref = api.energy(par, sysm)
    for _ in range(2):
        rc, out = _noalloc(api, L, par, sysm)
        assert rc == 0
        assert np.all(np.abs(out - ref) <= 1e-12 * np.abs(ref))


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
    assert rc == 0 and np.all(np.abs(out - api.energy(par, small)) <= 1e-12 * np.abs(out))
