"""Step windows of nb_step (small n, many steps): the middle steps of a call
run as replays of one captured CUDA graph of 8 steps whose epilogues read the
step index from device counters.  They must give bitwise the results of the
plain launches (tuning kind 6 with R = 0 turns the windows off; kind 7 with
R = 0 keeps small systems on the multi-kernel steps), with the RF
trap (time from the step index), friction and Langevin noise (the Philox
counter holds the step index), across call lengths of every residue modulo
the window, repeated calls that reuse the cached window, and changes of
arguments that must recapture it."""
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
    yield nbm
    nbm.set_tuning("force", "fp64", 0, 0, 0)


def _setup(nb, n, precision, noise=True, seed=5):
    w = W.cloud_rf_16384(n=n)
    phys = dict(w["phys"], noise_T=0.5e-3 if noise else 0.0)
    par = nb.Params.from_phys(phys, precision=precision)
    return w, phys, par


def _run(nb, par, w, calls, windows, precision, stream=None):
    nb.set_tuning("force", "fp64", 0, 0, 0)  # clear all overrides
    nb.set_tuning("small_steps", precision, 0, 1 << 40, 1, R=0)  # the multi-kernel steps
    if not windows:
        nb.set_tuning("step_windows", precision, 0, 1 << 40, 1, R=0)
    s = nb.System(w["pos"], w["vel"])
    nb.forces(par, s, total=True, stream=stream)
    lib = nb.lib()
    torch.cuda.synchronize()
    l0 = lib.nb_launch_count()
    for k in calls:
        nb.step(par, s, k, stream=stream)
    torch.cuda.synchronize()
    launches = lib.nb_launch_count() - l0
    nb.sync_status(stream)
    nb.set_tuning("force", "fp64", 0, 0, 0)
    return s, launches


def _equal(a, b):
    for t in ("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az"):
        assert torch.equal(getattr(a, t), getattr(b, t)), t
    assert a.step == b.step


@pytest.mark.parametrize("precision", ["fp64", "df64", "mixed_split"])
@pytest.mark.parametrize("n", [1, 100, 2000])
def test_windows_bitwise_equal_plain_launches(nb, precision, n):
    w, phys, par = _setup(nb, n, precision)
    # lengths 32..41 cover every residue of the prefix modulo the window;
    # the repeated lengths reuse the cached window
    calls = [41, 32, 33, 34, 35, 36, 37, 38, 39, 40, 41, 100]
    plain, lp = _run(nb, par, w, calls, False, precision)
    win, lw = _run(nb, par, w, calls, True, precision)
    _equal(plain, win)
    assert lp == lw, (lp, lw)  # the replays count the kernels they run
    assert win.step == sum(calls)


def test_windows_recapture_on_changed_arguments(nb):
    """A second system (other arrays), other parameters (dt, seed) and a
    precision change each need a new window; interleaving them on one stream
    must still give the plain-launch results."""
    w1, _, par1 = _setup(nb, 500, "fp64")
    w2, phys2, _ = _setup(nb, 700, "fp64")
    par2 = nb.Params.from_phys(dict(phys2, dt=phys2["dt"] * 0.5, seed=99), precision="fp64")
    par2s = nb.Params.from_phys(dict(phys2, dt=phys2["dt"] * 0.5, seed=99), precision="mixed_split")

    def interleaved(windows):
        nb.set_tuning("force", "fp64", 0, 0, 0)
        for p in ("fp64", "mixed_split"):
            nb.set_tuning("small_steps", p, 0, 1 << 40, 1, R=0)
        if not windows:
            for p in ("fp64", "mixed_split"):
                nb.set_tuning("step_windows", p, 0, 1 << 40, 1, R=0)
        a = nb.System(w1["pos"], w1["vel"])
        b = nb.System(w2["pos"], w2["vel"])
        nb.forces(par1, a, total=True)
        nb.forces(par2, b, total=True)
        for k in (40, 50):
            nb.step(par1, a, k)
            nb.step(par2, b, k)
            nb.step(par2s, b, k)
        torch.cuda.synchronize()
        nb.sync_status()
        nb.set_tuning("force", "fp64", 0, 0, 0)
        return a, b

    pa, pb = interleaved(False)
    wa, wb = interleaved(True)
    _equal(pa, wa)
    _equal(pb, wb)


def test_window_cache_reuse_and_eviction(nb):
    """Four systems alternating on one stream keep their four windows (one
    capture each, no recapture); a fifth evicts the least recently used,
    which the next call recaptures; every run equals plain launches."""
    ws = [_setup(nb, 300 + 10 * k, "fp64")[0] for k in range(5)]
    par = nb.Params.from_phys(dict(ws[0]["phys"], noise_T=0.5e-3))

    def run(windows, order):
        nb.set_tuning("force", "fp64", 0, 0, 0)
        nb.set_tuning("small_steps", "fp64", 0, 1 << 40, 1, R=0)
        if not windows:
            nb.set_tuning("step_windows", "fp64", 0, 1 << 40, 1, R=0)
        sys_ = [nb.System(w["pos"], w["vel"]) for w in ws]
        for s in sys_:
            nb.forces(par, s, total=True)
        for k in order:
            nb.step(par, sys_[k], 33)
        torch.cuda.synchronize()
        nb.sync_status()
        nb.set_tuning("force", "fp64", 0, 0, 0)
        return sys_

    order = [0, 1, 2, 3, 0, 1, 2, 3, 4, 0, 4, 3]
    plain = run(False, order)
    win = run(True, order)
    for a, b in zip(plain, win):
        _equal(a, b)


def test_windows_on_a_user_stream_and_default_stream(nb):
    w, _, par = _setup(nb, 300, "fp64")
    plain, _ = _run(nb, par, w, [64], False, "fp64")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        on_stream, _ = _run(nb, par, w, [64], True, "fp64", stream=s)
    torch.cuda.synchronize()
    _equal(plain, on_stream)


def test_no_windows_inside_a_caller_capture(nb):
    """While the caller's stream is being captured, nb_step launches plainly
    (its kernels join the caller's graph); one replay of that graph equals the
    same steps run eagerly, noise and RF trap included (one replay repeats the
    captured step index, which is the eager one)."""
    w, _, par = _setup(nb, 400, "fp64")
    eager, _ = _run(nb, par, w, [40], True, "fp64")
    sysm = nb.System(w["pos"], w["vel"])
    nb.forces(par, sysm, total=True)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        nb.step(par, nb.System(w["pos"], w["vel"]), 1, stream=s)  # sets up this stream's scratch
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        nb.step(par, sysm, 40)
    g.replay()
    torch.cuda.synchronize()
    nb.sync_status()
    assert sysm.step == 40  # advanced on the host when the call was captured
    for t in ("x", "vy", "az"):
        assert torch.equal(getattr(eager, t), getattr(sysm, t)), t


def test_windows_off_above_default_n(nb):
    """n = 8192 runs plain launches by default: the same results with the
    windows forced on (tuning kind 6 R = 1)."""
    w, _, par = _setup(nb, 8192, "mixed_split", noise=False)
    plain, lp = _run(nb, par, w, [34], False, "mixed_split")
    nb.set_tuning("step_windows", "mixed_split", 0, 1 << 40, 1, R=1)
    s = nb.System(w["pos"], w["vel"])
    nb.forces(par, s, total=True)
    nb.step(par, s, 34)
    torch.cuda.synchronize()
    nb.sync_status()
    nb.set_tuning("force", "fp64", 0, 0, 0)
    _equal(plain, s)


@pytest.mark.parametrize("precision", ["fp64", "mixed_split"])
@pytest.mark.parametrize("n", [100, 3001, 9000])
def test_epilogue_lanes_bitwise(nb, precision, n):
    """The eight-lane epilogues (the default) and the one-thread-per-ion
    epilogues (tuning kind 8, R = 0) add the chunk partials in the same order
    and apply the same tail: bitwise the same forces, VJP and steps, through
    one-sided and symmetric plans, with noise and the RF trap."""
    w, phys, par = _setup(nb, n, precision)
    lam = np.random.default_rng(n).standard_normal((3, n))
    out, acc, vjp = [], [], []
    for R in (1, 0):
        nb.set_tuning("force", "fp64", 0, 0, 0)
        nb.set_tuning("small_steps", precision, 0, 1 << 40, 1, R=0)
        nb.set_tuning("epilogue_lanes", "fp64", 0, 1 << 40, 1, R=R)
        s = nb.System(w["pos"], w["vel"])
        nb.forces(par, s, total=True)
        acc.append(s.acc().clone())
        vjp.append(nb.forces_vjp(par, s, lam, total=True))
        nb.step(par, s, 37)
        torch.cuda.synchronize()
        nb.sync_status()
        out.append(s)
    nb.set_tuning("force", "fp64", 0, 0, 0)
    assert torch.equal(acc[0], acc[1])
    assert torch.equal(vjp[0], vjp[1])
    _equal(out[0], out[1])
