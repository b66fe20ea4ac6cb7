"""The ensemble kernel (nb_step_batched) against the FP64 oracle, instance
by instance, plus its determinism, shape independence and CUDA-graph
capture."""
import math

import numpy as np
import pytest
import torch

from paper_2106_11143_gb300 import workloads as W

import floors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_11143_gb300 as nbm
    nbm.lib()
    return nbm


def small_ensemble(sizes, seed=11):
    """Kibble-Zurek-style ensemble with the given instance sizes."""
    w = W.kz_ensemble(n_inst=len(sizes), n_min=1, n_max=2, seed=seed)
    sizes = np.asarray(sizes, dtype=np.int64)
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    rng = np.random.default_rng(seed)
    pos = np.zeros((3, off[-1]))
    for k, m in enumerate(sizes):
        pos[2, off[k]:off[k + 1]] = W.chain_positions(int(m), 2 * math.pi * 100e3)
    vel = W.thermal_velocities(int(off[-1]), 0.5e-3, W.MASS_40U, rng)
    return off, pos, vel, w["phys"]


def oracle_instance(orc, phys, off, pos, vel, k, nsteps, eps=0.0):
    i0, i1 = int(off[k]), int(off[k + 1])
    ph = dict(phys)
    ph["instance"] = k
    p = orc.make_params(**ph)
    x = pos[:, i0:i1] * (1.0 + eps)
    v = vel[:, i0:i1]
    ax, ay, az = orc.accel(p, ph["t0"], *x, *v)
    st = dict(x=x[0], y=x[1], z=x[2], vx=v[0], vy=v[1], vz=v[2], ax=ax, ay=ay, az=az, step=0)
    return orc.run(p, st, nsteps)




def run_gpu(nb, phys, off, pos, vel, nsteps, chunks=1, precision="fp64"):
    par = nb.Params.from_phys(phys, precision=precision)
    sysm = nb.System(pos, vel)
    nb.init_batched(par, sysm, off)
    for _ in range(chunks):
        nb.step_batched(par, sysm, off, nsteps // chunks)
    nb.sync_status()
    return sysm


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_batched_matches_oracle_per_instance(nb, orc, precision):
    sizes = [1, 2, 3, 33, 100, 257, 600, 31]
    off, pos, vel, phys = small_ensemble(sizes)
    nsteps = 40
    sysm = run_gpu(nb, phys, off, pos, vel, nsteps, chunks=2, precision=precision)
    assert sysm.step == nsteps
    gp = sysm.pos().cpu().numpy()
    gv = sysm.vel().cpu().numpy()
    V = math.sqrt(W.K_B * 0.5e-3 / W.MASS_40U)
    for k in range(len(sizes)):
        ref = oracle_instance(orc, phys, off, pos, vel, k, nsteps)
        ulp = oracle_instance(orc, phys, off, pos, vel, k, nsteps, eps=2.0 ** -52)
        i0, i1 = off[k], off[k + 1]
        rp = np.stack([ref["x"], ref["y"], ref["z"]])
        rv = np.stack([ref["vx"], ref["vy"], ref["vz"]])
        up = np.stack([ulp["x"], ulp["y"], ulp["z"]])
        uv = np.stack([ulp["vx"], ulp["vy"], ulp["vz"]])
        ep, ev = floors.per_ion(gp[:, i0:i1] - rp), floors.per_ion(gv[:, i0:i1] - rv)
        sp, sv = np.max(np.abs(up - rp)), np.max(np.abs(uv - rv))
        print("instance %d (n=%d): gpu dp=%.3g dv=%.3g | self dp=%.3g dv=%.3g"
              % (k, sizes[k], np.max(ep), np.max(ev), sp, sv))
        ph = dict(phys)
        ph["instance"] = k
        fp, fv = floors.contract_floor(orc, orc.make_params(**ph), [pos[:, i0:i1], rp], nsteps, phys["dt"],
                                       vels=[vel[:, i0:i1], rv])
        assert np.all(ep <= 10 * sp + fp), k
        assert np.all(ev <= 10 * sv + fv), k


def test_batched_equals_standalone_instances(nb):
    """Instance k of the ensemble is the standalone system with params.instance = k."""
    sizes = [5, 64, 300]
    off, pos, vel, phys = small_ensemble(sizes, seed=3)
    nsteps = 10
    ens = run_gpu(nb, phys, off, pos, vel, nsteps)
    for k in range(len(sizes)):
        i0, i1 = off[k], off[k + 1]
        par = nb.Params.from_phys(phys, instance=k)
        single = nb.System(pos[:, i0:i1], vel[:, i0:i1])
        nb.forces(par, single, total=True)
        nb.step(par, single, nsteps)
        nb.sync_status()
        scale = np.max(np.abs(pos[:, i0:i1])) + 1e-9
        d = np.max(np.abs(ens.pos()[:, i0:i1].cpu().numpy() - single.pos().cpu().numpy()))
        assert d <= 1e-9 * scale, (k, d)


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_batched_bitwise_deterministic_and_shape_independent(nb, precision):
    sizes = [7, 200, 129, 1000]
    off, pos, vel, phys = small_ensemble(sizes, seed=5)
    a = run_gpu(nb, phys, off, pos, vel, 12, precision=precision)
    b = run_gpu(nb, phys, off, pos, vel, 12, chunks=3, precision=precision)
    nb.set_tuning("ensemble", precision, 0, 1 << 40, 128)
    try:
        c = run_gpu(nb, phys, off, pos, vel, 12, precision=precision)
    finally:
        nb.set_tuning("ensemble", "fp64", 0, 0, 0)
    for t in ("x", "vy", "az"):
        assert torch.equal(getattr(a, t), getattr(b, t))
        assert torch.equal(getattr(a, t), getattr(c, t))


def test_batched_cuda_graph_capture(nb):
    """One ensemble launch captured in a CUDA graph and replayed equals the
    eager launch (the replay repeats the captured step window)."""
    sizes = [50, 120, 7]
    off, pos, vel, phys = small_ensemble(sizes, seed=8)
    par = nb.Params.from_phys(phys)
    eager = run_gpu(nb, phys, off, pos, vel, 3)
    sysm = nb.System(pos, vel)
    nb.init_batched(par, sysm, off)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        nb.step_batched(par, nb.System(pos, vel), off, 1, stream=s)  # sets up this stream's scratch
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        nb.step_batched(par, sysm, off, 3)
    g.replay()
    torch.cuda.synchronize()
    for t in ("x", "vz", "ay"):
        assert torch.equal(getattr(eager, t), getattr(sysm, t))


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_full_ensemble_sampled(nb, orc, precision):
    """The 512-instance Kibble-Zurek ensemble (N_k uniform in 32..4096): two
    steps on the GPU in one launch; the largest and smallest instances
    checked against the oracle."""
    w = W.kz_ensemble()
    off, pos, vel, phys = w["offsets"], w["pos"], w["vel"], w["phys"]
    nsteps = 2
    sysm = run_gpu(nb, phys, off, pos, vel, nsteps, precision=precision)
    gp = sysm.pos().cpu().numpy()
    gv = sysm.vel().cpu().numpy()
    assert np.all(np.isfinite(gp)) and np.all(np.isfinite(gv))
    sizes = np.diff(off)
    picks = list(np.argsort(sizes)[:2]) + list(np.argsort(sizes)[-2:])
    for k in picks:
        ref = oracle_instance(orc, phys, off, pos, vel, int(k), nsteps)
        ulp = oracle_instance(orc, phys, off, pos, vel, int(k), nsteps, eps=2.0 ** -52)
        i0, i1 = off[k], off[k + 1]
        rv = np.stack([ref["vx"], ref["vy"], ref["vz"]])
        rp = np.stack([ref["x"], ref["y"], ref["z"]])
        uv = np.stack([ulp["vx"], ulp["vy"], ulp["vz"]])
        up = np.stack([ulp["x"], ulp["y"], ulp["z"]])
        ev, sv = floors.per_ion(gv[:, i0:i1] - rv), np.max(np.abs(uv - rv))
        ep, sp = floors.per_ion(gp[:, i0:i1] - rp), np.max(np.abs(up - rp))
        print("instance %d (n=%d): gpu dp=%.3g dv=%.3g | self dp=%.3g dv=%.3g"
              % (k, sizes[k], np.max(ep), np.max(ev), sp, sv))
        ph = dict(phys)
        ph["instance"] = int(k)
        fp, fv = floors.contract_floor(orc, orc.make_params(**ph), [pos[:, i0:i1], rp], nsteps, phys["dt"],
                                       vels=[vel[:, i0:i1], rv])
        assert np.all(ev <= 10 * sv + fv), k
        assert np.all(ep <= 10 * sp + fp), k


@pytest.mark.parametrize("precision", ["fp64", "df64"])
@pytest.mark.parametrize("charges", [False, True])
def test_batched_symmetric_phase_matches_one_sided(nb, charges, precision):
    """The half-pair force phase (instances of at most 4096 ions: a
    round-robin schedule of 32-ion tile pairs, odd tile counts with a bye, a
    4096-ion instance at the shared-memory limit) against the one-sided phase
    (tuning R = 0), one step and ten steps."""
    sizes = [1, 31, 33, 65, 200, 4096]
    off, pos, vel, phys = small_ensemble(sizes, seed=12)
    pos = pos + 1e-7 * np.random.default_rng(3).standard_normal(pos.shape)  # off the axis
    q = W.E_CHARGE * np.random.default_rng(4).choice([1.0, 2.0], size=pos.shape[1]) if charges else None
    par = nb.Params.from_phys(phys, precision=precision)

    def run(nsteps, one_sided):
        if one_sided:
            nb.set_tuning("ensemble", precision, 0, 1 << 40, 256, R=0)
        try:
            sysm = nb.System(pos, vel, q=q)
            nb.init_batched(par, sysm, off)
            nb.step_batched(par, sysm, off, nsteps)
            nb.sync_status()
        finally:
            nb.set_tuning("ensemble", "fp64", 0, 0, 0)
        return sysm

    a1, b1 = run(1, False), run(1, True)
    acc_a, acc_b = a1.acc().cpu().numpy(), b1.acc().cpu().numpy()
    assert not np.array_equal(acc_a, acc_b)  # genuinely the other phase
    assert np.max(np.abs(acc_a - acc_b)) <= 1e-12 * np.max(np.abs(acc_b))
    a10, b10 = run(10, False), run(10, True)
    scale = np.max(np.abs(pos))
    assert np.max(np.abs(a10.pos().cpu().numpy() - b10.pos().cpu().numpy())) <= 1e-12 * scale


def test_batched_largest_instance(nb):
    """An instance at the size limit (6144 ions: the one-sided force phase with
    196 KB of positions in shared memory) beside small ones, against the
    standalone system."""
    sizes = [6144, 40, 5000]
    off, pos, vel, phys = small_ensemble(sizes, seed=14)
    pos = pos + 1e-7 * np.random.default_rng(5).standard_normal(pos.shape)
    nsteps = 5
    ens = run_gpu(nb, phys, off, pos, vel, nsteps)
    for k in range(len(sizes)):
        i0, i1 = off[k], off[k + 1]
        single = nb.System(pos[:, i0:i1], vel[:, i0:i1])
        par = nb.Params.from_phys(phys, instance=k)
        nb.forces(par, single, total=True)
        nb.step(par, single, nsteps)
        nb.sync_status()
        scale = np.max(np.abs(pos[:, i0:i1]))
        d = np.max(np.abs(ens.pos()[:, i0:i1].cpu().numpy() - single.pos().cpu().numpy()))
        assert d <= 1e-12 * scale, (k, d)


# ---------------------------------------------------------------------------
# nb_step_batched_each: a parameter set of its own per instance


def each_params(phys, n_inst):
    """Per-instance parameters that differ in every field the ensemble kernel
    reads: ramp, friction, temperature, time origin, step, mass, softening,
    trap kind and noise word (one instance without noise, one RF-driven)."""
    out = []
    for k in range(n_inst):
        ph = dict(phys)
        ph["omega_rate"] = tuple(r * (0.5 + 0.25 * k) for r in phys["omega_rate"])
        ph["gamma"] = phys["gamma"] * (1.0 + 0.5 * k)
        ph["noise_T"] = 0.0 if k % 3 == 1 else phys["noise_T"] * (1.0 + k)
        ph["dt"] = phys["dt"] * (1.0 + 0.1 * k)
        ph["t0"] = 1e-7 * k
        ph["mass"] = phys["mass"] * (1.0 + 0.05 * k)
        ph["soft2"] = (1e-6 * k) ** 2
        ph["instance"] = 1000 + 7 * k
        if k == 2:
            ph.update(trap="rf", q_mathieu=0.3, omega_rf=2 * math.pi * 10e6, rf_phase=0.4)
        out.append(ph)
    return out


def oracle_each(orc, ph, x, v, nsteps):
    p = orc.make_params(**ph)
    ax, ay, az = orc.accel(p, ph["t0"], *x, *v)
    st = dict(x=x[0], y=x[1], z=x[2], vx=v[0], vy=v[1], vz=v[2], ax=ax, ay=ay, az=az, step=0)
    return p, orc.run(p, st, nsteps)


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_batched_each_matches_oracle_per_instance(nb, orc, precision):
    sizes = [3, 33, 100, 257, 600, 31]
    off, pos, vel, phys = small_ensemble(sizes, seed=21)
    pos = pos + 1e-7 * np.random.default_rng(6).standard_normal(pos.shape)  # off the axis
    per = each_params(phys, len(sizes))
    pars = [nb.Params.from_phys(ph, precision=precision) for ph in per]
    nsteps = 40
    sysm = nb.System(pos, vel)
    nb.init_batched(pars, sysm, off)
    nb.step_batched_each(pars, sysm, off, nsteps // 2)
    nb.step_batched_each(pars, sysm, off, nsteps - nsteps // 2)
    nb.sync_status()
    assert sysm.step == nsteps
    gp, gv = sysm.pos().cpu().numpy(), sysm.vel().cpu().numpy()
    for k, ph in enumerate(per):
        i0, i1 = off[k], off[k + 1]
        x, v = pos[:, i0:i1], vel[:, i0:i1]
        p, ref = oracle_each(orc, ph, x, v, nsteps)
        _, ulp = oracle_each(orc, ph, x * (1.0 + 2.0 ** -52), v, nsteps)
        rp = np.stack([ref["x"], ref["y"], ref["z"]])
        rv = np.stack([ref["vx"], ref["vy"], ref["vz"]])
        up = np.stack([ulp["x"], ulp["y"], ulp["z"]])
        uv = np.stack([ulp["vx"], ulp["vy"], ulp["vz"]])
        ep, ev = floors.per_ion(gp[:, i0:i1] - rp), floors.per_ion(gv[:, i0:i1] - rv)
        sp, sv = np.max(np.abs(up - rp)), np.max(np.abs(uv - rv))
        print("instance %d (n=%d): gpu dp=%.3g dv=%.3g | self dp=%.3g dv=%.3g"
              % (k, sizes[k], np.max(ep), np.max(ev), sp, sv))
        fp, fv = floors.contract_floor(orc, p, [x, rp], nsteps, ph["dt"], vels=[v, rv])
        assert np.all(ep <= 10 * sp + fp), k
        assert np.all(ev <= 10 * sv + fv), k
        # and not under its neighbour's parameters (with this one's noise word)
        _, other = oracle_each(orc, dict(per[(k + 1) % len(per)], instance=ph["instance"]), x, v, nsteps)
        op = np.stack([other["x"], other["y"], other["z"]])
        assert np.max(np.abs(gp[:, i0:i1] - op)) > 100 * np.max(np.abs(gp[:, i0:i1] - rp)), k


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_batched_each_with_shared_entries_is_bitwise_the_shared_call(nb, precision):
    """A table whose entry k is the shared parameters with instance word
    instance + k gives bitwise the result of nb_step_batched."""
    sizes = [7, 200, 129, 1000, 33]
    off, pos, vel, phys = small_ensemble(sizes, seed=22)
    par = nb.Params.from_phys(phys, precision=precision, instance=40)
    shared = run_gpu(nb, dict(phys, instance=40), off, pos, vel, 12, precision=precision)
    pars = [nb.Params.from_phys(phys, precision=precision, instance=40 + k) for k in range(len(sizes))]
    sysm = nb.System(pos, vel)
    nb.init_batched(par, sysm, off)
    nb.step_batched_each(pars, sysm, off, 12)
    nb.sync_status()
    for t in ("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az"):
        assert torch.equal(getattr(shared, t), getattr(sysm, t)), t


def test_batched_each_table_reuse_and_graph_capture(nb):
    """The stream's table is refilled when the entries change (a table A
    call then a table B call on one stream equals the same calls with the
    scratch released in between), a captured launch replays the eager one,
    and a capture with other entries than the stream's last uncaptured call
    is refused before anything is enqueued."""
    sizes = [50, 120, 7]
    off, pos, vel, phys = small_ensemble(sizes, seed=23)
    ph = each_params(phys, 3)
    per_a = [nb.Params.from_phys(p) for p in ph]
    per_b = [nb.Params.from_phys(dict(ph[2 - k], instance=5 + k)) for k in range(3)]

    def start():
        sysm = nb.System(pos, vel)
        nb.init_batched(per_a, sysm, off)
        return sysm

    both = start()
    nb.step_batched_each(per_a, both, off, 3)
    nb.step_batched_each(per_b, both, off, 4)
    nb.sync_status()
    ref = start()
    nb.step_batched_each(per_a, ref, off, 3)
    nb.sync_status()
    nb.release()  # drops the stream's table: the next call fills a new one
    nb.step_batched_each(per_b, ref, off, 4)
    nb.sync_status()
    for t in ("x", "vz", "ay"):
        assert torch.equal(getattr(both, t), getattr(ref, t)), t

    eager = start()
    nb.step_batched_each(per_a, eager, off, 3)
    nb.sync_status()
    sysm = start()
    scratch = start()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        nb.step_batched_each(per_a, scratch, off, 1, stream=s)  # fills this stream's table
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        nb.step_batched_each(per_a, sysm, off, 3)
        with pytest.raises(nb.NBError):
            nb.step_batched_each(per_b, sysm, off, 3)
    g.replay()
    torch.cuda.synchronize()
    for t in ("x", "vz", "ay"):
        assert torch.equal(getattr(eager, t), getattr(sysm, t)), t


def test_batched_each_at_the_instance_limit(nb):
    """1024 instances (the limit; the device table's size) of 1-4 ions: a
    table of the shared parameters with instance words instance + k gives
    bitwise the shared call, and 1025 instances are refused."""
    rng = np.random.default_rng(24)
    sizes = rng.integers(1, 5, size=1024)
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    w = W.kz_ensemble(n_inst=2, n_min=1, n_max=2, seed=24)
    phys = dict(w["phys"], instance=7)
    pos = np.zeros((3, off[-1]))
    for k, m in enumerate(sizes):
        pos[2, off[k]:off[k + 1]] = W.chain_positions(int(m), 2 * math.pi * 100e3)
    vel = W.thermal_velocities(int(off[-1]), 0.5e-3, W.MASS_40U, rng)
    shared = run_gpu(nb, phys, off, pos, vel, 6)
    pars = [nb.Params.from_phys(phys, instance=7 + k) for k in range(len(sizes))]
    sysm = nb.System(pos, vel)
    nb.init_batched(pars[0], sysm, off)
    nb.step_batched_each(pars, sysm, off, 6)
    nb.sync_status()
    for t in ("x", "vz", "az"):
        assert torch.equal(getattr(shared, t), getattr(sysm, t)), t
    off2 = np.concatenate([off, [off[-1] + 1]])
    big = nb.System(np.zeros((3, int(off2[-1]))), np.zeros((3, int(off2[-1]))))
    with pytest.raises(nb.NBError):
        nb.step_batched_each(pars + pars[:1], big, off2, 1)
