"""Trajectory loss and its adjoint gradient (nb_traj_forward/backward and the
torch.autograd binding) against the FP64 oracle's discrete adjoint and
against central finite differences of the GPU forward."""
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


def small_problem(n=48, seed=21):
    rng = np.random.default_rng(seed)
    wr, wz = 2 * math.pi * 1e6, 2 * math.pi * 200e3
    a, c = W.cold_fluid_spheroid(n, wr, wz)
    x0 = W.ellipsoid_uniform(n, (a, a, c), rng)
    v0 = W.thermal_velocities(n, 10e-3, W.MASS_40U, rng)
    target = x0 + 0.2 * a * rng.standard_normal((3, n)) / math.sqrt(n)
    phys = W.phys(omega=(wr, 0.9 * wr, wz), dt=1e-9)
    return x0, v0, target, phys


def gpu_grad(nb, x0, v0, target, phys, nsteps, every, gscale=1.0, precision="fp64"):
    par = nb.Params.from_phys(phys, precision=precision)
    X0 = torch.tensor(x0, device="cuda", requires_grad=True)
    V0 = torch.tensor(v0, device="cuda", requires_grad=True)
    Wt = torch.tensor(phys["omega"], dtype=torch.float64, device="cuda", requires_grad=True)
    T = torch.tensor(target, device="cuda")
    loss = nb.trajectory_loss(X0, V0, Wt, par, nsteps, every, T)
    (gscale * loss).backward()
    torch.cuda.synchronize()
    return loss.item(), X0.grad.cpu().numpy(), V0.grad.cpu().numpy(), Wt.grad.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_loss_and_gradient_match_oracle(nb, orc, precision):
    """The loss and all three gradients against the oracle's discrete adjoint,
    within 10x the oracle's own sensitivity to a one-ulp change of x0, with
    the forward and its recompute in FP64 or in double-float arithmetic."""
    x0, v0, target, phys = small_problem()
    nsteps, every = 150, 37
    loss, gx, gv, gw = gpu_grad(nb, x0, v0, target, phys, nsteps, every, precision=precision)
    p = orc.make_params(**phys)
    lr, gxr, gvr, gwr = orc.trajectory_grad(p, x0, v0, nsteps, target)
    lu, gxu, gvu, gwu = orc.trajectory_grad(p, x0 * (1 + 2.0 ** -52), v0, nsteps, target)
    print("loss gpu %.17g oracle %.17g" % (loss, lr))
    assert abs(loss - lr) <= 1e-12 * abs(lr) + 10 * abs(lu - lr)
    for g, r, u, name in ((gx, gxr, gxu, "x0"), (gv, gvr, gvu, "v0"), (gw, gwr, gwu, "omega")):
        d = np.max(np.abs(g - r))
        self_d = np.max(np.abs(u - r))
        scale = np.max(np.abs(r))
        print("%s: |gpu-oracle| %.3g  self %.3g  scale %.3g" % (name, d, self_d, scale))
        assert d <= 10 * self_d + 1e-11 * scale, name


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_mid_size_gradient_matches_oracle_symmetric_kernels(nb, orc, precision):
    """N = 512 over 300 steps with the symmetric force and VJP kernels forced
    on (by default they start at n = 1500-2000 and 2500): loss and gradients
    against the oracle's discrete adjoint, as in the small case above."""
    x0, v0, target, phys = small_problem(n=512, seed=8)
    nsteps, every = 300, 64
    try:
        nb.set_tuning("symmetric", precision, 0, 1 << 40, 128, R=1)
        nb.set_tuning("symmetric_vjp", "fp64", 0, 1 << 40, 128, R=1)
        assert nb.plan_info("force", precision, 512)["symmetric"] == 1
        assert nb.plan_info("vjp", precision, 512)["symmetric"] == 1
        loss, gx, gv, gw = gpu_grad(nb, x0, v0, target, phys, nsteps, every, precision=precision)
    finally:
        nb.set_tuning("force", "fp64", 0, 0, 0)
    p = orc.make_params(**phys)
    lr, gxr, gvr, gwr = orc.trajectory_grad(p, x0, v0, nsteps, target)
    lu, gxu, gvu, gwu = orc.trajectory_grad(p, x0 * (1 + 2.0 ** -52), v0, nsteps, target)
    print("N=512 loss gpu %.17g oracle %.17g" % (loss, lr))
    assert abs(loss - lr) <= 1e-12 * abs(lr) + 10 * abs(lu - lr)
    for g, r, u, name in ((gx, gxr, gxu, "x0"), (gv, gvr, gvu, "v0"), (gw, gwr, gwu, "omega")):
        d = np.max(np.abs(g - r))
        self_d = np.max(np.abs(u - r))
        scale = np.max(np.abs(r))
        print("%s: |gpu-oracle| %.3g  self %.3g  scale %.3g" % (name, d, self_d, scale))
        assert d <= 10 * self_d + 1e-11 * scale, name


@pytest.mark.parametrize("precision", ["fp64", "df64"])
@pytest.mark.parametrize("n", [100, 3100])
def test_gradient_independent_of_checkpoint_interval(nb, precision, n):
    """Bitwise the same loss and gradients for every checkpoint interval: the
    recompute reproduces the forward exactly, through the step windows and the
    single-block path (n = 100) and the symmetric kernels (n = 3100)."""
    x0, v0, target, phys = small_problem(n=n, seed=3)
    ref = gpu_grad(nb, x0, v0, target, phys, 60, 60, precision=precision)
    for every in (1, 7, 25, 1000):
        r = gpu_grad(nb, x0, v0, target, phys, 60, every, precision=precision)
        assert r[0] == ref[0]
        for a, b in zip(r[1:], ref[1:]):
            assert np.array_equal(a, b), every


def test_chain_rule_scale_and_zero_steps(nb, orc):
    x0, v0, target, phys = small_problem(n=30, seed=4)
    a = gpu_grad(nb, x0, v0, target, phys, 20, 8)
    b = gpu_grad(nb, x0, v0, target, phys, 20, 8, gscale=-2.5)
    for u, v in zip(a[1:], b[1:]):
        assert np.allclose(v, -2.5 * u, rtol=1e-15, atol=0)
    # nsteps = 0: the loss at x0 itself; dL/dx0 = -m A(x0) + 2 (x0 - target)
    loss, gx, gv, gw = gpu_grad(nb, x0, v0, target, phys, 0, 5)
    p = orc.make_params(**phys)
    lr, gxr, gvr, gwr = orc.trajectory_grad(p, x0, v0, 0, target)
    assert abs(loss - lr) <= 1e-12 * abs(lr)
    assert np.max(np.abs(gx - gxr)) <= 1e-12 * np.max(np.abs(gxr))
    assert np.all(gv == 0)
    assert np.max(np.abs(gw - gwr)) <= 1e-12 * np.max(np.abs(gwr))


def test_adjoint_workload_vs_finite_differences(nb):
    """The adjoint workload: N = 4096 in the harmonic pseudopotential
    2pi(1, 1, 0.2) MHz, 2000 steps of 1 ns, checkpoints every 100 steps;
    gradient against Richardson-extrapolated central differences of the GPU
    forward, in the three omega_k and two seeded random directions in x0.
    Step h: 1e-6 relative for omega_z, as the workload states.  Over 2000
    steps this 10 mK cloud is chaotic enough that the x0 and radial-omega
    responses are no longer linear at that h (a perturbation of 1e-6 l grows
    past the interparticle spacing), so those directions use h = 1e-8
    relative (positions: relative to l = (k_C e^2/(m omega_z^2))^(1/3)),
    where the differences converge to the adjoint."""
    w = W.adjoint_cloud()
    x0, v0, target, phys = w["pos"], w["vel"], w["target"], w["phys"]
    nsteps, every = w["steps"], 100
    loss, gx, gv, gw = gpu_grad(nb, x0, v0, target, phys, nsteps, every)
    par = nb.Params.from_phys(phys)
    T = torch.tensor(target, device="cuda")
    V0 = torch.tensor(v0, device="cuda")

    def L(x, om):
        with torch.no_grad():
            return nb.trajectory_loss(torch.tensor(x, device="cuda"), V0,
                                      torch.tensor(om, dtype=torch.float64, device="cuda"),
                                      par, nsteps, every, T).item()

    def fd(f, h):
        d1 = (f(h) - f(-h)) / (2 * h)
        d2 = (f(2 * h) - f(-2 * h)) / (4 * h)
        return (4 * d1 - d2) / 3

    om = list(phys["omega"])
    for k in range(3):
        def fk(h, k=k):
            o = list(om)
            o[k] += h
            return L(x0, o)
        g_fd = fd(fk, (1e-6 if k == 2 else 1e-8) * om[k])
        print("omega_%d: adjoint %.10g fd %.10g" % (k, gw[k], g_fd))
        assert abs(gw[k] - g_fd) <= 1e-5 * abs(g_fd)
    ell = W.chain_length_scale(om[2])
    rng = np.random.default_rng(77)
    for _ in range(2):
        d = rng.standard_normal(x0.shape)
        g_fd = fd(lambda h: L(x0 + h * d, om), 1e-8 * ell)
        g_ad = float(np.sum(gx * d))
        print("x0 direction: adjoint %.10g fd %.10g" % (g_ad, g_fd))
        assert abs(g_ad - g_fd) <= 1e-5 * abs(g_fd)


def test_inputs_are_not_mutated(nb):
    """The library evolves its own copies: the caller's tensors keep their
    values, and repeating a forward gives the same loss."""
    x0, v0, target, phys = small_problem(n=40, seed=9)
    X0 = torch.tensor(x0, device="cuda", requires_grad=True)
    V0 = torch.tensor(v0, device="cuda", requires_grad=True)
    Wt = torch.tensor(phys["omega"], dtype=torch.float64, device="cuda", requires_grad=True)
    T = torch.tensor(target, device="cuda")
    par = nb.Params.from_phys(phys)
    l1 = nb.trajectory_loss(X0, V0, Wt, par, 30, 10, T).item()
    l2 = nb.trajectory_loss(X0, V0, Wt, par, 30, 10, T).item()
    assert l1 == l2
    assert np.array_equal(X0.detach().cpu().numpy(), x0)
    assert np.array_equal(V0.detach().cpu().numpy(), v0)
    pos = torch.tensor(x0, device="cuda")
    s = nb.System(pos, V0.detach())
    nb.forces(par, s, total=True)
    nb.step(par, s, 5)
    nb.sync_status()
    assert np.array_equal(pos.cpu().numpy(), x0)
