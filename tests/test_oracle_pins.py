"""Pins for the FP64 CPU oracle: each test checks it against something other
than itself -- a value printed in the paper, a closed form, an invariant, an
independent high-precision evaluation, or a finite difference -- so that a
dropped term, a wrong sign or index, or a transposed operand fails one of
them.  CPU only."""
import math
import os

import numpy as np

from paper_2106_11143_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def P(orc, **kw):
    return orc.make_params(**W.phys(**kw))


def rel(a, b):
    return abs(a - b) / abs(b)


# --------------------------------------------------------------------------
# Table 1 (Sec. IV): constants and units.
def _table1_rows():
    rows = []
    with open(os.path.join(GOLD, "table1.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                b, T, dx, dv = line.split()
                rows.append((int(b), float(T), float(dx), float(dv)))
    return rows


def test_table1_error_model_constants():
    """Sec. IV two-ion model: dx/d = (3/2) dt^2 (Q^2 k_C/m) d_min^-3 eps with
    d_min = 4 Q^2 k_C/(kB T), and dv/v = (3/16) dt/(Q^2 k_C) sqrt(kB^3 T^3/m)
    eps, evaluated with CODATA constants for 40 u, reproduce the twelve
    printed entries within their one-significant-figure rounding band."""
    Q2k = W.E_CHARGE ** 2 * W.K_COULOMB
    m, dt = W.MASS_40U, 5e-9
    for b, T, dx_p, dv_p in _table1_rows():
        eps = 2.0 ** -b
        dmin = 4 * Q2k / (W.K_B * T)
        dx = 1.5 * dt * dt * Q2k / m * dmin ** -3 * eps
        dv = 3.0 / 16.0 * dt / Q2k * math.sqrt((W.K_B * T) ** 3 / m) * eps
        assert 0.75 < dx / dx_p < 1.34, (b, T, dx, dx_p)
        assert 0.75 < dv / dv_p < 1.34, (b, T, dv, dv_p)


# --------------------------------------------------------------------------
# Closed-form equilibria: Coulomb scaling + trap (Eq. 1).
def test_two_ion_equilibrium_static(orc):
    """Two ions on the axis of a harmonic trap balance at spacing d with
    d^3 = q^2 / (2 pi eps0 m omega_z^2)."""
    wz = 2 * math.pi * 200e3
    p = P(orc, omega=(2 * math.pi * 1e6, 2 * math.pi * 1e6, wz))
    d = (W.E_CHARGE ** 2 / (2 * math.pi * W.EPS0 * W.MASS_40U * wz ** 2)) ** (1 / 3)
    assert abs(d - 16.385e-6) < 0.01e-6
    z = np.array([-d / 2, d / 2])
    ax, ay, az = orc.accel(p, 0.0, np.zeros(2), np.zeros(2), z)
    aC = W.K_COULOMB * W.E_CHARGE ** 2 / (W.MASS_40U * d * d)
    assert np.all(np.abs(az) <= 1e-12 * aC)
    assert np.all(ax == 0) and np.all(ay == 0)
    # the Coulomb part alone is repulsive with magnitude aC
    cx, cy, cz, _, _ = orc.coulomb(p, np.zeros(2), np.zeros(2), z)
    assert rel(cz[1], aC) < 1e-14 and rel(-cz[0], aC) < 1e-14


def test_two_ion_relaxation_with_friction(orc):
    """Damped Verlet relaxes two displaced ions to the closed-form spacing."""
    wz = 2 * math.pi * 200e3
    m = W.MASS_40U
    p = P(orc, omega=(2 * math.pi * 1e6, 2 * math.pi * 1e6, wz), gamma=2 * m * wz, dt=2e-9)
    d = (W.E_CHARGE ** 2 / (2 * math.pi * W.EPS0 * m * wz ** 2)) ** (1 / 3)
    z = np.array([-0.7 * d, 0.55 * d])
    zero = np.zeros(2)
    ax, ay, az = orc.accel(p, 0.0, zero, zero, z, zero, zero, zero)
    st = dict(x=zero, y=zero, z=z, vx=zero, vy=zero, vz=zero, ax=ax, ay=ay, az=az, step=0)
    st = orc.run(p, st, 40000)
    assert rel(st["z"][1] - st["z"][0], d) < 1e-10
    assert abs(st["z"][1] + st["z"][0]) < 1e-10 * d


def test_three_ion_chain(orc):
    """Three-ion chain: outer ions at +-(5/4)^(1/3) l, l = (k_C e^2/(m wz^2))^(1/3)."""
    wz = 2 * math.pi * 200e3
    p = P(orc, omega=(2 * math.pi * 1e6, 2 * math.pi * 1e6, wz))
    ell = W.chain_length_scale(wz)
    assert abs(ell - 13.0e-6) < 0.05e-6
    s = (5 / 4) ** (1 / 3) * ell
    z = np.array([-s, 0.0, s])
    ax, ay, az = orc.accel(p, 0.0, np.zeros(3), np.zeros(3), z)
    aC = W.K_COULOMB * W.E_CHARGE ** 2 / (W.MASS_40U * s * s)
    assert np.all(np.abs(az) <= 1e-12 * aC)


# --------------------------------------------------------------------------
# Invariants of the pair sum.
def test_newton_third_law(orc):
    rng = np.random.default_rng(11)
    n = 700
    pos = W.ellipsoid_uniform(n, (20e-6, 20e-6, 100e-6), rng)
    q = W.E_CHARGE * rng.choice([-1.0, 1.0, 2.0], size=n)
    p = P(orc)
    ax, ay, az, _, _ = orc.coulomb(p, pos[0], pos[1], pos[2], q)
    F = W.MASS_40U * np.stack([ax, ay, az])
    tot = np.abs(F).sum(axis=1)
    assert np.all(np.abs(F.sum(axis=1)) <= 1e-12 * tot)


def test_ring_symmetry(orc):
    """Ions on a ring: force radial, magnitude k_C e^2/(4 R^2) sum_k 1/sin(pi k/N)."""
    for n in (2, 3, 7, 64, 501):
        R = 37e-6
        pos = W.ring(n, R)
        p = P(orc)
        ax, ay, az, phi, _ = orc.coulomb(p, pos[0], pos[1], pos[2], want_phi=True)
        k = np.arange(1, n)
        mag = W.K_COULOMB * W.E_CHARGE ** 2 / (4 * R * R) * np.sum(1 / np.sin(np.pi * k / n)) / W.MASS_40U
        th = 2 * np.pi * np.arange(n) / n
        radial = ax * np.cos(th) + ay * np.sin(th)
        tang = -ax * np.sin(th) + ay * np.cos(th)
        # Input positions carry the rounding of cos/sin(2 pi i/N) (~ eps R); the
        # nearest-neighbour pair forces exceed the net force by ~N, so that
        # rounding reaches the result as ~N^2 eps.
        tol = 2e-15 + 2.2e-16 * n * n
        assert np.all(np.abs(radial - mag) <= tol * mag)
        assert np.all(np.abs(tang) <= tol * mag)
        assert np.all(az == 0)
        # potential: phi_i = e/(2R) sum_k 1/sin(pi k/N)
        phi_cf = W.E_CHARGE / (2 * R) * np.sum(1 / np.sin(np.pi * k / n))
        assert np.all(np.abs(phi - phi_cf) <= 1e-13 * phi_cf)


def _mp_coulomb(pos, q, i, dps=40):
    import mpmath as mp
    mp.mp.dps = dps
    n = pos.shape[1]
    acc = [mp.mpf(0)] * 3
    absf = mp.mpf(0)
    phi = mp.mpf(0)
    for j in range(n):
        if j == i:
            continue
        d = [mp.mpf(float(pos[c, i])) - mp.mpf(float(pos[c, j])) for c in range(3)]
        r = mp.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
        for c in range(3):
            acc[c] += mp.mpf(float(q[j])) * d[c] / r ** 3
        absf += abs(mp.mpf(float(q[j]))) / r ** 2
        phi += mp.mpf(float(q[j])) / r
    pref = mp.mpf(W.K_COULOMB) * mp.mpf(float(q[i])) / mp.mpf(W.MASS_40U)
    return [pref * a for a in acc], abs(pref) * absf, phi


def test_bruteforce_high_precision(orc):
    """Tiny systems against a 40-digit evaluation of the same definition.
    Each FP64 pair term carries about eight roundings (difference, r^2, sqrt,
    divide, cube, two products), so its relative error is below ~8 ulp; the
    compensated sum adds almost nothing.  Conditioned error <= 2e-15."""
    rng = np.random.default_rng(5)
    for n in (2, 3, 5, 8):
        pos = W.ellipsoid_uniform(n, (20e-6, 20e-6, 100e-6), rng)
        q = W.E_CHARGE * rng.choice([-1.0, 1.0, 2.0], size=n)
        p = P(orc)
        ax, ay, az, phi, absf = orc.coulomb(p, pos[0], pos[1], pos[2], q, want_phi=True, want_absf=True)
        for i in range(n):
            acc, af, ph = _mp_coulomb(pos, q, i)
            err = math.sqrt(sum((float(a) - b) ** 2 for a, b in zip(acc, (ax[i], ay[i], az[i]))))
            assert err <= 2e-15 * float(af)
            assert rel(absf[i], float(af)) < 1e-14
            assert abs(phi[i] - float(ph)) <= 1e-15 * abs(float(ph))


def test_softening_plummer(orc):
    """With softening the pair term is d/(r^2+eps^2)^(3/2): two ions at distance d."""
    d, eps2 = 3e-6, (1e-6) ** 2
    p = P(orc, soft2=eps2)
    ax, ay, az, phi, _ = orc.coulomb(p, np.array([0.0, d]), np.zeros(2), np.zeros(2), want_phi=True)
    expect = W.K_COULOMB * W.E_CHARGE ** 2 / W.MASS_40U * d / (d * d + eps2) ** 1.5
    assert rel(ax[1], expect) < 1e-14 and rel(-ax[0], expect) < 1e-14
    assert rel(phi[0], W.E_CHARGE / math.sqrt(d * d + eps2)) < 1e-14


def test_permutation_and_order_invariance(orc):
    rng = np.random.default_rng(9)
    n = 300
    pos = W.ellipsoid_uniform(n, (20e-6, 20e-6, 100e-6), rng)
    p = P(orc)
    a = orc.coulomb(p, *pos, want_absf=True)
    perm = rng.permutation(n)
    b = orc.coulomb(p, pos[0][perm], pos[1][perm], pos[2][perm])
    r = orc.coulomb(p, *pos, reverse=True)
    for c in range(3):
        assert np.all(np.abs(b[c] - a[c][perm]) <= 2e-16 * a[4][perm])
        assert np.all(np.abs(r[c] - a[c]) <= 2e-16 * a[4])


def test_determinism_across_threads(orc):
    rng = np.random.default_rng(3)
    pos = W.ellipsoid_uniform(257, (20e-6, 20e-6, 100e-6), rng)
    p = P(orc)
    nt = orc.get_threads()
    orc.set_threads(1)
    a = orc.coulomb(p, *pos)
    orc.set_threads(max(2, nt))
    b = orc.coulomb(p, *pos)
    orc.set_threads(nt)
    for c in range(3):
        assert np.array_equal(a[c], b[c])


# --------------------------------------------------------------------------
# Integrator (Sec. II) against exact discrete solutions.
def test_verlet_harmonic_closed_form(orc):
    """Velocity Verlet for x'' = -w^2 x is the linear recurrence
    x_{n+1} - 2 cos(th) x_n + x_{n-1} = 0 with cos(th) = 1 - (w dt)^2/2, so
    x_n = x0 cos(n th) + dt v0 sin(n th)/sin(th) exactly."""
    w = (2 * math.pi * 1e6, 2 * math.pi * 0.7e6, 2 * math.pi * 200e3)
    dt = 5e-9
    p = P(orc, omega=w, dt=dt)
    x0 = np.array([1e-6]), np.array([-2e-6]), np.array([5e-6])
    v0 = np.array([0.3]), np.array([0.1]), np.array([-0.2])
    ax, ay, az = orc.accel(p, 0.0, *x0)
    st = dict(x=x0[0], y=x0[1], z=x0[2], vx=v0[0], vy=v0[1], vz=v0[2], ax=ax, ay=ay, az=az, step=0)
    nsteps = 5000
    st = orc.run(p, st, nsteps)
    for c, key in enumerate("xyz"):
        th = math.acos(1 - (w[c] * dt) ** 2 / 2)
        xn = x0[c][0] * math.cos(nsteps * th) + dt * v0[c][0] * math.sin(nsteps * th) / math.sin(th)
        amp = math.hypot(x0[c][0], dt * v0[c][0] / math.sin(th))
        assert abs(st[key][0] - xn) <= 1e-11 * amp
    assert st["step"] == nsteps


def test_free_damped_ion_recurrence(orc):
    """A free ion with friction: v_{n+1} = rho v_n, rho = (1-c)/(1+c),
    c = gamma dt/(2m); x_{n+1} = x_n + dt (1 - c) v_n."""
    m, dt, g = W.MASS_40U, 2e-9, 3e-20
    p = P(orc, gamma=g, dt=dt)
    c = g * dt / (2 * m)
    rho = (1 - c) / (1 + c)
    v0 = np.array([1.5])
    zero = np.zeros(1)
    st = dict(x=zero, y=zero, z=zero, vx=v0, vy=zero, vz=zero,
              ax=-g / m * v0, ay=zero, az=zero, step=0)
    n = 3000
    st = orc.run(p, st, n)
    v_cf = v0[0] * rho ** n
    x_cf = dt * (1 - c) * v0[0] * (1 - rho ** n) / (1 - rho)
    assert rel(st["vx"][0], v_cf) < 1e-12
    assert rel(st["x"][0], x_cf) < 1e-12
    assert rel(st["ax"][0], -g / m * v_cf) < 1e-12


def test_rf_single_ion_matches_ode(orc):
    """RF trap (Eq. 1 with the Mathieu q): one ion integrated by the oracle with
    a small step agrees with a high-accuracy ODE solution of
    x'' = -(q W^2/2) cos(W t + ph) x, y'' = +(...) y, z'' = -wz^2 z."""
    from scipy.integrate import solve_ivp
    q, Om, ph, wz = 0.3, 2 * math.pi * 10e6, 0.4, 2 * math.pi * 200e3
    dt = 2e-10
    nsteps = 2000  # four RF periods
    p = P(orc, trap="rf", q_mathieu=q, omega_rf=Om, rf_phase=ph, omega=(0, 0, wz), dt=dt)
    x0 = np.array([2e-6]), np.array([-1e-6]), np.array([3e-6])
    v0 = np.array([0.5]), np.array([0.2]), np.array([-0.1])
    ax, ay, az = orc.accel(p, 0.0, *x0)
    st = dict(x=x0[0], y=x0[1], z=x0[2], vx=v0[0], vy=v0[1], vz=v0[2], ax=ax, ay=ay, az=az, step=0)
    st = orc.run(p, st, nsteps)

    def rhs(t, s):
        c = 0.5 * q * Om * Om * math.cos(Om * t + ph)
        return [s[3], s[4], s[5], -c * s[0], c * s[1], -wz * wz * s[2]]
    T = nsteps * dt
    sol = solve_ivp(rhs, (0, T), [x0[0][0], x0[1][0], x0[2][0], v0[0][0], v0[1][0], v0[2][0]],
                    rtol=1e-12, atol=1e-20, method="DOP853")
    ref = sol.y[:, -1]
    for c, key in enumerate("xyz"):
        assert abs(st[key][0] - ref[c]) < 2e-4 * 3e-6, (key, st[key][0], ref[c])
    # the sign matters: flipping the RF sign on x gives a clearly different orbit
    p_bad = P(orc, trap="rf", q_mathieu=-q, omega_rf=Om, rf_phase=ph, omega=(0, 0, wz), dt=dt)
    st_bad = orc.run(p_bad, dict(x=x0[0], y=x0[1], z=x0[2], vx=v0[0], vy=v0[1], vz=v0[2],
                                 ax=ax, ay=ay, az=az, step=0), nsteps)
    assert abs(st_bad["x"][0] - ref[0]) > 1e-2 * 3e-6


def test_energy_conservation_dt2(orc):
    """No friction, static trap: the Verlet energy error stays bounded and its
    maximum shrinks about 4x when dt halves (second order)."""
    rng = np.random.default_rng(21)
    n = 24
    pos = W.ellipsoid_uniform(n, (15e-6, 15e-6, 60e-6), rng)
    vel = W.thermal_velocities(n, 1e-3, W.MASS_40U, rng)
    errs = []
    for dt, nsteps in ((4e-9, 2500), (2e-9, 5000)):
        p = P(orc, omega=(2 * math.pi * 1e6, 2 * math.pi * 1e6, 2 * math.pi * 200e3), dt=dt)
        ax, ay, az = orc.accel(p, 0.0, *pos)
        st = dict(x=pos[0], y=pos[1], z=pos[2], vx=vel[0], vy=vel[1], vz=vel[2],
                  ax=ax, ay=ay, az=az, step=0)
        e0 = orc.energy(p, 0, *pos, *vel)[3]
        emax = 0.0
        for _ in range(50):
            st = orc.run(p, st, nsteps // 50)
            e = orc.energy(p, st["step"], st["x"], st["y"], st["z"], st["vx"], st["vy"], st["vz"])[3]
            emax = max(emax, abs(e - e0) / abs(e0))
        errs.append(emax)
    assert errs[0] < 1e-4
    assert 2.8 < errs[0] / errs[1] < 5.5, errs


def test_energy_closed_forms(orc):
    """Ring energies: Coulomb (N k_C e^2/(4R)) sum_k 1/sin(pi k/N); kinetic
    (m/2) sum v^2; harmonic trap (m/2) sum w_k^2 x_k^2; RF trap potential
    (m/2)(c (x^2 - y^2) + wz^2 z^2) with c = (q W^2/2) cos(W t + ph)."""
    n, R = 16, 20e-6
    pos = W.ring(n, R)
    pos[2] = 1e-6
    vel = np.tile(np.array([[0.1], [0.2], [-0.3]]), (1, n))
    w = (2 * math.pi * 1e6, 2 * math.pi * 0.9e6, 2 * math.pi * 200e3)
    p = P(orc, omega=w)
    e = orc.energy(p, 0, *pos, *vel)
    k = np.arange(1, n)
    uc = n * W.K_COULOMB * W.E_CHARGE ** 2 / (4 * R) * np.sum(1 / np.sin(np.pi * k / n))
    m = W.MASS_40U
    assert rel(e[2], uc) < 1e-13
    assert rel(e[0], 0.5 * m * n * (0.01 + 0.04 + 0.09)) < 1e-14
    ut = 0.5 * m * np.sum(w[0] ** 2 * pos[0] ** 2 + w[1] ** 2 * pos[1] ** 2 + w[2] ** 2 * pos[2] ** 2)
    assert rel(e[1], ut) < 1e-13
    assert e[3] == e[0] + e[1] + e[2]
    q, Om, ph, dt, step = 0.3, 2 * math.pi * 10e6, 0.25, 2e-9, 7
    p = P(orc, trap="rf", q_mathieu=q, omega_rf=Om, rf_phase=ph, omega=(0, 0, w[2]), dt=dt)
    e = orc.energy(p, step, *pos, *vel)
    c = 0.5 * q * Om * Om * math.cos(Om * step * dt + ph)
    ut = 0.5 * m * np.sum(c * (pos[0] ** 2 - pos[1] ** 2) + w[2] ** 2 * pos[2] ** 2)
    assert abs(e[1] - ut) <= 1e-13 * abs(ut)


def test_energy_is_potential_of_force(orc):
    """-grad(U_coulomb + U_trap)/m equals the oracle acceleration (central FD)."""
    rng = np.random.default_rng(4)
    n = 6
    pos = W.ellipsoid_uniform(n, (10e-6, 10e-6, 30e-6), rng)
    zero = np.zeros((3, n))
    p = P(orc, omega=(2 * math.pi * 1e6, 2 * math.pi * 0.8e6, 2 * math.pi * 200e3))
    a = np.stack(orc.accel(p, 0.0, *pos))
    h = 1e-11
    for i in range(n):
        for c in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[c, i] += h
            pm[c, i] -= h
            up = orc.energy(p, 0, *pp, *zero)
            um = orc.energy(p, 0, *pm, *zero)
            g = ((up[1] + up[2]) - (um[1] + um[2])) / (2 * h)
            assert abs(-g / W.MASS_40U - a[c, i]) <= 1e-6 * np.abs(a).max()


# --------------------------------------------------------------------------
# Derivatives: VJP and the trajectory adjoint against finite differences.
def test_forces_vjp_matches_fd(orc):
    rng = np.random.default_rng(8)
    n = 12
    pos = W.ellipsoid_uniform(n, (10e-6, 10e-6, 30e-6), rng)
    q = W.E_CHARGE * rng.choice([1.0, 2.0], size=n)
    lam = rng.standard_normal((3, n))
    delta = rng.standard_normal((3, n))
    for include_trap in (False, True):
        p = P(orc, omega=(2 * math.pi * 1e6, 2 * math.pi * 0.8e6, 2 * math.pi * 200e3))
        g = np.stack(orc.forces_vjp(p, 0.0, *pos, *lam, q=q, include_trap=include_trap))
        h = 1e-12

        def A(x):
            if include_trap:
                return np.stack(orc.accel(p, 0.0, *x, q=q))
            return np.stack(orc.coulomb(p, *x, q=q)[:3])
        d1 = (np.sum(lam * A(pos + h * delta)) - np.sum(lam * A(pos - h * delta))) / (2 * h)
        d2 = (np.sum(lam * A(pos + 2 * h * delta)) - np.sum(lam * A(pos - 2 * h * delta))) / (4 * h)
        fd = (4 * d1 - d2) / 3
        assert rel(np.sum(g * delta), fd) < 1e-7


def _verlet_1d(x0, v0, w, dt, T):
    """Exact discrete velocity-Verlet solution of x'' = -w^2 x after T steps
    (Sec. II update; cos th = 1 - (w dt)^2/2): x_T and its derivatives with
    respect to x0, v0 and w."""
    th = math.acos(1 - (w * dt) ** 2 / 2)
    s, c, sT, cT = math.sin(th), math.cos(th), math.sin(T * th), math.cos(T * th)
    xT = x0 * cT + dt * v0 * sT / s
    dx_dth = -T * x0 * sT + dt * v0 * (T * cT * s - sT * c) / (s * s)
    dth_dw = w * dt * dt / s
    return xT, cT, dt * sT / s, dx_dth * dth_dw


def test_trajectory_loss_single_ion_closed_form(orc):
    """One ion (no Coulomb term) in a static harmonic trap: the trajectory
    loss L = (m/2) sum_k w_k^2 x_T,k^2 + |x_T - target|^2 and its gradients
    follow from the exact discrete Verlet solution x_T = x0 cos(T th) +
    dt v0 sin(T th)/sin(th), component by component.  A forward that drops
    the dt^2 a/2 drift term, takes a_0 at the wrong state, or a loss that
    drops the trap energy or the target term fails here."""
    m, dt, T = W.MASS_40U, 3e-9, 700
    w = (2 * math.pi * 1.1e6, 2 * math.pi * 0.8e6, 2 * math.pi * 210e3)
    x0 = np.array([[1.3e-6], [-2.1e-6], [4.7e-6]])
    v0 = np.array([[0.21], [-0.07], [0.33]])
    tgt = np.array([[0.4e-6], [0.9e-6], [-3.0e-6]])
    p = P(orc, omega=w, dt=dt)
    loss, gx, gv, gw = orc.trajectory_grad(p, x0, v0, T, tgt)
    L_ref = 0.0
    for k in range(3):
        xT, dxx, dxv, dxw = _verlet_1d(x0[k, 0], v0[k, 0], w[k], dt, T)
        dLdx = m * w[k] ** 2 * xT + 2 * (xT - tgt[k, 0])
        L_ref += 0.5 * m * w[k] ** 2 * xT ** 2 + (xT - tgt[k, 0]) ** 2
        amp = abs(dLdx) * math.hypot(1.0, dt / math.sin(math.acos(1 - (w[k] * dt) ** 2 / 2)))
        assert abs(gx[k, 0] - dLdx * dxx) <= 1e-9 * amp, k
        assert abs(gv[k, 0] - dLdx * dxv) <= 1e-9 * amp, k
        gw_ref = m * w[k] * xT ** 2 + dLdx * dxw
        assert rel(gw[k], gw_ref) < 1e-8, (k, gw[k], gw_ref)
    assert rel(loss, L_ref) < 1e-11


def test_trajectory_loss_matches_run_and_energy(orc):
    """With Coulomb interactions: the adjoint's own forward and loss equal a
    run of the pinned integrator (or_run, Sec. II) followed by the pinned
    energies (or_energy) and the squared distance to the target, evaluated
    here separately.  The target sits 3 pm from the run's final positions, so
    the three terms are of one size (about 1e-22 in the loss's plain SI sum)
    and a forward that strays by more than about 1e-14 m changes the loss."""
    rng = np.random.default_rng(31)
    n, nsteps = 6, 250
    a, c = W.cold_fluid_spheroid(n, 2 * math.pi * 1e6, 2 * math.pi * 200e3)
    x0 = W.ellipsoid_uniform(n, (a, a, c), rng)
    v0 = W.thermal_velocities(n, 1e-3, W.MASS_40U, rng)
    p = P(orc, omega=(2 * math.pi * 1e6, 2 * math.pi * 0.9e6, 2 * math.pi * 200e3), dt=2e-9)
    ax, ay, az = orc.accel(p, 0.0, *x0)
    st = dict(x=x0[0], y=x0[1], z=x0[2], vx=v0[0], vy=v0[1], vz=v0[2], ax=ax, ay=ay, az=az, step=0)
    st = orc.run(p, st, nsteps)
    xT = np.stack([st["x"], st["y"], st["z"]])
    target = xT + 3e-12 * rng.choice([-1.0, 1.0], size=(3, n))
    loss = orc.trajectory_grad(p, x0, v0, nsteps, target)[0]
    e = orc.energy(p, 0, *xT, st["vx"], st["vy"], st["vz"])
    d2 = float(np.sum((xT - target) ** 2))
    ref = math.fsum([e[1], e[2], d2])
    for term in (e[1], e[2], d2):  # trap, Coulomb and target terms all count
        assert term > 0.05 * ref, (e, d2)
    assert rel(loss, ref) < 1e-9, (loss, ref)


def test_trajectory_grad_matches_fd(orc):
    """Discrete adjoint of the Verlet trajectory vs Richardson-extrapolated
    central differences, in random x0 directions and in each omega_k."""
    rng = np.random.default_rng(12)
    n, nsteps = 8, 300
    a, c = W.cold_fluid_spheroid(n, 2 * math.pi * 1e6, 2 * math.pi * 200e3)
    x0 = W.ellipsoid_uniform(n, (a, a, c), rng)
    v0 = W.thermal_velocities(n, 1e-3, W.MASS_40U, rng)
    target = x0 + 1e-7 * rng.standard_normal((3, n))
    w = [2 * math.pi * 1e6, 2 * math.pi * 0.9e6, 2 * math.pi * 200e3]
    p = P(orc, omega=tuple(w), dt=1e-9)
    loss, gx, gv, gw = orc.trajectory_grad(p, x0, v0, nsteps, target)
    ell = W.chain_length_scale(w[2])

    def L(x, wv=w):
        return orc.trajectory_grad(P(orc, omega=tuple(wv), dt=1e-9), x, v0, nsteps, target)[0]

    def fd(f, h):
        d1 = (f(h) - f(-h)) / (2 * h)
        d2 = (f(2 * h) - f(-2 * h)) / (4 * h)
        return (4 * d1 - d2) / 3
    for _ in range(3):
        dirn = rng.standard_normal((3, n))
        g_fd = fd(lambda h: L(x0 + h * dirn), 1e-6 * ell)
        assert rel(np.sum(gx * dirn), g_fd) < 1e-5
    for k in range(3):
        def fw(h, k=k):
            wv = list(w)
            wv[k] += h
            return L(x0, wv)
        g_fd = fd(fw, 1e-6 * w[k])
        assert rel(gw[k], g_fd) < 1e-5, (k, gw[k], g_fd)


# --------------------------------------------------------------------------
# Counter-based RNG.
def test_philox_known_answers(orc):
    with open(os.path.join(GOLD, "philox4x32_10_kat.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        assert orc.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def test_normals_statistics(orc):
    xs = np.array([orc.normals3(77, 3, s, i) for s in range(60) for i in range(500)])
    assert abs(xs.mean()) < 0.02
    assert abs(xs.var() - 1.0) < 0.03
    assert abs(np.corrcoef(xs[:, 0], xs[:, 2])[0, 1]) < 0.03
    assert not np.array_equal(orc.normals3(77, 3, 5, 9), orc.normals3(77, 4, 5, 9))
    assert np.array_equal(orc.normals3(77, 3, 5, 9), orc.normals3(77, 3, 5, 9))


def test_langevin_equipartition(orc):
    """Free ions with friction and the Langevin kick thermalise to the set
    temperature (fluctuation-dissipation): <m v^2> / kB = T within sampling."""
    n, T, m = 400, 0.5e-3, W.MASS_40U
    p = P(orc, gamma=1e-19, dt=5e-9, noise_T=T, seed=99, soft2=1.0)  # huge softening: no Coulomb
    p.k_coulomb = 0.0
    z = np.zeros(n)
    st = dict(x=z, y=z, z=z, vx=z, vy=z, vz=z, ax=z, ay=z, az=z, step=0)
    st = orc.run(p, st, 3000)  # gamma/m * t = 22 relaxation times
    v2 = np.concatenate([st["vx"], st["vy"], st["vz"]]) ** 2
    T_est = m * v2.mean() / W.K_B
    assert abs(T_est / T - 1) < 0.1


# --------------------------------------------------------------------------
# Two species (Sec. II: interactions 1-1, 2-2 and 1-2 in one all-pairs sum).
def test_two_species_equilibrium(orc):
    """Ions of charge q1, q2 in the trap of the reference species (Q, M):
    the trap field is fixed, so force balance gives
    d^3 = k_C Q (q1 + q2) / (M w_z^2) and z1 = q2 d/(q1 + q2) -- independent
    of the masses."""
    wz = 2 * math.pi * 200e3
    p = P(orc, omega=(2 * math.pi * 1e6, 2 * math.pi * 1e6, wz))
    Q, M = W.E_CHARGE, W.MASS_40U
    q = np.array([Q, 2 * Q])
    m = np.array([M, 9 * W.AMU])
    d = (W.K_COULOMB * Q * (q[0] + q[1]) / (M * wz * wz)) ** (1 / 3)
    z = np.array([q[1] * d / (q[0] + q[1]), -q[0] * d / (q[0] + q[1])])
    a = np.stack(orc.accel(p, 0.0, np.zeros(2), np.zeros(2), z, q=q, masses=m))
    aC = W.K_COULOMB * q[0] * q[1] / (m * d * d)
    assert np.all(np.abs(a[2]) <= 1e-12 * aC)
    # and the same positions are NOT a balance if the masses are ignored in the trap term
    a_bad = np.stack(orc.accel(p, 0.0, np.zeros(2), np.zeros(2), np.array([d / 2, -d / 2]), q=q, masses=m))
    assert np.max(np.abs(a_bad[2]) / aC) > 1e-3


def test_two_species_momentum(orc):
    rng = np.random.default_rng(12)
    n = 500
    pos = W.ellipsoid_uniform(n, (20e-6, 20e-6, 100e-6), rng)
    q = W.E_CHARGE * rng.choice([1.0, 2.0], size=n)
    m = W.AMU * rng.choice([40.0, 9.0, 138.0], size=n)
    ax, ay, az, _, absf = orc.coulomb(P(orc), *pos, q=q, masses=m, want_absf=True)
    F = m * np.stack([ax, ay, az])
    tot = np.abs(F).sum(axis=1)
    assert np.all(np.abs(F.sum(axis=1)) <= 1e-12 * tot)


def test_two_species_harmonic_verlet(orc):
    """A single ion of charge q_i and mass m_i oscillates at w_i^2 = s_i w^2,
    s_i = (q_i/m_i)/(Q/M); Verlet reproduces the exact discrete solution."""
    w, dt = 2 * math.pi * 300e3, 4e-9
    p = P(orc, omega=(w, w, w), dt=dt)
    q, m = np.array([2 * W.E_CHARGE]), np.array([9 * W.AMU])
    s = (q[0] / m[0]) / (W.E_CHARGE / W.MASS_40U)
    x0 = np.array([3e-6]); v0 = np.array([0.2]); zero = np.zeros(1)
    ax, ay, az = orc.accel(p, 0.0, x0, zero, zero, q=q, masses=m)
    st = dict(x=x0, y=zero, z=zero, vx=v0, vy=zero, vz=zero, ax=ax, ay=ay, az=az, step=0)
    nsteps = 2000
    st = orc.run(p, st, nsteps, q=q, masses=m)
    th = math.acos(1 - s * (w * dt) ** 2 / 2)
    xn = x0[0] * math.cos(nsteps * th) + dt * v0[0] * math.sin(nsteps * th) / math.sin(th)
    assert abs(st["x"][0] - xn) <= 1e-11 * math.hypot(x0[0], dt * v0[0] / math.sin(th))


def test_two_species_energy_is_potential_of_force(orc):
    rng = np.random.default_rng(14)
    n = 5
    pos = W.ellipsoid_uniform(n, (10e-6, 10e-6, 30e-6), rng)
    q = W.E_CHARGE * np.array([1.0, 2.0, 1.0, 1.0, 2.0])
    m = W.AMU * np.array([40.0, 9.0, 9.0, 138.0, 40.0])
    zero = np.zeros((3, n))
    p = P(orc, omega=(2 * math.pi * 1e6, 2 * math.pi * 0.8e6, 2 * math.pi * 200e3))
    a = np.stack(orc.accel(p, 0.0, *pos, q=q, masses=m))
    h = 1e-11
    for i in range(n):
        for c in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[c, i] += h
            pm[c, i] -= h
            up = orc.energy(p, 0, *pp, *zero, q=q, masses=m)
            um = orc.energy(p, 0, *pm, *zero, q=q, masses=m)
            g = ((up[1] + up[2]) - (um[1] + um[2])) / (2 * h)
            assert abs(-g / m[i] - a[c, i]) <= 1e-6 * np.abs(a).max()
