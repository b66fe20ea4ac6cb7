"""Seeded synthetic inputs shaped like the paper's trapped-ion workloads.

This module holds input generators and physical constants only: no part of
the force, trap, integrator, energy or adjoint arithmetic lives here.  Both
the CUDA library's tests and the CPU oracle's tests draw their inputs from
it, so the two sides see identical arrays.

Every workload is a plain dict:
  n      -- number of ions
  pos    -- float64 array (3, n): rows x, y, z in metres
  vel    -- float64 array (3, n): rows vx, vy, vz in m/s
  q      -- per-ion charge in coulombs, or None for a single species
  phys   -- dict of physical parameters (SI units) with the keys
            k_coulomb, mass, charge, soft2, trap ('harmonic' | 'rf'),
            omega (3,), omega_rate (3,), q_mathieu, omega_rf, rf_phase,
            gamma, dt, t0, noise_T, seed
  steps  -- number of Verlet steps the workload runs

The physical setting is the paper's: singly charged ions (Ca+ analogue,
mass 40 u) in a linear RF trap or its harmonic pseudopotential (Sec. II,
Eq. 1), with laser-cooling friction, at N from 10 to 1e5 (Sec. I).
"""
import math

import numpy as np

# CODATA 2018 (exact where the SI fixes them).
E_CHARGE = 1.602176634e-19      # C
EPS0 = 8.8541878128e-12         # F/m
K_B = 1.380649e-23              # J/K
AMU = 1.66053906660e-27         # kg
K_COULOMB = 1.0 / (4.0 * math.pi * EPS0)
MASS_40U = 40.0 * AMU
TWO_PI = 2.0 * math.pi


def phys(**kw):
    """Physical-parameter dict with the paper's defaults (one species, 40 u,
    charge +e, no softening, static harmonic trap, no friction, no noise)."""
    p = dict(k_coulomb=K_COULOMB, mass=MASS_40U, charge=E_CHARGE, soft2=0.0,
             trap="harmonic", omega=(0.0, 0.0, 0.0), omega_rate=(0.0, 0.0, 0.0),
             q_mathieu=0.0, omega_rf=0.0, rf_phase=0.0, gamma=0.0, dt=1e-9, t0=0.0,
             noise_T=0.0, seed=0)
    for k, v in kw.items():
        if k not in p:
            raise KeyError(k)
        p[k] = v
    p["omega"] = tuple(float(v) for v in p["omega"])
    p["omega_rate"] = tuple(float(v) for v in p["omega_rate"])
    return p


def ellipsoid_uniform(n, semi_axes, rng):
    """n points uniform in the ellipsoid with the given semi-axes (m)."""
    g = rng.standard_normal((3, n))
    g /= np.linalg.norm(g, axis=0, keepdims=True)
    r = rng.random(n) ** (1.0 / 3.0)
    return g * r * np.asarray(semi_axes, dtype=np.float64)[:, None]


def thermal_velocities(n, temperature, mass, rng):
    """Maxwell-Boltzmann velocities: N(0, kB T / m) per component."""
    return rng.standard_normal((3, n)) * math.sqrt(K_B * temperature / mass)


def min_pair_distance(pos):
    """Smallest distance between two distinct ions (0 if two coincide)."""
    from scipy.spatial import cKDTree
    if pos.shape[1] < 2:
        return math.inf
    d, _ = cKDTree(pos.T).query(pos.T, k=2)
    return float(d[:, 1].min())


def spheroid_depolarization(a, c):
    """Depolarisation factors (N_x, N_y, N_z) of a spheroid with equatorial
    semi-axis a and polar semi-axis c (prolate c > a, oblate c < a, sphere)."""
    if abs(c - a) <= 1e-12 * a:
        return (1.0 / 3.0,) * 3
    if c > a:
        e = math.sqrt(1.0 - (a / c) ** 2)
        nz = (1.0 - e * e) / e ** 3 * (math.atanh(e) - e)
    else:
        e = math.sqrt((a / c) ** 2 - 1.0)
        nz = (1.0 + e * e) / e ** 3 * (e - math.atan(e))
    nx = 0.5 * (1.0 - nz)
    return (nx, nx, nz)


def cold_fluid_omegas(n, a, c, mass=MASS_40U, charge=E_CHARGE):
    """Trap frequencies (rad/s) for which a uniform-density spheroid of n ions
    with semi-axes (a, a, c) is a cold-fluid equilibrium:
    omega_k^2 = N_k omega_p^2, omega_p^2 = charge^2 density / (eps0 m)."""
    density = n / (4.0 / 3.0 * math.pi * a * a * c)
    wp2 = charge * charge * density / (EPS0 * mass)
    return tuple(math.sqrt(nk * wp2) for nk in spheroid_depolarization(a, c))


def cold_fluid_spheroid(n, omega_r, omega_z, mass=MASS_40U, charge=E_CHARGE):
    """Inverse of cold_fluid_omegas: semi-axes (a, c) of the uniform spheroid
    of n ions held by radial/axial frequencies omega_r, omega_z."""
    target = (omega_z / omega_r) ** 2
    lo, hi = 1e-3, 1e3  # aspect ratio c/a
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        nx, _, nz = spheroid_depolarization(1.0, mid)
        if nz / nx > target:
            lo = mid
        else:
            hi = mid
    ratio = math.sqrt(lo * hi)
    nx, _, nz = spheroid_depolarization(1.0, ratio)
    wp2 = omega_r ** 2 / nx
    density = wp2 * EPS0 * mass / (charge * charge)
    a = (n / (4.0 / 3.0 * math.pi * ratio * density)) ** (1.0 / 3.0)
    return a, ratio * a


def chain_length_scale(omega_z, mass=MASS_40U, charge=E_CHARGE):
    """l = (k_C e^2 / (m omega_z^2))^(1/3), the natural length of an ion chain."""
    return (K_COULOMB * charge * charge / (mass * omega_z * omega_z)) ** (1.0 / 3.0)


def chain_positions(n, omega_z, mass=MASS_40U, charge=E_CHARGE):
    """Axial positions of an n-ion chain at the quantiles of the continuum
    density lambda(z) ~ 1 - z^2/L^2 with L = l (3 n ln n)^(1/3) (n >= 2)."""
    if n == 1:
        return np.zeros(1)
    ell = chain_length_scale(omega_z, mass, charge)
    L = ell * (3.0 * n * math.log(n)) ** (1.0 / 3.0)
    # CDF of (1 - s^2) on [-1, 1]: F(s) = (2 + 3 s - s^3) / 4; invert by bisection.
    u = (np.arange(n) + 0.5) / n
    lo, hi = -np.ones(n), np.ones(n)
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        f = (2.0 + 3.0 * mid - mid ** 3) / 4.0
        lo = np.where(f < u, mid, lo)
        hi = np.where(f < u, hi, mid)
    return L * 0.5 * (lo + hi)


def _workload(n, pos, vel, phys_, steps, q=None, name=""):
    return dict(n=int(n), pos=np.ascontiguousarray(pos, dtype=np.float64),
                vel=np.ascontiguousarray(vel, dtype=np.float64), q=q, phys=phys_,
                steps=int(steps), name=name)


def cloud_harmonic_1024(n=1024, seed=1):
    """N = 1024 ions of 40 u uniform in a 20 x 20 x 100 um ellipsoid, 10 mK
    velocities, static pseudopotential 2pi(1, 1, 0.2) MHz, dt = 1 ns,
    100 steps, no friction."""
    rng = np.random.default_rng(seed)
    pos = ellipsoid_uniform(n, (20e-6, 20e-6, 100e-6), rng)
    vel = thermal_velocities(n, 10e-3, MASS_40U, rng)
    p = phys(omega=(TWO_PI * 1e6, TWO_PI * 1e6, TWO_PI * 200e3), dt=1e-9, seed=seed)
    return _workload(n, pos, vel, p, 100, name="cloud-harmonic-N%d" % n)


def cloud_rf_16384(n=16384, seed=2):
    """N = 16384 ions, same species and distribution, full time-dependent linear
    Paul trap (Mathieu a = 0, q = 0.3, RF 2pi 10 MHz, axial 2pi 200 kHz),
    friction 1e-20 kg/s, dt = 2 ns, 1000 steps."""
    rng = np.random.default_rng(seed)
    pos = ellipsoid_uniform(n, (20e-6, 20e-6, 100e-6), rng)
    vel = thermal_velocities(n, 10e-3, MASS_40U, rng)
    p = phys(trap="rf", q_mathieu=0.3, omega_rf=TWO_PI * 10e6,
             omega=(0.0, 0.0, TWO_PI * 200e3), gamma=1e-20, dt=2e-9, seed=seed)
    return _workload(n, pos, vel, p, 1000, name="cloud-rf-N%d" % n)


def cloud_large(n=100000, seed=3):
    """N = 1e5 ions uniform in a 200 x 200 x 1000 um ellipsoid held by the
    harmonic pseudopotential for which that spheroid is a cold-fluid
    equilibrium, 10 mK velocities, dt = 1 ns, 50 steps."""
    rng = np.random.default_rng(seed)
    a, c = 200e-6, 1000e-6
    pos = ellipsoid_uniform(n, (a, a, c), rng)
    vel = thermal_velocities(n, 10e-3, MASS_40U, rng)
    p = phys(omega=cold_fluid_omegas(100000, a, c), dt=1e-9, seed=seed)
    return _workload(n, pos, vel, p, 50, name="cloud-large-N%d" % n)


def kz_ensemble(n_inst=512, n_min=32, n_max=4096, seed=4, temperature=0.5e-3, steps=20000):
    """Kibble-Zurek quench ensemble: n_inst independent chains, N_k uniform in
    [n_min, n_max], axial 2pi 100 kHz, radial frequency ramped linearly from
    2pi 1.2 MHz to 2pi 0.6 MHz over `steps` steps of 5 ns, friction 1e-20 kg/s,
    Langevin noise at the Doppler temperature 0.5 mK.

    Returns dict(sizes, offsets, pos (3, total), vel (3, total), phys)."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(n_min, n_max + 1, size=n_inst)
    offsets = np.zeros(n_inst + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    total = int(offsets[-1])
    wz = TWO_PI * 100e3
    dt = 5e-9
    w0, w1 = TWO_PI * 1.2e6, TWO_PI * 0.6e6
    rate = (w1 - w0) / (steps * dt)
    pos = np.zeros((3, total))
    for k, nk in enumerate(sizes):
        pos[2, offsets[k]:offsets[k + 1]] = chain_positions(int(nk), wz)
    vel = thermal_velocities(total, temperature, MASS_40U, rng)
    p = phys(omega=(w0, w0, wz), omega_rate=(rate, rate, 0.0), gamma=1e-20, dt=dt,
             noise_T=temperature, seed=seed)
    return dict(sizes=sizes.astype(np.int64), offsets=offsets, pos=pos, vel=vel, phys=p,
                steps=steps, name="kz-ensemble-%dx[%d..%d]" % (n_inst, n_min, n_max))


def kz_quench_sweep(n_inst=512, n_min=32, n_max=4096, seed=6, temperature=0.5e-3, steps=20000, span=10.0):
    """The Kibble-Zurek ensemble with a quench rate of its own per instance
    (defect statistics against quench time, Sec. I): instance k ramps the
    radial frequency linearly at rate r_k, log-spaced from kz_ensemble's rate
    (k = 0) down to that rate / span, every ramp passing the midpoint
    frequency (w0 + w1) / 2 at the middle of the run, so the slowest quench
    changes the trap least; the instance word of the noise is k.  Sizes,
    chains, velocities, friction, step and temperature as kz_ensemble.

    Returns kz_ensemble's dict with "phys" a list of n_inst dicts."""
    w = kz_ensemble(n_inst=n_inst, n_min=n_min, n_max=n_max, seed=seed, temperature=temperature, steps=steps)
    base = w["phys"]
    w0, w1 = TWO_PI * 1.2e6, TWO_PI * 0.6e6
    t_mid = 0.5 * steps * base["dt"]
    rate0 = base["omega_rate"][0]
    per = []
    for k in range(n_inst):
        r = rate0 / span ** (k / max(n_inst - 1, 1))
        wr = 0.5 * (w0 + w1) - r * t_mid
        p = dict(base)
        p["omega"] = (wr, wr, base["omega"][2])
        p["omega_rate"] = (r, r, 0.0)
        p["instance"] = k
        per.append(p)
    w["phys"] = per
    w["name"] = "kz-quench-sweep-%dx[%d..%d]-span%g" % (n_inst, n_min, n_max, span)
    return w


def adjoint_cloud(n=4096, seed=5, steps=2000):
    """N = 4096 ions in the harmonic pseudopotential 2pi(1, 1, 0.2) MHz,
    uniform in the cold-fluid spheroid that trap holds, 10 mK velocities,
    dt = 1 ns; plus a target lattice: the n simple-cubic points (spacing
    n^(-1/3) of the mean density) nearest the centroid, assigned to ions in
    sorted-z order (ties by index) and jittered by 1 % of the spacing."""
    rng = np.random.default_rng(seed)
    wr, wz = TWO_PI * 1e6, TWO_PI * 200e3
    a, c = cold_fluid_spheroid(n, wr, wz)
    pos = ellipsoid_uniform(n, (a, a, c), rng)
    vel = thermal_velocities(n, 10e-3, MASS_40U, rng)
    p = phys(omega=(wr, wr, wz), dt=1e-9, seed=seed)
    density = n / (4.0 / 3.0 * math.pi * a * a * c)
    h = density ** (-1.0 / 3.0)
    k = int(math.ceil((2.0 * n) ** (1.0 / 3.0))) + 2
    g = np.arange(-k, k + 1) * h
    gx, gy, gz = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([gx.ravel(), gy.ravel(), gz.ravel()])
    order = np.lexsort((np.arange(pts.shape[1]), np.sum(pts * pts, axis=0)))
    pts = pts[:, order[:n]]
    pts = pts[:, np.lexsort((np.arange(n), pts[2]))]
    ion_order = np.lexsort((np.arange(n), pos[2]))
    target = np.empty((3, n))
    target[:, ion_order] = pts
    target += 0.01 * h * rng.uniform(-1.0, 1.0, size=(3, n))
    w = _workload(n, pos, vel, p, steps, name="adjoint-cloud-N%d" % n)
    w["target"] = target
    return w


def ring(n, radius):
    """n ions equally spaced on a circle of the given radius in the z = 0 plane."""
    th = TWO_PI * np.arange(n) / n
    return np.stack([radius * np.cos(th), radius * np.sin(th), np.zeros(n)])


def random_cloud(n, seed, semi_axes=(20e-6, 20e-6, 100e-6), temperature=10e-3):
    """Generic seeded uniform ellipsoid cloud with thermal velocities."""
    rng = np.random.default_rng(seed)
    return ellipsoid_uniform(n, semi_axes, rng), thermal_velocities(n, temperature, MASS_40U, rng)
