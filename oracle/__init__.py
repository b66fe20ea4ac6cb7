"""FP64 CPU oracle for the trapped-ion direct N-body method (arXiv 2106.11143).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA library; it takes plain numpy arrays (SoA, float64) and returns numpy
arrays.

Every function follows a passage of the paper (see nb_oracle.c):
  coulomb      -- Eq. 1 pair sum, Sec. III double loop (1/sqrt, cubed)
  accel        -- Eq. 1: Coulomb + trap + friction
  run          -- Sec. II velocity Verlet (friction solved implicitly)
  energy       -- kinetic / trap / Coulomb energies (plain definitions)
  forces_vjp   -- J^T lambda of the Eq. 1 acceleration (plain derivative)
  trajectory_grad -- discrete adjoint of the Verlet trajectory
  philox4x32_10, normals3 -- counter-based RNG from its published definition
"""
import ctypes as C

import numpy as np

from . import build as _build

_lib = None


class OrParams(C.Structure):
    _fields_ = [
        ("k_coulomb", C.c_double), ("mass", C.c_double), ("charge", C.c_double),
        ("soft2", C.c_double), ("trap", C.c_int32), ("pad0", C.c_int32),
        ("omega", C.c_double * 3), ("omega_rate", C.c_double * 3),
        ("q_mathieu", C.c_double), ("omega_rf", C.c_double), ("rf_phase", C.c_double),
        ("gamma", C.c_double), ("dt", C.c_double), ("t0", C.c_double),
        ("noise_T", C.c_double), ("seed", C.c_uint64), ("instance", C.c_uint32),
        ("pad1", C.c_uint32),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        d = C.POINTER(C.c_double)
        _lib.or_coulomb_range.argtypes = [C.POINTER(OrParams), C.c_int64, C.c_int64, C.c_int64,
                                          d, d, d, d, d, d, d, d, d, C.c_int]
        _lib.or_trap.argtypes = [C.POINTER(OrParams), C.c_double, C.c_int64, d, d, d, d, d, d]
        _lib.or_accel.argtypes = [C.POINTER(OrParams), C.c_double, C.c_int64, d, d, d, d, d, d, d,
                                  d, d, d, C.c_int]
        _lib.or_run.argtypes = [C.POINTER(OrParams), C.c_int64, d, d, d, d, d, d, d, d, d, d,
                                C.POINTER(C.c_int64), C.c_int64, C.c_int]
        _lib.or_run.restype = C.c_int
        _lib.or_energy.argtypes = [C.POINTER(OrParams), C.c_int64, C.c_int64, d, d, d, d, d, d, d, d]
        _lib.or_forces_vjp.argtypes = [C.POINTER(OrParams), C.c_double, C.c_int64, d, d, d, d,
                                       d, d, d, d, d, d, C.c_int]
        _lib.or_trajectory_grad.argtypes = [C.POINTER(OrParams), C.c_int64, d, d, d, C.c_int64,
                                            d, d, d, d, d]
        _lib.or_trajectory_grad.restype = C.c_int
        u32 = C.POINTER(C.c_uint32)
        _lib.or_philox4x32_10.argtypes = [u32, u32, u32]
        _lib.or_normals3.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_int64, d]
        _lib.or_set_threads.argtypes = [C.c_int]
        _lib.or_set_masses.argtypes = [C.POINTER(C.c_double)]
        _lib.or_get_threads.restype = C.c_int
    return _lib


def make_params(k_coulomb, mass, charge, soft2=0.0, trap="harmonic", omega=(0.0, 0.0, 0.0),
                omega_rate=(0.0, 0.0, 0.0), q_mathieu=0.0, omega_rf=0.0, rf_phase=0.0,
                gamma=0.0, dt=1e-9, t0=0.0, noise_T=0.0, seed=0, instance=0):
    p = OrParams()
    p.k_coulomb, p.mass, p.charge, p.soft2 = k_coulomb, mass, charge, soft2
    p.trap = {"harmonic": 0, "rf": 1}[trap]
    p.omega = (C.c_double * 3)(*omega)
    p.omega_rate = (C.c_double * 3)(*omega_rate)
    p.q_mathieu, p.omega_rf, p.rf_phase = q_mathieu, omega_rf, rf_phase
    p.gamma, p.dt, p.t0, p.noise_T = gamma, dt, t0, noise_T
    p.seed, p.instance = int(seed), int(instance)
    return p


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _Masses:
    """Per-ion masses (two species) for the duration of one oracle call."""

    def __init__(self, masses):
        self.m = None if masses is None else _f64(masses)

    def __enter__(self):
        lib().or_set_masses(_ptr(self.m))
        return self

    def __exit__(self, *a):
        lib().or_set_masses(None)


def set_threads(n):
    lib().or_set_threads(int(n))


def get_threads():
    return lib().or_get_threads()


def coulomb(p, x, y, z, q=None, reverse=False, i0=0, i1=None, want_phi=False, want_absf=False,
            masses=None):
    """Coulomb acceleration of particles [i0, i1) (Eq. 1, j != i).

    Returns (ax, ay, az, phi or None, absf or None); phi = sum q_j/s_ij,
    absf = sum of the magnitudes of the pair accelerations (conditioning)."""
    x, y, z = _f64(x), _f64(y), _f64(z)
    q = None if q is None else _f64(q)
    n = x.shape[0]
    i1 = n if i1 is None else i1
    m = i1 - i0
    ax, ay, az = np.empty(m), np.empty(m), np.empty(m)
    phi = np.empty(m) if want_phi else None
    absf = np.empty(m) if want_absf else None
    with _Masses(masses):
        lib().or_coulomb_range(C.byref(p), n, i0, i1, _ptr(x), _ptr(y), _ptr(z), _ptr(q),
                               _ptr(ax), _ptr(ay), _ptr(az), _ptr(phi), _ptr(absf), int(reverse))
    return ax, ay, az, phi, absf


def trap(p, t, x, y, z):
    x, y, z = _f64(x), _f64(y), _f64(z)
    n = x.shape[0]
    ax, ay, az = np.empty(n), np.empty(n), np.empty(n)
    lib().or_trap(C.byref(p), t, n, _ptr(x), _ptr(y), _ptr(z), _ptr(ax), _ptr(ay), _ptr(az))
    return ax, ay, az


def accel(p, t, x, y, z, vx=None, vy=None, vz=None, q=None, reverse=False, masses=None):
    """Total Verlet-state acceleration: Coulomb + trap(t) - (gamma/m) v."""
    x, y, z = _f64(x), _f64(y), _f64(z)
    n = x.shape[0]
    vs = [None, None, None] if vx is None else [_f64(vx), _f64(vy), _f64(vz)]
    q = None if q is None else _f64(q)
    ax, ay, az = np.empty(n), np.empty(n), np.empty(n)
    with _Masses(masses):
        lib().or_accel(C.byref(p), t, n, _ptr(x), _ptr(y), _ptr(z), _ptr(vs[0]), _ptr(vs[1]),
                       _ptr(vs[2]), _ptr(q), _ptr(ax), _ptr(ay), _ptr(az), int(reverse))
    return ax, ay, az


def run(p, state, nsteps, q=None, reverse=False, masses=None):
    """Velocity Verlet for nsteps (Sec. II).  state: dict with x,y,z,vx,vy,vz,
    ax,ay,az (float64 arrays, updated copies are returned) and 'step'."""
    s = {k: _f64(state[k]).copy() for k in ("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az")}
    step = C.c_int64(int(state.get("step", 0)))
    q = None if q is None else _f64(q)
    n = s["x"].shape[0]
    with _Masses(masses):
        rc = lib().or_run(C.byref(p), n, _ptr(q), *[_ptr(s[k]) for k in
                          ("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az")],
                          C.byref(step), int(nsteps), int(reverse))
    if rc != 0:
        raise MemoryError("oracle run failed")
    s["step"] = step.value
    return s


def energy(p, step, x, y, z, vx, vy, vz, q=None, masses=None):
    """(kinetic, trap, Coulomb, total) energies in J at time t0 + step*dt."""
    out = np.empty(4)
    q = None if q is None else _f64(q)
    arrs = [_f64(a) for a in (x, y, z, vx, vy, vz)]
    with _Masses(masses):
        lib().or_energy(C.byref(p), int(step), arrs[0].shape[0], *[_ptr(a) for a in arrs], _ptr(q),
                        _ptr(out))
    return out


def forces_vjp(p, t, x, y, z, lx, ly, lz, q=None, include_trap=False, masses=None):
    """J^T lambda of the acceleration with respect to positions."""
    arrs = [_f64(a) for a in (x, y, z)]
    lam = [_f64(a) for a in (lx, ly, lz)]
    n = arrs[0].shape[0]
    q = None if q is None else _f64(q)
    gx, gy, gz = np.empty(n), np.empty(n), np.empty(n)
    with _Masses(masses):
        lib().or_forces_vjp(C.byref(p), t, n, *[_ptr(a) for a in arrs], _ptr(q),
                            *[_ptr(a) for a in lam], _ptr(gx), _ptr(gy), _ptr(gz), int(include_trap))
    return gx, gy, gz


def trajectory_grad(p, x0, v0, nsteps, target, q=None):
    """Loss and gradients of a Verlet trajectory (harmonic trap, gamma = 0).

    x0, v0, target: (3, n) arrays (rows x, y, z).  Returns
    (loss, grad_x0 (3,n), grad_v0 (3,n), grad_omega (3,))."""
    x0 = _f64(x0).reshape(3, -1)
    v0 = _f64(v0).reshape(3, -1)
    target = _f64(target).reshape(3, -1)
    n = x0.shape[1]
    q = None if q is None else _f64(q)
    loss = np.empty(1)
    gx0, gv0, gw = np.empty((3, n)), np.empty((3, n)), np.empty(3)
    rc = lib().or_trajectory_grad(C.byref(p), n, _ptr(q), _ptr(x0), _ptr(v0), int(nsteps),
                                  _ptr(target), _ptr(loss), _ptr(gx0), _ptr(gv0), _ptr(gw))
    if rc == 2:
        raise ValueError("trajectory_grad supports the static harmonic trap without friction or noise")
    if rc != 0:
        raise MemoryError("oracle trajectory_grad failed")
    return float(loss[0]), gx0, gv0, gw


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xffffffff for v in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def normals3(seed, instance, step, ion):
    out = np.empty(3)
    lib().or_normals3(int(seed), int(instance), int(step), int(ion), _ptr(out))
    return out
