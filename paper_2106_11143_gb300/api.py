"""ctypes binding of libnb.so (include/nb.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI.  Device arrays are torch float64 CUDA tensors; the
binding passes their data pointers and the current torch stream.  There is
no CPU fallback -- if libnb.so is missing, every call raises.
"""
import ctypes as C
import os
from dataclasses import dataclass, fields

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnb.so")

PRECISIONS = {"fp64": 0, "mixed": 1, "mixed_split": 2, "df64": 3, "sqrtdiv": 4, "rsq": 5, "mixed_split_rsq": 8,
              "rsq_nr1": 6, "rsq_nr2": 7}
TRAPS = {"harmonic": 0, "rf": 1}
NB_ACC_COULOMB, NB_ACC_TOTAL = 0, 1


class NbParams(C.Structure):
    _fields_ = [
        ("k_coulomb", C.c_double), ("mass", C.c_double), ("charge", C.c_double),
        ("soft2", C.c_double), ("trap", C.c_int32), ("precision", C.c_int32),
        ("omega", C.c_double * 3), ("omega_rate", C.c_double * 3),
        ("q_mathieu", C.c_double), ("omega_rf", C.c_double), ("rf_phase", C.c_double),
        ("gamma", C.c_double), ("dt", C.c_double), ("t0", C.c_double),
        ("noise_T", C.c_double), ("seed", C.c_uint64), ("instance", C.c_uint32),
        ("reserved", C.c_uint32),
    ]


_dp = C.POINTER(C.c_double)


class NbSystem(C.Structure):
    _fields_ = [
        ("n", C.c_int64),
        ("x", _dp), ("y", _dp), ("z", _dp),
        ("vx", _dp), ("vy", _dp), ("vz", _dp),
        ("ax", _dp), ("ay", _dp), ("az", _dp),
        ("q", _dp), ("step", C.c_int64), ("m", _dp),
    ]


class NBError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__("%s: %s (status %d)%s" % (where, _lib_strerror(status), status,
                                                   (": " + detail) if detail else ""))


_LIB = None


def lib():
    """Load libnb.so (raises if it has not been built: no fallback exists)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libnb.so is not built (run paper_2106_11143_gb300/build.py); "
                               "this package has no CPU fallback")
        L = C.CDLL(LIB_PATH)
        P, S, V = C.POINTER(NbParams), C.POINTER(NbSystem), C.c_void_p
        L.nb_forces.argtypes = [P, S, _dp, C.c_int, V]
        L.nb_step.argtypes = [P, S, C.c_int64, V]
        L.nb_energy.argtypes = [P, S, _dp, V]
        L.nb_forces_vjp.argtypes = [P, S, _dp, _dp, _dp, _dp, _dp, _dp, C.c_int, V]
        L.nb_sync_status.argtypes = [V]
        L.nb_strerror.argtypes = [C.c_int]
        L.nb_strerror.restype = C.c_char_p
        L.nb_last_error.restype = C.c_char_p
        L.nb_version.restype = C.c_char_p
        I64P = C.POINTER(C.c_int64)
        U16P = C.POINTER(C.c_uint16)
        L.nb_step_batched.argtypes = [P, C.c_int32, I64P, S, C.c_int64, V]
        L.nb_step_batched_each.argtypes = [P, C.c_int32, I64P, S, C.c_int64, V]
        L.nb_plan_batched.argtypes = [C.c_int32, I64P, C.c_int32, U16P, U16P, _dp, _dp]
        L.nb_set_tuning.argtypes = [C.c_int32, C.c_int32, C.c_int64, C.c_int64, C.c_int32,
                                    C.c_int32, C.c_int32]
        L.nb_energy_noalloc.argtypes = [P, S, _dp, V]
        L.nb_traj_ckpt_doubles.argtypes = [C.c_int64, C.c_int64, C.c_int64]
        L.nb_traj_ckpt_doubles.restype = C.c_int64
        L.nb_traj_forward.argtypes = [P, S, C.c_int64, C.c_int64, _dp, _dp, _dp, V]
        L.nb_traj_backward.argtypes = [P, S, C.c_int64, C.c_int64, _dp, _dp, _dp, _dp, _dp, _dp, V]
        L.nb_timing_enable.argtypes = [C.c_int64]
        L.nb_timing_read.argtypes = [C.POINTER(C.c_int64), C.POINTER(C.c_double)]
        L.nb_launch_count.restype = C.c_uint64
        L.nb_rinv3_probe.argtypes = [C.c_int32, C.c_int64, _dp, _dp, _dp, C.c_double, _dp, V]
        L.nb_rsqrt_seed_probe.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, V]
        L.nb_plan_info.argtypes = [C.c_int32, C.c_int32, C.c_int64, I64P]
        L.nb_pipe_probe.argtypes = [C.c_int32, C.c_int64, _dp, V]
        L.nb_forces_range.argtypes = [P, S, C.c_int64, C.c_int64, C.c_int, V]
        L.nb_step_range_drift.argtypes = [P, S, C.c_int64, C.c_int64, V]
        L.nb_step_range_kick.argtypes = [P, S, C.c_int64, C.c_int64, V]
        I32P = C.POINTER(C.c_int32)
        L.nb_sym_schedule.argtypes = [C.c_int32, I32P, I32P, I32P]
        L.nb_sym_wait_probe.argtypes = [C.c_int32, C.c_int32, I32P, V]
        for f in ("nb_forces", "nb_step", "nb_energy", "nb_forces_vjp", "nb_sync_status",
                  "nb_release", "nb_timing_enable", "nb_timing_read", "nb_step_batched", "nb_step_batched_each",
                  "nb_plan_batched", "nb_set_tuning", "nb_energy_noalloc", "nb_traj_forward",
                  "nb_traj_backward", "nb_rinv3_probe", "nb_rsqrt_seed_probe", "nb_plan_info",
                  "nb_pipe_probe", "nb_sym_schedule", "nb_forces_range", "nb_step_range_drift",
                  "nb_step_range_kick", "nb_sym_wait_probe"):
            getattr(L, f).restype = C.c_int
        _LIB = L
    return _LIB


def _lib_strerror(status):
    try:
        return lib().nb_strerror(status).decode()
    except Exception:
        return "status"


def _check(status, where):
    if status != 0:
        raise NBError(status, where, lib().nb_last_error().decode())


@dataclass
class Params:
    """Physical parameters (SI) and the pair-arithmetic precision."""
    k_coulomb: float
    mass: float
    charge: float
    soft2: float = 0.0
    trap: str = "harmonic"
    precision: str = "fp64"
    omega: tuple = (0.0, 0.0, 0.0)
    omega_rate: tuple = (0.0, 0.0, 0.0)
    q_mathieu: float = 0.0
    omega_rf: float = 0.0
    rf_phase: float = 0.0
    gamma: float = 0.0
    dt: float = 1e-9
    t0: float = 0.0
    noise_T: float = 0.0
    seed: int = 0
    instance: int = 0

    @classmethod
    def from_phys(cls, phys, precision="fp64", **kw):
        names = {f.name for f in fields(cls)}
        d = {k: v for k, v in phys.items() if k in names}
        d["precision"] = precision
        d.update(kw)
        return cls(**d)

    def to_c(self):
        p = NbParams()
        p.k_coulomb, p.mass, p.charge, p.soft2 = self.k_coulomb, self.mass, self.charge, self.soft2
        p.trap = TRAPS[self.trap]
        p.precision = PRECISIONS[self.precision]
        p.omega = (C.c_double * 3)(*self.omega)
        p.omega_rate = (C.c_double * 3)(*self.omega_rate)
        p.q_mathieu, p.omega_rf, p.rf_phase = self.q_mathieu, self.omega_rf, self.rf_phase
        p.gamma, p.dt, p.t0, p.noise_T = self.gamma, self.dt, self.t0, self.noise_T
        p.seed, p.instance, p.reserved = int(self.seed), int(self.instance), 0
        return p


def _dev(a, device):
    if isinstance(a, torch.Tensor):
        return a.to(device=device, dtype=torch.float64).contiguous()
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=device)


def _ptr(t):
    return None if t is None else C.cast(C.c_void_p(t.data_ptr()), _dp)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


STATE_NAMES = ("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az")


def _packed_state(n, device):
    """One (9, n_pad) float64 device tensor for the Verlet state, rows padded
    to 32 doubles (256 B) so that every array starts aligned."""
    return torch.zeros(len(STATE_NAMES), max(32, -(-n // 32) * 32), dtype=torch.float64, device=device)


class System:
    """Ion state in device memory: SoA float64 tensors x, y, z, vx, vy, vz,
    ax, ay, az (length n), optional per-ion charges q and masses m (several
    species), and the step counter.  The nine state arrays are rows of one
    device tensor, `state` (9 x n_pad, rows padded to 256 B; the first n
    columns are the ions), so the whole state moves to or from the host in one
    copy.  The constructor copies pos/vel/q/m: the library updates its own
    arrays in place, never the caller's."""

    def __init__(self, pos, vel=None, q=None, device="cuda", step=0, m=None):
        pos = _dev(pos, device).reshape(3, -1)
        n = pos.shape[1]
        self.n = n
        self._bind(_packed_state(n, device))
        self.state[0:3, :n].copy_(pos)
        if vel is not None:
            self.state[3:6, :n].copy_(_dev(vel, device).reshape(3, n))
        self.q = None if q is None else _dev(q, device).reshape(n).clone()
        self.m = None if m is None else _dev(m, device).reshape(n).clone()
        self.step = int(step)

    def _bind(self, state):
        self.state = state
        for k, name in enumerate(STATE_NAMES):
            setattr(self, name, state[k, :self.n])

    def to_c(self):
        s = NbSystem()
        s.n = self.n
        for k in STATE_NAMES:
            setattr(s, k, _ptr(getattr(self, k)))
        s.q = _ptr(self.q)
        s.m = _ptr(self.m)
        s.step = self.step
        return s

    def view(self, i0, i1):
        """A System sharing memory with ions [i0, i1) of this one (its
        `state` is the (9, i1 - i0) column slice)."""
        v = System.__new__(System)
        v.n = int(i1 - i0)
        v.state = self.state[:, i0:i1]
        for k in STATE_NAMES:
            setattr(v, k, getattr(self, k)[i0:i1])
        v.q = None if self.q is None else self.q[i0:i1]
        v.m = None if self.m is None else self.m[i0:i1]
        v.step = self.step
        return v

    def state_dict(self):
        """The full Verlet state as CPU tensors (positions, velocities, the
        acceleration of the current state, q, m, step), for torch.save.  A
        system rebuilt from it continues bitwise as the original would: the
        acceleration is part of the state, and the step counter sets the time
        and the Langevin noise stream."""
        d = {k: getattr(self, k).detach().cpu().clone() for k in STATE_NAMES}
        d["q"] = None if self.q is None else self.q.detach().cpu().clone()
        d["m"] = None if self.m is None else self.m.detach().cpu().clone()
        d["step"] = int(self.step)
        return d

    @classmethod
    def from_state(cls, d, device="cuda"):
        """A System holding the state saved by state_dict (copied to `device`)."""
        s = cls.__new__(cls)
        s.n = int(d["x"].numel())
        s._bind(_packed_state(s.n, device))
        for k in STATE_NAMES:
            t = d[k]
            if t.dtype != torch.float64 or t.numel() != s.n:
                raise ValueError("state entry %s must be float64 of length %d" % (k, s.n))
            getattr(s, k).copy_(t.reshape(s.n))
        s.q = None if d.get("q") is None else d["q"].to(device, torch.float64).clone()
        s.m = None if d.get("m") is None else d["m"].to(device, torch.float64).clone()
        s.step = int(d["step"])
        return s

    def pos(self):
        return torch.stack([self.x, self.y, self.z])

    def vel(self):
        return torch.stack([self.vx, self.vy, self.vz])

    def acc(self):
        return torch.stack([self.ax, self.ay, self.az])


CKPT_MAGIC = b"NBCKPT1\n"


def save_checkpoint(path, system, params=None):
    """Write the Verlet state (x, v, a, optional q and m, the step counter) and
    optionally the parameters to `path`, framework-free: the magic line
    NBCKPT1, the byte length of a JSON header as a little-endian uint64, the
    header ({"format", "version", "n", "step", "arrays", "params"}), then
    each array of `arrays` as n little-endian float64.  The step counter sets
    t and the noise stream, so a run resumed from the file continues bit for
    bit (see load_checkpoint)."""
    import dataclasses
    import json
    import struct
    names = list(STATE_NAMES) + [k for k in ("q", "m") if getattr(system, k) is not None]
    header = {"format": "nb-checkpoint", "version": 1, "n": int(system.n), "step": int(system.step),
              "arrays": names, "params": None if params is None else dataclasses.asdict(params)}
    if header["params"] is not None:
        for k in ("omega", "omega_rate"):
            header["params"][k] = [float(v) for v in header["params"][k]]
    hb = json.dumps(header, sort_keys=True).encode()
    with open(path, "wb") as f:
        f.write(CKPT_MAGIC)
        f.write(struct.pack("<Q", len(hb)))
        f.write(hb)
        for k in names:
            a = getattr(system, k).detach().to("cpu", torch.float64).contiguous().numpy()
            f.write(a.astype("<f8", copy=False).tobytes())


def load_checkpoint(path, device="cuda"):
    """Read a file written by save_checkpoint: returns (System on `device`,
    Params or None).  Raises ValueError on a malformed file."""
    import json
    import struct
    with open(path, "rb") as f:
        if f.read(len(CKPT_MAGIC)) != CKPT_MAGIC:
            raise ValueError("not an nb checkpoint")
        (hl,) = struct.unpack("<Q", f.read(8))
        header = json.loads(f.read(hl).decode())
        if header.get("format") != "nb-checkpoint" or header.get("version") != 1:
            raise ValueError("unknown checkpoint format or version")
        n = int(header["n"])
        names = header["arrays"]
        if not set(STATE_NAMES) <= set(names) or not set(names) <= set(STATE_NAMES) | {"q", "m"}:
            raise ValueError("checkpoint arrays %s" % names)
        arrays = {}
        for k in names:
            b = f.read(8 * n)
            if len(b) != 8 * n:
                raise ValueError("checkpoint truncated in array %s" % k)
            arrays[k] = torch.from_numpy(np.frombuffer(b, dtype="<f8").astype(np.float64))
        if f.read(1):
            raise ValueError("trailing bytes after the checkpoint arrays")
    d = {k: arrays[k] for k in STATE_NAMES}
    d["q"], d["m"], d["step"] = arrays.get("q"), arrays.get("m"), header["step"]
    system = System.from_state(d, device=device)
    par = header["params"]
    if par is not None:
        par = Params(**{k: (tuple(v) if k in ("omega", "omega_rate") else v) for k, v in par.items()})
    return system, par


def forces(params, system, total=False, want_phi=False, stream=None):
    """nb_forces: write system.ax/ay/az (Coulomb, or the total Verlet-state
    acceleration when total=True).  Returns phi (device tensor) if asked."""
    phi = torch.empty(system.n, dtype=torch.float64, device=system.x.device) if want_phi else None
    s = system.to_c()
    _check(lib().nb_forces(C.byref(params.to_c()), C.byref(s), _ptr(phi),
                           NB_ACC_TOTAL if total else NB_ACC_COULOMB, _stream(stream)), "nb_forces")
    return phi


def step(params, system, nsteps, stream=None):
    """nb_step: nsteps velocity-Verlet steps in place."""
    s = system.to_c()
    _check(lib().nb_step(C.byref(params.to_c()), C.byref(s), int(nsteps), _stream(stream)),
           "nb_step")
    system.step = s.step


def forces_range(params, system, i0, i1, total=False, stream=None):
    """nb_forces_range: the acceleration of ions [i0, i1) from all n ions,
    written into system.ax/ay/az[i0:i1] only."""
    s = system.to_c()
    _check(lib().nb_forces_range(C.byref(params.to_c()), C.byref(s), int(i0), int(i1),
                                 NB_ACC_TOTAL if total else NB_ACC_COULOMB, _stream(stream)), "nb_forces_range")


def step_range_drift(params, system, i0, i1, stream=None):
    """nb_step_range_drift: the drift half of a Verlet step for ions [i0, i1)."""
    s = system.to_c()
    _check(lib().nb_step_range_drift(C.byref(params.to_c()), C.byref(s), int(i0), int(i1), _stream(stream)),
           "nb_step_range_drift")


def step_range_kick(params, system, i0, i1, stream=None):
    """nb_step_range_kick: forces from all n (drifted) positions and the kick
    of ions [i0, i1); advances system.step by one."""
    s = system.to_c()
    _check(lib().nb_step_range_kick(C.byref(params.to_c()), C.byref(s), int(i0), int(i1), _stream(stream)),
           "nb_step_range_kick")
    system.step = s.step


def energy(params, system, stream=None):
    """nb_energy: (kinetic, trap, Coulomb, total) in J as a numpy array."""
    out = np.empty(4)
    s = system.to_c()
    _check(lib().nb_energy(C.byref(params.to_c()), C.byref(s),
                           out.ctypes.data_as(_dp), _stream(stream)), "nb_energy")
    return out


def forces_vjp(params, system, lam, total=False, stream=None):
    """nb_forces_vjp: J^T lam for lam of shape (3, n); returns (3, n)."""
    lam = _dev(lam, system.x.device).reshape(3, system.n)
    lx, ly, lz = (lam[k].contiguous() for k in range(3))
    g = torch.empty(3, system.n, dtype=torch.float64, device=system.x.device)
    s = system.to_c()
    _check(lib().nb_forces_vjp(C.byref(params.to_c()), C.byref(s), _ptr(lx), _ptr(ly), _ptr(lz),
                               _ptr(g[0]), _ptr(g[1]), _ptr(g[2]),
                               NB_ACC_TOTAL if total else NB_ACC_COULOMB, _stream(stream)),
           "nb_forces_vjp")
    return g


def _offsets(offsets):
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    return off, off.ctypes.data_as(C.POINTER(C.c_int64))


def step_batched(params, system, offsets, nsteps, stream=None):
    """nb_step_batched: every instance [offsets[k], offsets[k+1]) of the packed
    system takes nsteps velocity-Verlet steps (one persistent launch)."""
    off, offp = _offsets(offsets)
    s = system.to_c()
    _check(lib().nb_step_batched(C.byref(params.to_c()), len(off) - 1, offp, C.byref(s),
                                 int(nsteps), _stream(stream)), "nb_step_batched")
    system.step = s.step


def step_batched_each(per_inst, system, offsets, nsteps, stream=None):
    """nb_step_batched_each: as step_batched, with instance k run under
    per_inst[k] (a sequence of Params, one per instance, same precision)."""
    off, offp = _offsets(offsets)
    n_inst = len(off) - 1
    if len(per_inst) != n_inst:
        raise ValueError("per_inst has %d entries for %d instances" % (len(per_inst), n_inst))
    tab = (NbParams * max(n_inst, 1))(*[p.to_c() for p in per_inst])
    s = system.to_c()
    _check(lib().nb_step_batched_each(tab, n_inst, offp, C.byref(s), int(nsteps), _stream(stream)),
           "nb_step_batched_each")
    system.step = s.step


def init_batched(params, system, offsets, stream=None):
    """Set the Verlet-state acceleration of every instance of a packed ensemble
    (nb_forces with NB_ACC_TOTAL on each instance's own ions); `params` is one
    Params for all instances or a sequence of one per instance."""
    off = np.asarray(offsets, dtype=np.int64)
    each = isinstance(params, (list, tuple))
    for k in range(len(off) - 1):
        if off[k + 1] > off[k]:
            forces(params[k] if each else params, system.view(int(off[k]), int(off[k + 1])), total=True,
                   stream=stream)


def plan_batched(offsets, n_bins):
    """nb_plan_batched: (order, bin_start, max_load, mean_load) of the ensemble schedule."""
    off, offp = _offsets(offsets)
    n_inst = len(off) - 1
    order = np.zeros(max(n_inst, 1), dtype=np.uint16)
    start = np.zeros(n_bins + 1, dtype=np.uint16)
    mx, mean = C.c_double(), C.c_double()
    _check(lib().nb_plan_batched(n_inst, offp, int(n_bins),
                                 order.ctypes.data_as(C.POINTER(C.c_uint16)),
                                 start.ctypes.data_as(C.POINTER(C.c_uint16)),
                                 C.byref(mx), C.byref(mean)), "nb_plan_batched")
    return order[:n_inst], start, mx.value, mean.value


PLAN_KINDS = {"force": 0, "potential": 1, "vjp": 2}
PLAN_FIELDS = ("block", "R", "jchunk", "n_it", "n_jc", "symmetric", "G", "single_block")


def sym_wait_probe(committed, round_, stream=None):
    """nb_sym_wait_probe: one bounded wait of the half-pair kernels' output
    order; True if block 0, with `committed` rounds published, reached
    `round_` (a wait that runs out leaves NB_ETIMEOUT for sync_status)."""
    ok = C.c_int32()
    _check(lib().nb_sym_wait_probe(int(committed), int(round_), C.byref(ok), _stream(stream)),
           "nb_sym_wait_probe")
    return bool(ok.value)


def plan_info(kind, precision, n):
    """nb_plan_info: the launch plan a call at n ions would use (host only)."""
    out = (C.c_int64 * 8)()
    _check(lib().nb_plan_info(PLAN_KINDS[kind] if isinstance(kind, str) else int(kind), PRECISIONS[precision],
                              int(n), out), "nb_plan_info")
    return dict(zip(PLAN_FIELDS, (int(v) for v in out)))


KINDS = {"force": 0, "potential": 1, "vjp": 2, "ensemble": 3, "symmetric": 4, "symmetric_vjp": 5,
         "step_windows": 6, "small_steps": 7, "epilogue_lanes": 8}


def set_tuning(kind, precision, n_lo, n_hi, block, R=1, blocks_per_sm=16):
    """nb_set_tuning: launch-shape override (block = 0 clears all)."""
    _check(lib().nb_set_tuning(KINDS[kind] if isinstance(kind, str) else int(kind),
                               PRECISIONS[precision], int(n_lo), int(n_hi), int(block), int(R),
                               int(blocks_per_sm)), "nb_set_tuning")


def rinv3_probe(precision, d, soft2=0.0, stream=None):
    """nb_rinv3_probe: the r^-3 that `precision` forms for each displacement
    column of d (shape (3, n), FP64); returns a device tensor of n doubles."""
    d = torch.as_tensor(d, dtype=torch.float64).reshape(3, -1)
    if d.device.type != "cuda":
        d = d.to("cuda")
    dx, dy, dz = (d[k].contiguous() for k in range(3))
    out = torch.empty(dx.numel(), dtype=torch.float64, device=dx.device)
    _check(lib().nb_rinv3_probe(PRECISIONS[precision], dx.numel(), _ptr(dx), _ptr(dy), _ptr(dz),
                                float(soft2), _ptr(out), _stream(stream)), "nb_rinv3_probe")
    return out


def rsqrt_seed_probe(x, stream=None):
    """nb_rsqrt_seed_probe: the FP32 hardware 1/sqrt seed of each element."""
    x = torch.as_tensor(x, dtype=torch.float32).reshape(-1)
    if x.device.type != "cuda":
        x = x.to("cuda")
    x = x.contiguous()
    y = torch.empty_like(x)
    _check(lib().nb_rsqrt_seed_probe(x.numel(), x.data_ptr(), y.data_ptr(), _stream(stream)),
           "nb_rsqrt_seed_probe")
    return y


PIPE_KINDS = {"dfma": 0, "dadd": 1, "dmul": 2, "ffma": 3, "fadd": 4, "mufu_rsq": 5}
# default rounds (each 4 x 8 instructions per thread, per shape): a few ms per kind
PIPE_ITERS = {"dfma": 1024, "dadd": 1024, "dmul": 1024, "ffma": 16384, "fadd": 16384, "mufu_rsq": 4096}
PIPE_SHAPES = ("4 chains, own operands", "4 chains, shared operands", "8 chains, shared operands")


def pipe_probe(kind, iters=None, stream=None):
    """nb_pipe_probe: measured throughput of one instruction kind on every SM
    (the fastest of three chain shapes).  Returns {"lanes_per_clk_per_sm",
    "sm_mhz", "shape"}."""
    out = (C.c_double * 3)()
    it = PIPE_ITERS[kind] if iters is None else int(iters)
    _check(lib().nb_pipe_probe(PIPE_KINDS[kind], it, out, _stream(stream)), "nb_pipe_probe")
    return {"lanes_per_clk_per_sm": out[0], "sm_mhz": out[1], "shape": PIPE_SHAPES[int(out[2])]}


def sym_schedule(nbk):
    """nb_sym_schedule: (P, Q, round) int32 arrays of the half-pair kernels'
    work items for nbk blocks (host only)."""
    m = nbk * (nbk + 1) // 2
    P, Q, R = (np.empty(m, dtype=np.int32) for _ in range(3))
    i32 = C.POINTER(C.c_int32)
    _check(lib().nb_sym_schedule(int(nbk), P.ctypes.data_as(i32), Q.ctypes.data_as(i32), R.ctypes.data_as(i32)),
           "nb_sym_schedule")
    return P, Q, R


def sync_status(stream=None):
    """nb_sync_status: synchronise and raise on a recorded device error."""
    _check(lib().nb_sync_status(_stream(stream)), "nb_sync_status")


def release():
    _check(lib().nb_release(), "nb_release")
