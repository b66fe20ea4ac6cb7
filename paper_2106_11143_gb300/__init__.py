"""GB300-native direct N-body library for trapped-ion Coulomb crystals.

All-pairs Coulomb acceleration, trap force and velocity-Verlet integration
of Pedregosa-Gutierrez & Dempsey, "Direct N-Body problem optimisation using
the AVX-512 instruction set" (arXiv 2106.11143), re-designed for sm_103a.
The compute lives in hand-written CUDA kernels behind the C ABI declared in
include/nb.h (libnb.so); this package is a thin ctypes binding over it plus
seeded workload generators.  There is no CPU fallback: calling into the
library without the built extension raises.
"""
from . import workloads  # noqa: F401  (pure numpy, no compute of the method)

_API = ("Params", "System", "forces", "step", "energy", "forces_vjp", "sync_status",
        "step_batched", "step_batched_each", "init_batched", "plan_batched", "set_tuning",
        "trajectory_loss", "TrajectoryLoss", "lib", "NBError", "PRECISIONS", "release", "rinv3_probe", "rsqrt_seed_probe", "save_checkpoint",
        "load_checkpoint", "plan_info", "pipe_probe", "sym_schedule", "forces_range", "step_range_drift",
        "step_range_kick", "sym_wait_probe")


def __getattr__(name):
    if name in ("trajectory_loss", "TrajectoryLoss"):
        from . import autograd
        return getattr(autograd, name)
    if name in _API:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
