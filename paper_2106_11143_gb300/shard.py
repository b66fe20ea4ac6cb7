"""i-range sharding of the velocity-Verlet step over several GPUs.

The paper gives each worker a fixed set of target ions (Sec. VI.C, static
OpenMP ownership).  Across GPUs the same partition applies: rank r owns the
contiguous ions [i0, i1) of `partition(n, world)` and keeps the whole system
on its own device, but advances only its own ions.  One step (Sec. II) is

  1. drift of the owned ions            nb_step_range_drift
  2. all-gather of the owned positions  (the step's only exchange:
                                         3 (i1 - i0) doubles per rank)
  3. forces on the owned ions from all
     n positions at t + dt, and their kick nb_step_range_kick

so every rank ends the step with all n positions and the velocities and
accelerations of its own ions.  The pair sums come from the one-sided kernel
with the chunks of the full one-sided plan, so a sharded run reproduces a
single-GPU run of the one-sided kernel bit for bit, whatever the number of
ranks.  The collective is torch.distributed's all_gather (NCCL between GPUs,
gloo on the host); nothing multicasts and no kernel reads another GPU's
memory.

Argument marshalling and the exchange only: the drift, forces and kick run
in libnb.so (the `kernels` argument lets host-side tests of the partition
and the exchange supply their own).
"""
import torch


def partition(n, world):
    """Contiguous, balanced ranges [(i0, i1)] of n ions over `world` ranks:
    the first n mod world ranges hold one ion more."""
    if n < 0 or world < 1:
        raise ValueError("need n >= 0 and world >= 1")
    base, extra = divmod(n, world)
    out, i0 = [], 0
    for r in range(world):
        i1 = i0 + base + (1 if r < extra else 0)
        out.append((i0, i1))
        i0 = i1
    return out


class LibraryKernels:
    """The range calls of libnb.so."""

    def __init__(self):
        from . import api
        self.api = api

    def forces(self, params, system, i0, i1):
        self.api.forces_range(params, system, i0, i1, total=True)

    def drift(self, params, system, i0, i1):
        self.api.step_range_drift(params, system, i0, i1)

    def kick(self, params, system, i0, i1):
        self.api.step_range_kick(params, system, i0, i1)


class ShardedSystem:
    """One rank's share of a sharded system.  `system` holds the full state
    on this rank's device (the same initial state on every rank); `group` is
    a torch.distributed process group (None: the default group, or a single
    rank when torch.distributed is not initialised)."""

    def __init__(self, params, system, group=None, kernels=None):
        import torch.distributed as dist
        self.dist = dist if dist.is_available() and dist.is_initialized() else None
        self.group = group
        self.world = self.dist.get_world_size(group) if self.dist else 1
        self.rank = self.dist.get_rank(group) if self.dist else 0
        self.params = params
        self.system = system
        self.kernels = kernels or LibraryKernels()
        self.ranges = partition(system.n, self.world)
        self.i0, self.i1 = self.ranges[self.rank]
        self.m = max(b - a for a, b in self.ranges)
        dev = system.x.device
        self._send = torch.zeros(3, self.m, dtype=torch.float64, device=dev)
        self._recv = [torch.zeros(3, self.m, dtype=torch.float64, device=dev) for _ in range(self.world)]

    def _gather(self, names):
        """Every rank's owned entries of the named state arrays to all ranks
        (one all-gather of 3 m doubles, m the largest range)."""
        if self.world == 1:
            return
        a, b = self.i0, self.i1
        for k, nm in enumerate(names):
            self._send[k, :b - a].copy_(getattr(self.system, nm)[a:b])
        self.dist.all_gather(self._recv, self._send, group=self.group)
        for r, (ra, rb) in enumerate(self.ranges):
            if r == self.rank:
                continue
            for k, nm in enumerate(names):
                getattr(self.system, nm)[ra:rb].copy_(self._recv[r][k, :rb - ra])

    def init_forces(self):
        """The total acceleration of the owned ions at the current state (the
        Verlet state nb_step expects on entry)."""
        self.kernels.forces(self.params, self.system, self.i0, self.i1)

    def step(self, nsteps=1):
        for _ in range(int(nsteps)):
            self.kernels.drift(self.params, self.system, self.i0, self.i1)
            self._gather(("x", "y", "z"))
            self.kernels.kick(self.params, self.system, self.i0, self.i1)

    def gather_state(self):
        """Velocities and accelerations of all ions on every rank (positions
        are already everywhere after each step), e.g. before a checkpoint."""
        self._gather(("vx", "vy", "vz"))
        self._gather(("ax", "ay", "az"))
