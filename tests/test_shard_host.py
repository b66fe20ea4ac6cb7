"""The i-range sharding driver (paper_2106_11143_gb300/shard.py) on CPU ranks:
the partition of the ions over ranks, and the step's exchange on two and
three gloo ranks.  The library's range kernels need a GPU, so here each rank
advances its own ions with host stand-ins built on the oracle (the same
velocity-Verlet update, Sec. II); the sharded run must reproduce the
oracle's unsharded run on every rank."""
import math
import os
import socket
import sys
from types import SimpleNamespace

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_partition_is_contiguous_and_balanced():
    from paper_2106_11143_gb300.shard import partition
    for n in (0, 1, 2, 7, 100, 100001):
        for world in (1, 2, 3, 8):
            r = partition(n, world)
            assert len(r) == world and r[0][0] == 0 and r[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            sizes = [b - a for a, b in r]
            assert max(sizes) - min(sizes) <= 1 and sum(sizes) == n
    with pytest.raises(ValueError):
        partition(5, 0)


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleRangeKernels:
    """Host stand-ins for the range calls: the oracle's acceleration (all
    ions, then the owned slice) and the Verlet drift and kick of or_run
    (gamma = 0, no noise) on the owned ions only."""

    def __init__(self, orc, p, dt):
        self.orc, self.p, self.dt = orc, p, dt

    def _acc(self, s, t):
        a = self.orc.accel(self.p, t, s.x.numpy(), s.y.numpy(), s.z.numpy())
        return [torch.from_numpy(np.asarray(c)) for c in a]

    def forces(self, params, s, i0, i1):
        a = self._acc(s, self.p.t0 + s.step * self.dt)
        for k, nm in enumerate(("ax", "ay", "az")):
            getattr(s, nm)[i0:i1] = a[k][i0:i1]

    def drift(self, params, s, i0, i1):
        dt = self.dt
        for c, v, a in (("x", "vx", "ax"), ("y", "vy", "ay"), ("z", "vz", "az")):
            r = getattr(s, c)
            r[i0:i1] = r[i0:i1] + getattr(s, v)[i0:i1] * dt + 0.5 * dt * dt * getattr(s, a)[i0:i1]

    def kick(self, params, s, i0, i1):
        dt = self.dt
        an = self._acc(s, self.p.t0 + (s.step + 1) * dt)
        for k, (v, a) in enumerate((("vx", "ax"), ("vy", "ay"), ("vz", "az"))):
            vv, aa = getattr(s, v), getattr(s, a)
            vv[i0:i1] = vv[i0:i1] + 0.5 * dt * (aa[i0:i1] + an[k][i0:i1])
            aa[i0:i1] = an[k][i0:i1]
        s.step += 1


def _case():
    from paper_2106_11143_gb300 import workloads as W
    rng = np.random.default_rng(17)
    n = 37
    a, c = W.cold_fluid_spheroid(n, 2 * math.pi * 1e6, 2 * math.pi * 200e3)
    pos = W.ellipsoid_uniform(n, (a, a, c), rng)
    vel = W.thermal_velocities(n, 1e-3, W.MASS_40U, rng)
    phys = W.phys(omega=(2 * math.pi * 1e6, 2 * math.pi * 0.9e6, 2 * math.pi * 200e3), dt=2e-9)
    return pos, vel, phys


def _rank_main(rank, world, port, nsteps, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import oracle
    from paper_2106_11143_gb300.shard import ShardedSystem
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    pos, vel, phys = _case()
    p = oracle.make_params(**phys)
    z = torch.zeros(pos.shape[1], dtype=torch.float64)
    s = SimpleNamespace(n=pos.shape[1], step=0, **{nm: torch.tensor(pos[k]) for k, nm in enumerate("xyz")},
                        **{nm: torch.tensor(vel[k]) for k, nm in enumerate(("vx", "vy", "vz"))},
                        ax=z.clone(), ay=z.clone(), az=z.clone())
    sh = ShardedSystem(None, s, kernels=OracleRangeKernels(oracle, p, phys["dt"]))
    sh.init_forces()
    # before the first step only the owned accelerations are set: others are 0
    own = np.zeros(s.n, dtype=bool)
    own[sh.i0:sh.i1] = True
    assert np.all(s.ax.numpy()[~own] == 0.0)
    sh.step(nsteps)
    sh.gather_state()
    np.save(os.path.join(out_dir, "rank%d.npy" % rank),
            np.stack([getattr(s, nm).numpy() for nm in ("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az")]))
    with open(os.path.join(out_dir, "rank%d.step" % rank), "w") as f:
        f.write("%d %d %d" % (s.step, sh.i0, sh.i1))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_steps_match_unsharded_oracle(tmp_path, orc, world):
    nsteps = 60
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, nsteps, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    pos, vel, phys = _case()
    p = orc.make_params(**phys)
    ax, ay, az = orc.accel(p, 0.0, *pos)
    st = dict(x=pos[0], y=pos[1], z=pos[2], vx=vel[0], vy=vel[1], vz=vel[2], ax=ax, ay=ay, az=az, step=0)
    ref = orc.run(p, st, nsteps)
    R = np.stack([ref[k] for k in ("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az")])
    scale = np.max(np.abs(R), axis=1, keepdims=True)
    ranges = []
    for r in range(world):
        got = np.load(tmp_path / ("rank%d.npy" % r))
        step, i0, i1 = map(int, open(tmp_path / ("rank%d.step" % r)).read().split())
        ranges.append((i0, i1))
        assert step == nsteps
        # every rank ends with the whole state, equal to the unsharded run
        assert np.all(np.abs(got - R) <= 1e-13 * scale), (r, float(np.max(np.abs(got - R) / scale)))
    assert ranges[0][0] == 0 and ranges[-1][1] == pos.shape[1]
    assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
