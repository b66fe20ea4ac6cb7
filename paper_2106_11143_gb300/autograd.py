"""torch.autograd binding of the trajectory adjoint (nb_traj_forward /
nb_traj_backward in include/nb.h).

TrajectoryLoss.apply(x0, v0, omega, params, nsteps, every, target) returns
the scalar loss  E_coulomb(x_T) + E_trap(x_T) + sum |x_T - target|^2  of an
nsteps velocity-Verlet trajectory (Sec. II) started at (x0, v0) in the
harmonic trap with angular frequencies omega, and back-propagates exact
gradients to x0 (3, n), v0 (3, n) and omega (3,) through the CUDA adjoint
kernels.  Argument marshalling only: the forward, the checkpointing, the
recompute and the reverse sweep all run in libnb.so.
"""
import ctypes as C
import dataclasses

import torch

from . import api


def _p(t):
    return api._ptr(t)


class TrajectoryLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, v0, omega, params, nsteps, every, target):
        dev = x0.device
        x0 = x0.detach().to(torch.float64).contiguous()
        v0 = v0.detach().to(torch.float64).contiguous()
        target = target.detach().to(device=dev, dtype=torch.float64).contiguous()
        n = x0.shape[1]
        # the force arithmetic of the forward and its recompute: df64 if asked, else fp64
        prec = "df64" if params.precision == "df64" else "fp64"
        par = dataclasses.replace(params, omega=tuple(float(w) for w in omega.detach().cpu().tolist()),
                                  precision=prec)
        sysm = api.System(x0, v0)
        L = api.lib()
        nck = L.nb_traj_ckpt_doubles(n, int(nsteps), int(every))
        if nck < 0:
            raise ValueError("invalid nsteps/every")
        ckpt = torch.empty(nck, dtype=torch.float64, device=dev)
        loss = torch.empty(1, dtype=torch.float64, device=dev)
        s = sysm.to_c()
        api._check(L.nb_traj_forward(C.byref(par.to_c()), C.byref(s), int(nsteps), int(every), _p(ckpt),
                                     _p(target), _p(loss), api._stream(None)), "nb_traj_forward")
        ctx.par, ctx.nsteps, ctx.every, ctx.n, ctx.q = par, int(nsteps), int(every), n, sysm.q
        ctx.save_for_backward(ckpt, target)
        ctx.final = sysm
        return loss[0]

    @staticmethod
    def backward(ctx, gout):
        ckpt, target = ctx.saved_tensors
        dev = ckpt.device
        n = ctx.n
        gs = gout.detach().to(device=dev, dtype=torch.float64).reshape(1).contiguous()
        gx = torch.empty(3, n, dtype=torch.float64, device=dev)
        gv = torch.empty(3, n, dtype=torch.float64, device=dev)
        gw = torch.empty(3, dtype=torch.float64, device=dev)
        s = api.NbSystem()
        s.n = n
        s.q = _p(ctx.q)
        L = api.lib()
        api._check(L.nb_traj_backward(C.byref(ctx.par.to_c()), C.byref(s), ctx.nsteps, ctx.every, _p(ckpt),
                                      _p(target), _p(gs), _p(gx), _p(gv), _p(gw), api._stream(None)),
                   "nb_traj_backward")
        return gx, gv, gw, None, None, None, None


def trajectory_loss(x0, v0, omega, params, nsteps, every, target):
    """Scalar loss tensor with gradients to x0, v0 and omega (see module doc)."""
    return TrajectoryLoss.apply(x0, v0, omega, params, nsteps, every, target)


def trajectory_final_state(loss_tensor):
    """The System holding x_T, v_T, a_T of the forward that produced loss_tensor."""
    return loss_tensor.grad_fn.final if loss_tensor.grad_fn is not None else None
