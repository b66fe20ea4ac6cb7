"""Per-ion trajectory tolerance that the force contract itself allows.

The force gate (conditioned error, Eq. 1's pair sum) lets ion i's Coulomb
acceleration be off by up to eps * S_i in every step, S_i = sum_{j != i}
|a_ij| its conditioning sum.  Through the velocity-Verlet update (Sec. II)
that error alone moves the ion's velocity by at most k dt eps S_i and its
position by at most k^2 dt^2 eps S_i after k steps (the sum over steps of
dt (s dt eps S_i) plus dt^2/2 eps S_i per step).  On top of that each step
rounds the ion's own drift and kick differently on the two sides (the GPU
contracts multiply-adds into FMAs, the oracle does not): about two ulp of
the ion's position and velocity per step, k 2^-51 |x_i| and k 2^-51 |v_i|.
S_i, |x_i| and |v_i| are the larger of their values at the first and the
last state of the run.  How the dynamics amplify errors is measured
separately, by the oracle's own one-ulp divergence."""
import numpy as np


def contract_floor(orc, p, states, nsteps, dt, vels=None, eps=1e-12, q=None):
    """(position floor, velocity floor), each an array of n, for a run of
    nsteps steps of dt; `states` are (3, n) position arrays along the run,
    `vels` the (3, n) velocity arrays of the same states."""
    S = None
    X = None
    for pos in states:
        pos = np.asarray(pos)
        absf = orc.coulomb(p, *pos, q=q, want_absf=True)[4]
        S = absf if S is None else np.maximum(S, absf)
        ax = np.max(np.abs(pos), axis=0)
        X = ax if X is None else np.maximum(X, ax)
    V = np.zeros_like(X)
    for v in vels or ():
        V = np.maximum(V, np.max(np.abs(np.asarray(v)), axis=0))
    k = float(nsteps)
    ulp2 = 2.0 ** -51
    return k * k * dt * dt * eps * S + k * ulp2 * X, k * dt * eps * S + k * ulp2 * V


def per_ion(d):
    """Largest component of a (3, n) difference, per ion."""
    return np.max(np.abs(np.asarray(d)), axis=0)
