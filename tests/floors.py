"""Per-ion trajectory tolerance that the force contract itself allows.

The force gate (conditioned error, Eq. 1's pair sum) lets ion i's Coulomb
acceleration be off by up to eps * S_i in every step, S_i = sum_{j != i}
|a_ij| its conditioning sum.  Through the velocity-Verlet update (Sec. II)
that error alone moves the ion's velocity by at most k dt eps S_i and its
position by at most k^2 dt^2 eps S_i after k steps (the sum over steps of
dt (s dt eps S_i) plus dt^2/2 eps S_i per step).  S_i is taken as the larger
of its values at the first and the last state of the run.  How the dynamics
amplify errors is measured separately, by the oracle's own one-ulp
divergence."""
import numpy as np


def contract_floor(orc, p, states, nsteps, dt, eps=1e-12, q=None):
    """(position floor, velocity floor), each an array of n, for a run of
    nsteps steps of dt; `states` are (3, n) position arrays along the run."""
    S = None
    for pos in states:
        absf = orc.coulomb(p, *np.asarray(pos), q=q, want_absf=True)[4]
        S = absf if S is None else np.maximum(S, absf)
    k = float(nsteps)
    return k * k * dt * dt * eps * S, k * dt * eps * S


def per_ion(d):
    """Largest component of a (3, n) difference, per ion."""
    return np.max(np.abs(np.asarray(d)), axis=0)
