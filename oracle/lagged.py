"""The coupling step with the source delayed by eps_R, FP64.

TEST INFRASTRUCTURE: only the test suite uses this module.  Eq.
ns_regularized_filtered forces the fluid at time t with the particle force
D(t - eps_R), spread with width sigma_R around the position x(t - eps_R).
With L = round(eps_R / dt) >= 1 steps the source of step n is D^(n-L) at
x^(n-L); the first L steps have none.  The self disturbance the particle
removes at step n is the one the previous step's source left (App. A.5):
that of D^(n-1-L) at x^(n-1-L), seen at x^n, at the matching gather's
variance 2 nu (eps_R + dt) + sigma_R^2; none while n < L + 1.

``History`` holds (x^k, D^k) of the steps since the last first step; the
step is written with the oracle's own gather, closed-form disturbance,
advance and scatter.
"""

from __future__ import annotations

import numpy as np

from . import Params, _params, advance, gather, scatter, self_velocity


def lag_steps(p):
    """L = round(eps_R / dt), at least 1 (half-way rounds away from zero)."""
    p = _params(p)
    q = p.eps_R / p.dt
    return max(1, int(np.floor(q + 0.5)))


class History:
    def __init__(self):
        self.x = []
        self.D = []


def _min_image(r, p):
    for a in range(3):
        La = p.L[a]
        r[a] = np.where(r[a] > 0.5 * La, r[a] - La, np.where(r[a] < -0.5 * La, r[a] + La, r[a]))
    return r


def step(p, u, state, hist, first_step=False):
    """One step in place; returns the source S.  ``hist`` is updated."""
    p = _params(p)
    L = lag_steps(p)
    if first_step:
        hist.x.clear()
        hist.D.clear()
    n = len(hist.x)
    up = gather(p, state.x, u)
    if p.self_removal and n >= L + 1:
        r = _min_image(state.x - hist.x[n - 1 - L], p)
        up = up - self_velocity(p, r, hist.D[n - 1 - L])
    q = Params.from_buffer_copy(p)
    q.self_removal = 0
    advance(q, up, state)
    if n >= L:
        S = scatter(p, hist.x[n - L], hist.D[n - L])
    else:
        S = np.zeros((3, int(p.n[2]), int(p.n[1]), int(p.n[0])))
    hist.x.append(state.x_prev.copy())
    hist.D.append(state.D.copy())
    return S
