"""FP64 CPU oracle of one round of batch rounding (Alg. 1) with a device projection stand-in.

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the library's product path.

The paper projects each device's relaxed binaries with a per-device MILP (Proj. bin_proj) that keeps
the device's variables closest to the relaxed solution; Gurobi is not available, so the stand-in
projects each (period, device) pair on its own: the on-status u is 0 or 1, and the device's p, q, r
move to the nearest point of the limits that u implies,

    u = 1:  pmin <= p <= pmax,  r >= 0 (0 for consumers),  p + r <= pmax,  qmin <= q <= qmax
    u = 0:  p = q = r = 0,

with the choice of u that is nearer (Euclidean distance over (p, q, r, u); ties to u = 1).  Ramp limits
couple periods and are left to the penalized objective.  Alg. 1 then fixes the unfixed pairs whose
projection moved them least (ties by pair index), a fraction of the unfixed pairs per round.
"""
from __future__ import annotations

import numpy as np

from .qg_oracle import device_sign, unpack, unpack_u


def project_on(p0, r0, pmin, pmax, rcap):
    """Euclidean projection of (p0, r0) onto {pmin <= p <= pmax, 0 <= r <= rcap, p + r <= pmax}
    (rcap = pmax for producers, 0 for consumers): the box projection when it meets p + r <= pmax,
    else the nearest point of the segment p + r = pmax inside the box."""
    p = np.clip(p0, pmin, pmax)
    r = np.clip(r0, 0.0, rcap)
    over = p + r > pmax
    # on the line p + r = pmax: minimize (p - p0)^2 + (pmax - p - r0)^2 over p, then keep r in [0, rcap]
    pl = 0.5 * (p0 + pmax - r0)
    pl = np.clip(pl, np.maximum(pmin, pmax - rcap), pmax)
    return np.where(over, pl, p), np.where(over, pmax - pl, r)


def project_binaries(case, x):
    """(u*, p*, q*, r*, dist), each (T, G): the stand-in projection of every (period, device) pair at
    x and the squared distance it moves (p, q, r, u)."""
    _, _, p, q, r = unpack(case, x)[:5]
    u = unpack_u(case, x)
    rcap = np.where(device_sign(case) < 0, 0.0, case.pmax)
    p1, r1 = project_on(p, r, case.pmin, case.pmax, rcap)
    q1 = np.clip(q, case.qmin, case.qmax)
    d1 = (p - p1) ** 2 + (q - q1) ** 2 + (r - r1) ** 2 + (u - 1.0) ** 2
    d0 = p * p + q * q + r * r + u * u
    on = d1 <= d0
    z = np.zeros_like(p)
    return (on.astype(np.float64), np.where(on, p1, z), np.where(on, q1, z), np.where(on, r1, z),
            np.where(on, d1, d0))


def select(dist, fixed, frac):
    """Flat (period-major) indices of the ceil(frac * unfixed) unfixed pairs with the smallest
    distance, ties broken by the lower index."""
    d = np.asarray(dist).ravel()
    free = np.flatnonzero(~np.asarray(fixed, bool).ravel())
    n = min(len(free), int(np.ceil(frac * len(free))))
    order = np.lexsort((free, d[free]))
    return np.sort(free[order[:n]])
