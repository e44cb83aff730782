"""FP64 CPU oracle for one TreePM kick-drift-kick step.

TEST INFRASTRUCTURE ONLY: the slow, obviously-correct reference that the
device-resident step is compared against.  Only the tests use it; the
product path never calls it.

The paper's step (Sec. 2.1) drifts all particles at the start of the step.
It then computes the gravity (short-range tree walk on the device,
long-range PM on the host, Sec. 3.1) and kicks with it.  The integrator is
GADGET's second-order leapfrog in kick-drift-kick form, written out with G = 1:

    v <- v + (dt / 2) a(x)        (half kick with the previous accelerations)
    x <- x + dt v                 (drift of every particle)
    a <- a_short(x) + a_long(x)   (keys, tree and walk rebuilt; the PM mesh)
    v <- v + (dt / 2) a(x)        (half kick)

The short-range part is the oracle's periodic direct sum (no tree, so the
result does not depend on an opening angle).  The long-range part is the PM
oracle (og_pm).  Positions are not wrapped in the drift: every force
routine wraps them itself.

Parity status (pins in tests/test_oracle_kdk.py): pinned by time
reversibility, momentum conservation and the period of a tight binary
(Kepler's law).
"""
from __future__ import annotations

import numpy as np

from . import direct
from . import og_pm


def accel(pos, mass, h, box, r_s, rcut, ngrid):
    """a_short + a_long [n, 3] at the positions pos (original order)."""
    a_s, _ = direct(pos, mass, h, box, r_s, rcut)
    return a_s + og_pm.pm_accel(pos, mass, box, ngrid, r_s)


def kdk(pos, vel, acc, mass, h, box, r_s, rcut, ngrid, dt, nsteps=1):
    """nsteps kick-drift-kick steps; returns (pos, vel, acc) after them."""
    pos = np.array(pos, dtype=np.float64)
    vel = np.array(vel, dtype=np.float64)
    acc = np.array(acc, dtype=np.float64)
    for _ in range(nsteps):
        vel = vel + (0.5 * dt) * acc
        pos = pos + dt * vel
        acc = accel(pos, mass, h, box, r_s, rcut, ngrid)
        vel = vel + (0.5 * dt) * acc
    return pos, vel, acc
