"""Pin of the oracle's FDTD comparator (textbook Yee with PEC walls)."""
import math

import numpy as np

import oracle
from oracle import fdtd

EZ = 2
C0 = 299792458.0


def test_yee_pec_box_eigenmode_recurrence():
    """The discrete mode Ez = sin(pi i/nx) sin(pi j/ny) (uniform in z) of a PEC box obeys
    E^{n+1} + E^{n-1} = (2 - c^2 dt^2 kappa) E^n at every Yee node, with the closed-form
    Yee eigenvalue kappa = sum_a 4 sin^2(k_a h_a / 2) / h_a^2, k = (pi/a, pi/b, 0)."""
    n, h = (12, 9, 5), (1e-2, 1.3e-2, 0.7e-2)
    dt = oracle.dt_cfl(0.9, *h)
    y = fdtd.Yee(n, h, dt)
    nx, ny, nz = n
    i = np.arange(nx + 1)
    j = np.arange(ny + 1)
    mode = np.outer(np.sin(math.pi * j / ny), np.sin(math.pi * i / nx))
    y.F[EZ][1:nz + 1] = mode[None, :, :]
    e0 = y.F[EZ].copy()
    y.step(1)
    e1 = y.F[EZ].copy()
    y.step(1)
    e2 = y.F[EZ].copy()
    kappa = 4 * math.sin(math.pi / (2 * nx)) ** 2 / h[0] ** 2 + 4 * math.sin(math.pi / (2 * ny)) ** 2 / h[1] ** 2
    lhs = (e2 + e0)[1:nz + 1, 1:ny, 1:nx]
    rhs = ((2 - (C0 * dt) ** 2 * kappa) * e1)[1:nz + 1, 1:ny, 1:nx]
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(e1))
    for c in (0, 1):
        assert not np.any(y.F[c])
