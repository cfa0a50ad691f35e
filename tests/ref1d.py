"""A 1D SBP-SAT leapfrog for one tangential pair, written with dense matrices.

It is the special case the 3D scheme reduces to for fields that are uniform in
x and y inside a guide with PEC x-faces and PMC y-faces: the pair (Ex, Hy)
along z (curl sign s = -1 in Eqs. (7)-(12)).  The operators come from the
printed Appendix matrices (tests/appendix.py), not from the oracle.
"""
import math

import numpy as np

from tests import appendix

EPS0 = 8.8541878128e-12
MU0 = 1.25663706212e-6
PEC, PMC, ABSORBING = 0, 1, 2


def gauss(t, tw, t0):
    return math.exp(-4.0 * math.pi * (t - t0) ** 2 / tw ** 2)


class Pair1D:
    """Ex on z+ (n+1 nodes), Hy on z- (n+2 nodes), eps_r per cell (n values)."""

    def __init__(self, n, h, dt, face_lo, face_hi, eps_cells=None):
        self.n, self.h, self.dt = n, h, dt
        e = np.ones(n) if eps_cells is None else np.asarray(eps_cells, float)
        # node means over the cells whose closed interval contains the node
        self.eps_e = np.array([e[max(i - 1, 0):min(i + 1, n)].mean() for i in range(n + 1)])
        self.eps_h = np.concatenate([[e[0]], e, [e[-1]]])
        Pp = h * appendix.p_plus(n)
        Pm = h * appendix.p_minus(n)
        Dp = np.linalg.solve(np.diag(Pp), appendix.q_plus(n)) / 1.0
        Dm = np.linalg.solve(np.diag(Pm), appendix.q_minus(n)) / 1.0
        s = -1.0
        AE = s * Dp.copy()            # dEx/dt part: s D+ Hy
        AH = s * Dm.copy()            # dHy/dt part: s D- Ex
        gE = np.zeros(n + 1)
        gH = np.zeros(n + 2)
        for side, ftype in ((-1, face_lo), (+1, face_hi)):
            phi = -s * side
            ie = 0 if side < 0 else n         # Ex end node
            ih = 0 if side < 0 else n + 1     # Hy end node
            if ftype == PEC:
                AH[ih, ie] += phi / Pm[ih]
            elif ftype == PMC:
                AE[ie, ih] += phi / Pp[ie]
            elif ftype == ABSORBING:
                eta_e = math.sqrt(MU0 / (EPS0 * self.eps_e[ie]))
                AE[ie, ih] += 0.5 * phi / Pp[ie]
                gE[ie] += 0.5 / eta_e / Pp[ie]
                AH[ih, ie] += 0.5 * phi / Pm[ih]
                gH[ih] += 0.5 * eta_e / Pm[ih]
        self.AE = AE / (EPS0 * self.eps_e[:, None])
        self.AH = AH / MU0
        self.gE = gE / (EPS0 * self.eps_e)
        self.gH = gH / MU0
        self.E = np.zeros(n + 1)
        self.H = np.zeros(n + 2)
        self.step_index = 0
        self.sources = []

    def add_sheet(self, k, amp, tw, t0):
        self.sources.append((k, amp, tw, t0))

    def step(self, nsteps, probe_e=None):
        dt = self.dt
        out = []
        for _ in range(nsteps):
            self.H = ((1 - 0.5 * dt * self.gH) * self.H + dt * (self.AH @ self.E)) / (1 + 0.5 * dt * self.gH)
            L = self.AE @ self.H
            t = (self.step_index + 0.5) * dt
            for k, amp, tw, t0 in self.sources:
                L[k] -= amp * gauss(t, tw, t0) / (EPS0 * self.eps_e[k])
            self.E = ((1 - 0.5 * dt * self.gE) * self.E + dt * L) / (1 + 0.5 * dt * self.gE)
            self.step_index += 1
            if probe_e is not None:
                out.append(self.E[probe_e])
        return np.array(out)


class PeriodicPair1D:
    """The pair (Ex, Hy) along z with the phase-shifted periodic SAT of Eqs. (EPBC2),
    (EPBC4) and the coefficients of Eq. (EPBCP), complex, dense (printed matrices).
    The field one period up equals e^{-j alpha} times the field here."""

    def __init__(self, n, h, dt, alpha):
        self.n, self.h, self.dt = n, h, dt
        Pp = h * appendix.p_plus(n)
        Pm = h * appendix.p_minus(n)
        Dp = np.linalg.solve(np.diag(Pp), appendix.q_plus(n))
        Dm = np.linalg.solve(np.diag(Pm), appendix.q_minus(n))
        s = -1.0
        AE = (s * Dp).astype(complex)
        AH = (s * Dm).astype(complex)
        ph_hi = np.exp(-1j * alpha)      # high face compares with e^{-j alpha} x low face
        ph_lo = np.exp(+1j * alpha)      # low face compares with e^{+j alpha} x high face
        for side in (-1, +1):
            coef = 0.5 * (-s * side)     # sigma / chi of Eq. (EPBCP) for this pair and face
            ie, ih = (0, 0) if side < 0 else (n, n + 1)
            je, jh = (n, n + 1) if side < 0 else (0, 0)
            ph = ph_lo if side < 0 else ph_hi
            AE[ie, ih] += coef / Pp[ie]
            AE[ie, jh] -= coef * ph / Pp[ie]
            AH[ih, ie] += coef / Pm[ih]
            AH[ih, je] -= coef * ph / Pm[ih]
        self.AE = AE / EPS0
        self.AH = AH / MU0
        self.E = np.zeros(n + 1, complex)
        self.H = np.zeros(n + 2, complex)

    def step(self, nsteps):
        for _ in range(nsteps):
            self.H = self.H + self.dt * (self.AH @ self.E)
            self.E = self.E + self.dt * (self.AE @ self.H)
