"""The FDTD comparator on the oracle side: the textbook Yee scheme with strong PEC walls.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: it checks the GPU comparator
mode.  Fields use the natural extents of the SBP grid (Table I); the Yee scheme lives on
the subset of those nodes it has: along a component's minus-grid axes the half nodes
1..n (the SBP boundary nodes 0 and n+1 are not part of it), along its plus-grid axes the
nodes 0..n, of which E updates only the interior 1..n-1 (tangential E on a PEC wall
stays zero).  Every difference is the two-point one; E nodes carry the node eps_r of the
SBP scheme (mean over the cells whose closed box contains the node); mu is mu0.

    H^{n+1/2} = H^{n-1/2} + dt/mu0 (curl E^n)
    E^{n+1}   = E^n + dt/(eps0 eps_r) (curl H^{n+1/2} - J(t^{n+1/2}))
"""
import numpy as np

from . import Block, waveform

EPS0 = 8.8541878128e-12
MU0 = 1.25663706212e-6


def _d(F, axis, lo, hi):
    """F[.., r, ..] - F[.., r-1, ..] for r in lo..hi along array axis `axis`."""
    a = [slice(None)] * 3
    b = [slice(None)] * 3
    a[axis] = slice(lo, hi + 1)
    b[axis] = slice(lo - 1, hi)
    return F[tuple(a)] - F[tuple(b)]


class Yee:
    """n = (nx, ny, nz) cells, h = (hx, hy, hz); arrays (ext_z, ext_y, ext_x)."""

    def __init__(self, n, h, dt, eps_r=None):
        self.n, self.h, self.dt = tuple(n), tuple(h), dt
        ref = Block(n, h, dt, (0,) * 6, eps_r=eps_r)       # node eps of the SBP grid
        self.F = [np.zeros(ref.shape(c)) for c in range(6)]
        self.eps = [ref.node_eps(c) for c in range(3)]
        self.sources = []
        self.step_index = 0

    def add_source(self, comp, i, j, k, kind, amp, tw, t0, f=0.0):
        self.sources.append((comp, i, j, k, kind, amp, tw, t0, f))

    def step(self, nsteps, probes=()):
        nx, ny, nz = self.n
        hx, hy, hz = self.h
        dt = self.dt
        out = []
        for _ in range(nsteps):
            Ex, Ey, Ez, Hx, Hy, Hz = self.F
            # H on its half nodes (array axes: 0 = z, 1 = y, 2 = x)
            Hx[1:nz + 1, 1:ny + 1, :] += dt / MU0 * (_d(Ey, 0, 1, nz)[:, 1:ny + 1, :] / hz
                                                    - _d(Ez, 1, 1, ny)[1:nz + 1, :, :] / hy)
            Hy[1:nz + 1, :, 1:nx + 1] += dt / MU0 * (_d(Ez, 2, 1, nx)[1:nz + 1, :, :] / hx
                                                    - _d(Ex, 0, 1, nz)[:, :, 1:nx + 1] / hz)
            Hz[:, 1:ny + 1, 1:nx + 1] += dt / MU0 * (_d(Ex, 1, 1, ny)[:, :, 1:nx + 1] / hy
                                                    - _d(Ey, 2, 1, nx)[:, 1:ny + 1, :] / hx)
            # E on its interior Yee nodes: D+ row r is v_{r+1} - v_r = _d(v, axis, r+1)
            t = (self.step_index + 0.5) * dt
            J = [np.zeros_like(Ex), np.zeros_like(Ey), np.zeros_like(Ez)]
            for comp, i, j, k, kind, amp, tw, t0, f in self.sources:
                sel = tuple(slice(None) if v < 0 else v for v in (k, j, i))
                J[comp][sel] += amp * waveform(kind, t, tw, t0, f)
            cx = (_d(Hz, 1, 2, ny)[1:nz, :, 1:nx + 1] / hy - _d(Hy, 0, 2, nz)[:, 1:ny, 1:nx + 1] / hz
                  - J[0][1:nz, 1:ny, 1:nx + 1])
            Ex[1:nz, 1:ny, 1:nx + 1] += dt / (EPS0 * self.eps[0][1:nz, 1:ny, 1:nx + 1]) * cx
            cy = (_d(Hx, 0, 2, nz)[:, 1:ny + 1, 1:nx] / hz - _d(Hz, 2, 2, nx)[1:nz, 1:ny + 1, :] / hx
                  - J[1][1:nz, 1:ny + 1, 1:nx])
            Ey[1:nz, 1:ny + 1, 1:nx] += dt / (EPS0 * self.eps[1][1:nz, 1:ny + 1, 1:nx]) * cy
            cz = (_d(Hy, 2, 2, nx)[1:nz + 1, 1:ny, :] / hx - _d(Hx, 1, 2, ny)[1:nz + 1, :, 1:nx] / hy
                  - J[2][1:nz + 1, 1:ny, 1:nx])
            Ez[1:nz + 1, 1:ny, 1:nx] += dt / (EPS0 * self.eps[2][1:nz + 1, 1:ny, 1:nx]) * cz
            self.step_index += 1
            if probes:
                out.append([self.F[c][k, j, i] for c, i, j, k in probes])
        return np.array(out)
