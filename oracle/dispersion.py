"""Numerical dispersion of the SBP-SAT scheme (Sec. "Dispersion Analysis") on the oracle.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: it checks the GPU dispersion
tool.  A periodic cube in vacuum with phase shifts alpha_a = k0_a * L_a across the
domain (Eqs. (EPBC1-6)) is advanced one leapfrog step from every unit vector to form
the amplification matrix Lambda of Eq. (EDISPLAMBDA) (U^n = [E^n, H^{n-1/2}]).  Each
eigenvalue lambda gives a numerical wavenumber k~ = ln(lambda) / (j c dt) (Eq.
(E_NUMWN)); the one nearest the analytic k0 defines the dispersion, dissipation and
global errors of Eqs. (E_DISPER), (E_DISSIP), (E_GLOB).

The FDTD comparator is the textbook Yee scheme on the same periodic cube (E on cell
edges, H on face centres, Bloch-periodic wrap), whose dispersion relation has the
closed form sin^2(w dt/2)/(c dt)^2 = sum_a sin^2(k_a h_a/2)/h_a^2.
"""
import cmath
import math

import numpy as np

from . import Block, EX, connect_phase, step

C0 = 299792458.0
EPS0 = 8.8541878128e-12
MU0 = 1.25663706212e-6


def phases(k0, h, n, theta, phi):
    """alpha_a = k0_a L_a for the direction (theta, phi) of the paper's oblique study."""
    k = (k0 * math.sin(theta) * math.cos(phi), k0 * math.sin(theta) * math.sin(phi), k0 * math.cos(theta))
    return tuple(k[a] * n[a] * h[a] for a in range(3))


def sbp_lambda(n, h, dt, alphas):
    """Amplification matrix of the SBP-SAT scheme with phase-shifted PBC on all faces
    (complex field = pair of oracle blocks), columns in the order of the oracle's natural
    field extents, components Ex..Hz."""
    re = Block(n, h, dt, (0,) * 6)
    im = Block(n, h, dt, (0,) * 6)
    for a in range(3):
        connect_phase(re, im, a, alphas[a])
    shapes = [re.shape(c) for c in range(6)]
    sizes = [int(np.prod(s)) for s in shapes]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    N = int(offs[-1])
    lam = np.zeros((N, N), complex)
    zero = [np.zeros(s) for s in shapes]
    for c in range(6):
        for q in range(sizes[c]):
            for b in (re, im):
                for cc in range(6):
                    b.set_field(cc, zero[cc])
            u = np.zeros(sizes[c])
            u[q] = 1.0
            re.set_field(c, u.reshape(shapes[c]))
            step([re, im], 1)
            col = np.concatenate([re.field(cc).ravel() + 1j * im.field(cc).ravel() for cc in range(6)])
            lam[:, offs[c] + q] = col
    return lam


def sbp_lambda_axis(n, h, dt, alpha):
    """Amplification matrix of the SBP-SAT scheme restricted to fields that are uniform in
    x and y, for a plane wave along z (the paper's normal-incidence case: phase alpha on the
    z faces, zero on the x and y faces).  With zero phase across x and y the periodic SAT
    leaves such fields uniform (the operators take constants to zero and the penalty
    differences vanish), so this subspace is invariant and its eigenvalues are eigenvalues
    of the full Lambda.  Columns and rows: component Ex..Hz, then the z index of the
    component's z extent; one leapfrog step of the oracle per column."""
    re = Block(n, h, dt, (0,) * 6)
    im = Block(n, h, dt, (0,) * 6)
    for a, al in enumerate((0.0, 0.0, alpha)):
        connect_phase(re, im, a, al)
    shapes = [re.shape(c) for c in range(6)]
    nzs = [s[0] for s in shapes]
    offs = np.concatenate([[0], np.cumsum(nzs)]).astype(int)
    N = int(offs[-1])
    lam = np.zeros((N, N), complex)
    spread = 0.0
    for c in range(6):
        for q in range(nzs[c]):
            for b in (re, im):
                for cc in range(6):
                    b.set_field(cc, np.zeros(shapes[cc]))
            u = np.zeros(shapes[c])
            u[q] = 1.0
            re.set_field(c, u)
            step([re, im], 1)
            for cc in range(6):
                F = re.field(cc) + 1j * im.field(cc)
                col = F[:, 0, 0]
                spread = max(spread, float(np.max(np.abs(F - col[:, None, None]))))
                lam[offs[cc]:offs[cc + 1], offs[c] + q] = col
    return lam, spread


def analyse_axis(n, h, cfl, k0h):
    """Numerical wavenumber nearest k0 and its three errors for a plane wave along z on an
    n x n x n periodic SBP-SAT cube (uniform-in-x,y subspace, so n can be large).
    Returns (k~, (dispersion, dissipation, global), spread), spread = the largest departure
    from x,y-uniformity seen in any column (0 up to rounding)."""
    hh = (h, h, h)
    dt = cfl / (C0 * math.sqrt(3.0 / (h * h)))
    k0 = k0h / h
    lam, spread = sbp_lambda_axis((n, n, n), hh, dt, k0 * n * h)
    kt, _ = wavenumbers(lam, dt)
    i = int(np.argmin(np.abs(kt - k0)))
    return kt[i], errors(k0, kt[i]), spread


def _bloch_fwd(F, axis, alpha, h):
    """(F[i+1] - F[i]) / h with F[n] = e^{-j alpha} F[0]."""
    up = np.roll(F, -1, axis=axis)
    idx = [slice(None)] * 3
    idx[axis] = -1
    up[tuple(idx)] *= cmath.exp(-1j * alpha)
    return (up - F) / h


def _bloch_bwd(F, axis, alpha, h):
    """(F[i] - F[i-1]) / h with F[-1] = e^{+j alpha} F[n-1]."""
    dn = np.roll(F, 1, axis=axis)
    idx = [slice(None)] * 3
    idx[axis] = 0
    dn[tuple(idx)] *= cmath.exp(1j * alpha)
    return (F - dn) / h


def yee_step(E, H, h, dt, alphas):
    """One Yee leapfrog step on a Bloch-periodic cube (arrays (nz, ny, nx); array axis
    2 - a is spatial axis a)."""
    ax = lambda a: 2 - a
    fw = lambda F, a: _bloch_fwd(F, ax(a), alphas[a], h[a])
    bw = lambda F, a: _bloch_bwd(F, ax(a), alphas[a], h[a])
    Ex, Ey, Ez = E
    Hx, Hy, Hz = H
    Hx = Hx - dt / MU0 * (fw(Ez, 1) - fw(Ey, 2))
    Hy = Hy - dt / MU0 * (fw(Ex, 2) - fw(Ez, 0))
    Hz = Hz - dt / MU0 * (fw(Ey, 0) - fw(Ex, 1))
    Ex = Ex + dt / EPS0 * (bw(Hz, 1) - bw(Hy, 2))
    Ey = Ey + dt / EPS0 * (bw(Hx, 2) - bw(Hz, 0))
    Ez = Ez + dt / EPS0 * (bw(Hy, 0) - bw(Hx, 1))
    return (Ex, Ey, Ez), (Hx, Hy, Hz)


def yee_lambda(n, h, dt, alphas):
    """Amplification matrix of the Yee scheme on the same periodic cube."""
    shape = (n[2], n[1], n[0])
    m = int(np.prod(shape))
    N = 6 * m
    lam = np.zeros((N, N), complex)
    for col in range(N):
        v = np.zeros(N, complex)
        v[col] = 1.0
        F = [v[c * m:(c + 1) * m].reshape(shape) for c in range(6)]
        E, H = yee_step(F[:3], F[3:], h, dt, alphas)
        lam[:, col] = np.concatenate([f.ravel() for f in E + H])
    return lam


def wavenumbers(lam, dt):
    """k~ = ln(lambda) / (j c dt) for every eigenvalue (Eq. (E_NUMWN))."""
    ev = np.linalg.eigvals(lam)
    ev = ev[np.abs(ev) > 1e-300]
    return np.log(ev) / (1j * C0 * dt), ev


def errors(k0, kt):
    """Dispersion, dissipation and global error of Eqs. (E_DISPER)-(E_GLOB) for the
    numerical wavenumber kt = k_real + j k_imag, over one wavelength lambda = 2 pi / k0.
    The dissipation factor over a wavelength is e^{k_imag lambda} (the modulus of
    e^{-j kt lambda})."""
    lamw = 2.0 * math.pi / k0
    disp = abs(cmath.exp(-1j * k0 * lamw) - cmath.exp(-1j * kt.real * lamw))
    diss = abs(1.0 - math.exp(kt.imag * lamw))
    glob = abs(cmath.exp(-1j * k0 * lamw) - cmath.exp(-1j * kt * lamw))
    return disp, diss, glob


def analyse(scheme, n, h, cfl, k0h, theta, phi):
    """Numerical wavenumber nearest k0 and its three errors for scheme 'sbp' or 'yee'.
    k0h = k0 * h (cubic cells); dt = cfl * dt_max with dt_max the 3D CFL limit."""
    hh = (h, h, h)
    dt = cfl / (C0 * math.sqrt(3.0 / (h * h)))
    k0 = k0h / h
    al = phases(k0, hh, n, theta, phi)
    lam = (sbp_lambda if scheme == "sbp" else yee_lambda)(n, hh, dt, al)
    kt, ev = wavenumbers(lam, dt)
    i = int(np.argmin(np.abs(kt - k0)))
    return kt[i], errors(k0, kt[i]), ev
