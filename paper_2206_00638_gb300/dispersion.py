"""Numerical dispersion of the SBP-SAT scheme, measured with the GPU path
(Sec. "Dispersion Analysis" of arXiv 2206.00638).

A small vacuum cube with phase-shifted periodic SATs on all faces (Eqs. (EPBC1-6),
``sbp_connect_phase``) carries a complex field as a pair of simulations.  Advancing the
pair one leapfrog step from every unit vector of U^n = [E^n, H^{n-1/2}] gives the
amplification matrix Lambda of Eq. (EDISPLAMBDA); each eigenvalue lambda gives a
numerical wavenumber k~ = ln(lambda) / (j c dt) (Eq. (E_NUMWN)), and the one nearest
the analytic k0 gives the dispersion, dissipation and global errors of Eqs.
(E_DISPER)-(E_GLOB).  Columns and rows follow the natural field extents, components
Ex..Hz, x fastest.
"""
from __future__ import annotations

import cmath
import math

import numpy as np

from . import sbpsat

C0 = 299792458.0


def direction_phases(k0: float, h, n, theta: float, phi: float):
    """alpha_a = k0_a * L_a for a wave along (theta, phi) (k0_x = k0 sin(theta) cos(phi),
    k0_y = k0 sin(theta) sin(phi), k0_z = k0 cos(theta)); L_a = n_a h_a."""
    k = (k0 * math.sin(theta) * math.cos(phi), k0 * math.sin(theta) * math.sin(phi), k0 * math.cos(theta))
    return tuple(k[a] * n[a] * h[a] for a in range(3))


def amplification_matrix(n, h, cfl: float, alphas, precision=sbpsat.FP64):
    """Lambda (complex, N x N) of one leapfrog step of the periodic cube; returns
    (Lambda, dt)."""
    import torch

    faces = (sbpsat.PEC,) * 6                 # replaced by the periodic faces below
    stream = torch.cuda.current_stream()      # the unit-vector writes below share it
    re = sbpsat.Sim(n, h, faces, cfl=cfl, precision=precision, stream=stream)
    im = sbpsat.Sim(n, h, faces, cfl=cfl, precision=precision, stream=stream)
    for a in range(3):
        sbpsat.connect_phase(re, im, a, alphas[a])
    dt = re.dt
    tdtype = torch.float64 if precision == sbpsat.FP64 else torch.float32
    shapes = [re.shape(c) for c in range(6)]
    sizes = [int(np.prod(s)) for s in shapes]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
    N = int(offs[-1])
    zero = [torch.zeros(s, dtype=tdtype, device="cuda") for s in shapes]
    unit = [torch.zeros(s, dtype=tdtype, device="cuda") for s in shapes]
    out_re = [torch.empty(s, dtype=tdtype, device="cuda") for s in shapes]
    out_im = [torch.empty(s, dtype=tdtype, device="cuda") for s in shapes]
    lam = torch.zeros((N, N), dtype=torch.complex128, device="cuda")
    for c in range(6):
        flat = unit[c].view(-1)
        for q in range(sizes[c]):
            for cc in range(6):
                im.set_field(cc, zero[cc])
                if cc != c:
                    re.set_field(cc, zero[cc])
            flat[q] = 1.0
            re.set_field(c, unit[c])
            flat[q] = 0.0          # ordered after the copy: same stream
            sbpsat.step_group([re, im], 1)
            for cc in range(6):
                re.field(cc, out=out_re[cc])
                im.field(cc, out=out_im[cc])
            col = torch.cat([torch.complex(out_re[cc].double().view(-1), out_im[cc].double().view(-1))
                             for cc in range(6)])
            lam[:, offs[c] + q] = col
    torch.cuda.synchronize()
    re.close()
    im.close()
    return lam.cpu().numpy(), dt


def nearest_wavenumber(lam: np.ndarray, dt: float, k0: float) -> complex:
    """The numerical wavenumber ln(lambda) / (j c dt) nearest to k0 over the spectrum."""
    ev = np.linalg.eigvals(lam)
    ev = ev[np.abs(ev) > 0]
    kt = np.log(ev) / (1j * C0 * dt)
    return complex(kt[int(np.argmin(np.abs(kt - k0)))])


def errors(k0: float, kt: complex):
    """(dispersion, dissipation, global) errors over one wavelength 2 pi / k0 of the
    numerical wavenumber kt = k_real + j k_imag; the dissipation factor over a
    wavelength is the modulus e^{k_imag lambda} of e^{-j kt lambda}."""
    wl = 2.0 * math.pi / k0
    ref = cmath.exp(-1j * k0 * wl)
    return (abs(ref - cmath.exp(-1j * kt.real * wl)),
            abs(1.0 - math.exp(kt.imag * wl)),
            abs(ref - cmath.exp(-1j * kt * wl)))


def analyse(k0h: float, theta: float = 0.0, phi: float = 0.0, n=(4, 4, 4), h: float = 1e-3, cfl: float = 0.99,
            precision=sbpsat.FP64):
    """Dispersion of the SBP-SAT scheme for a plane wave of k0 = k0h / h along
    (theta, phi) on an n-cell periodic cube of spacing h at dt = cfl * dt_max."""
    k0 = k0h / h
    hh = (h, h, h)
    lam, dt = amplification_matrix(n, hh, cfl, direction_phases(k0, hh, n, theta, phi), precision)
    kt = nearest_wavenumber(lam, dt, k0)
    disp, diss, glob = errors(k0, kt)
    return {"k0": k0, "k_numerical": kt, "dispersion": disp, "dissipation": diss, "global": glob, "dt": dt}
