"""Pins of the oracle's phase-shifted periodic SAT (Eqs. (EPBC1-6), (EPBCP)) and of its
dispersion analysis (Sec. "Dispersion Analysis", Eqs. (EDISPLAMBDA), (E_NUMWN),
(E_DISPER)-(E_GLOB))."""
import math

import numpy as np
import pytest

import oracle
from oracle import dispersion as dsp
from tests import ref1d

EX, EY, EZ, HX, HY, HZ = range(6)
PEC, PMC = 0, 1


def _random_complex(blocks, seed):
    rng = np.random.default_rng(seed)
    for b in blocks:
        for c in range(6):
            b.set_field(c, rng.uniform(-1, 1, b.shape(c)) * (1.0 if c < 3 else 1 / 377.0))


def test_zero_phase_equals_self_periodic_link():
    """alpha = 0: the real part evolves exactly as a block joined to itself (zero-phase
    periodic SAT), the imaginary part stays zero."""
    n, h = (6, 5, 7), (1e-3, 1.2e-3, 0.9e-3)
    dt = oracle.dt_cfl(0.9, *h)
    faces = (PEC, PMC, PMC, PEC, PEC, PEC)
    ref = oracle.Block(n, h, dt, faces)
    oracle.connect(ref, 5, ref, 4)
    re, im = oracle.Block(n, h, dt, faces), oracle.Block(n, h, dt, faces)
    oracle.connect_phase(re, im, 2, 0.0)
    _random_complex([ref], 3)
    for c in range(6):
        re.set_field(c, ref.field(c))
    oracle.step([ref], 60)
    oracle.step([re, im], 60)
    for c in range(6):
        assert np.array_equal(re.field(c), ref.field(c)), c
        assert not np.any(im.field(c)), c


@pytest.mark.parametrize("alpha", [0.3, 1.7, -2.5])
def test_reduces_to_1d_periodic_pair(alpha):
    """Fields uniform in x and y (zero-phase periodic x, y faces) with phase alpha along z
    evolve exactly as the 1D complex pair (Ex, Hy) written with the printed matrices."""
    nz, h = 24, 1e-3
    n = (4, 5, nz)
    dt = oracle.dt_cfl(0.95, h, h, h)
    re, im = oracle.Block(n, (h,) * 3, dt, (0,) * 6), oracle.Block(n, (h,) * 3, dt, (0,) * 6)
    oracle.connect_phase(re, im, 0, 0.0)
    oracle.connect_phase(re, im, 1, 0.0)
    oracle.connect_phase(re, im, 2, alpha)
    ref = ref1d.PeriodicPair1D(nz, h, dt, alpha)
    rng = np.random.default_rng(7)
    e0 = rng.uniform(-1, 1, nz + 1) + 1j * rng.uniform(-1, 1, nz + 1)
    h0 = (rng.uniform(-1, 1, nz + 2) + 1j * rng.uniform(-1, 1, nz + 2)) / 377.0
    ref.E, ref.H = e0.copy(), h0.copy()
    for blk, part in ((re, np.real), (im, np.imag)):
        blk.set_field(EX, np.broadcast_to(part(e0)[:, None, None], blk.shape(EX)).copy())
        blk.set_field(HY, np.broadcast_to(part(h0)[:, None, None], blk.shape(HY)).copy())
    oracle.step([re, im], 120)
    ref.step(120)
    ex = re.field(EX) + 1j * im.field(EX)
    hy = re.field(HY) + 1j * im.field(HY)
    assert np.max(np.abs(ex - ref.E[:, None, None])) < 1e-12 * np.max(np.abs(ref.E))
    assert np.max(np.abs(hy - ref.H[:, None, None])) < 1e-12 * np.max(np.abs(ref.H))
    for c in (EY, EZ, HX, HZ):
        assert np.max(np.abs(re.field(c))) + np.max(np.abs(im.field(c))) < 1e-12


def test_complex_energy_conserved_with_phase():
    """Phase shifts on all three axes: the energy of the complex field (real part plus
    imaginary part, Eq. (16) leapfrog form) is conserved (Eq. (EPBCE) with (EPBCP))."""
    n, h = (6, 5, 7), (1e-3, 1.2e-3, 0.9e-3)
    dt = oracle.dt_cfl(0.95, *h)
    eps = np.random.default_rng(2).uniform(1, 4, (n[2], n[1], n[0]))
    re, im = oracle.Block(n, h, dt, (0,) * 6, eps_r=eps), oracle.Block(n, h, dt, (0,) * 6, eps_r=eps)
    for a, al in enumerate((0.7, -1.9, 2.8)):
        oracle.connect_phase(re, im, a, al)
    _random_complex([re, im], 5)
    W0 = oracle.energy([re, im])
    oracle.step([re, im], 300)
    W1 = oracle.energy([re, im])
    assert abs(W1 - W0) / W0 < 1e-12


def test_amplification_matrix_unitary_spectrum():
    """Vacuum cube, oblique phases, dt = 0.99 dt_max: every eigenvalue of Lambda lies on
    the unit circle (energy-neutral PBC SATs: no dissipation)."""
    h = 1e-3
    dt = 0.99 / (dsp.C0 * math.sqrt(3) / h)
    lam = dsp.sbp_lambda((4, 4, 4), (h,) * 3, dt, (0.4, -0.9, 1.3))
    ev = np.linalg.eigvals(lam)
    assert np.max(np.abs(np.abs(ev) - 1.0)) < 1e-9


@pytest.mark.parametrize("k0h, theta, phi", [(2 * math.pi / 20, 0.0, 0.0), (2 * math.pi / 10, 0.0, 0.0),
                                             (2 * math.pi / 20, 0.7, 0.4), (2 * math.pi / 8, 1.1, 2.0)])
def test_yee_comparator_matches_closed_form(k0h, theta, phi):
    """The FDTD (Yee) comparator's numerical wavenumber, from the eigenvalues of its
    amplification matrix, equals the closed-form Yee dispersion relation."""
    h, cfl, n = 1e-3, 0.99, (4, 4, 4)
    kt, (disp, diss, glob), _ = dsp.analyse("yee", n, h, cfl, k0h, theta, phi)
    dt = cfl / (dsp.C0 * math.sqrt(3.0) / h)
    k0 = k0h / h
    ka = (k0 * math.sin(theta) * math.cos(phi), k0 * math.sin(theta) * math.sin(phi), k0 * math.cos(theta))
    rhs = sum(math.sin(k * h / 2) ** 2 for k in ka) / h ** 2
    w = 2.0 / dt * math.asin(dsp.C0 * dt * math.sqrt(rhs))
    assert abs(kt.real - w / dsp.C0) < 1e-9 * k0
    assert abs(kt.imag) < 1e-9 * k0 and diss < 1e-8


def test_sbp_dispersion_against_fdtd_normal_incidence():
    """Normal incidence along z at dt = 0.99 dt_max: the SBP-SAT scheme has the larger
    dispersion error and a vanishing dissipation error, and both errors shrink as the
    mesh is refined (the paper's Fig. on normal incidence)."""
    h, cfl, n = 1e-3, 0.99, (4, 4, 4)
    prev = None
    for ppw in (8, 10, 20, 40):
        k0h = 2 * math.pi / ppw
        _, (d_sbp, x_sbp, g_sbp), _ = dsp.analyse("sbp", n, h, cfl, k0h, 0.0, 0.0)
        _, (d_fd, x_fd, g_fd), _ = dsp.analyse("yee", n, h, cfl, k0h, 0.0, 0.0)
        assert d_sbp > d_fd
        assert x_sbp < 1e-8 and x_fd < 1e-8
        if prev is not None:
            assert d_sbp < prev
        prev = d_sbp


def test_error_largest_at_normal_incidence():
    """Both schemes have their largest error when the wave travels along an axis (the
    paper's oblique study at dt = 0.99 dt_max and lambda/20)."""
    h, cfl, n, k0h = 1e-3, 0.99, (4, 4, 4), 2 * math.pi / 20
    for scheme in ("sbp", "yee"):
        _, (_, _, g_axis), _ = dsp.analyse(scheme, n, h, cfl, k0h, 0.0, 0.0)
        for th, ph in ((math.pi / 4, 0.0), (math.pi / 4, math.pi / 4), (0.9553, math.pi / 4)):
            _, (_, _, g), _ = dsp.analyse(scheme, n, h, cfl, k0h, th, ph)
            assert g < g_axis, (scheme, th, ph)


@pytest.mark.parametrize("errors_fn", ["oracle", "product"])
def test_error_measures_closed_forms(errors_fn):
    """Eqs. (E_DISPER)-(E_GLOB) over one wavelength lambda = 2 pi / k0, for k~ = a + j b:
    e^{-j k0 lambda} = 1, so the dispersion error is |1 - e^{-j a lambda}| = 2 |sin(a lambda / 2)|,
    the dissipation error |1 - r| with r = |e^{-j k~ lambda}| = e^{b lambda}, and the global
    error follows from the law of cosines, |1 - r e^{-j a lambda}|^2 = 1 - 2 r cos(a lambda) + r^2.
    Checked on the oracle's measures and on the GPU tool's own copy (pure arithmetic, no GPU)."""
    if errors_fn == "oracle":
        fn = dsp.errors
    else:
        from paper_2206_00638_gb300 import dispersion as gdsp
        fn = gdsp.errors
    k0 = 1234.5
    lam = 2 * math.pi / k0
    for a, b in ((k0 * 1.013, 0.0), (k0 * 0.97, -0.8), (k0 * 1.2, 0.3), (k0 * 0.5, -5.0), (k0, 0.0)):
        disp, diss, glob = fn(k0, complex(a, b))
        r = math.exp(b * lam)
        assert disp == pytest.approx(2 * abs(math.sin(a * lam / 2)), abs=1e-12)
        assert diss == pytest.approx(abs(1 - r), abs=1e-12)
        assert glob == pytest.approx(math.sqrt(max(1 - 2 * r * math.cos(a * lam) + r * r, 0.0)), abs=1e-12)


def test_yee_errors_follow_closed_form_wavenumber():
    """The whole measurement chain (amplification matrix, eigenvalues, nearest wavenumber,
    error measures) on the Yee comparator at normal incidence gives the errors of the
    closed-form Yee wavenumber, 2 |sin(pi k~ / k0)| for dispersion and global error, 0 for
    dissipation."""
    h, cfl, n = 1e-3, 0.99, (4, 4, 4)
    dt = cfl / (dsp.C0 * math.sqrt(3.0) / h)
    for ppw in (10, 20):
        k0h = 2 * math.pi / ppw
        k0 = k0h / h
        kt = 2.0 / (dsp.C0 * dt) * math.asin(dsp.C0 * dt / h * math.sin(k0h / 2))
        _, (disp, diss, glob), _ = dsp.analyse("yee", n, h, cfl, k0h, 0.0, 0.0)
        want = 2 * abs(math.sin(math.pi * kt / k0))
        assert disp == pytest.approx(want, rel=1e-8) and glob == pytest.approx(want, rel=1e-8)
        assert diss < 1e-9


def test_axis_subspace_gives_the_full_spectrum_wavenumber():
    """For a wave along z the x,y-uniform fields form an invariant subspace (zero phase across
    x and y): its amplification matrix stays uniform to rounding, and the wavenumber nearest
    k0 is the one of the full Lambda of the 4^3 cube."""
    h, cfl = 1e-3, 0.99
    k0h = 2 * math.pi / 20
    kt_full, _, _ = dsp.analyse("sbp", (4, 4, 4), h, cfl, k0h, 0.0, 0.0)
    kt_axis, _, spread = dsp.analyse_axis(4, h, cfl, k0h)
    assert spread < 1e-12
    assert abs(kt_axis - kt_full) < 1e-9 * abs(kt_full)


def test_sbp_dispersion_excess_falls_as_one_over_cube_size():
    """The interior rows of the SBP operators are the Yee differences; the periodic seam
    (closure rows and SAT) adds a phase error per period that does not depend on the cube
    size n.  A wavelength then crosses ppw / n seams, so the SBP-SAT dispersion error exceeds
    the Yee error by an amount proportional to 1/n: halving it per doubling of n (lambda/20,
    dt = 0.99 dt_max, n = 4, 8, 16), and no dissipation."""
    h, cfl = 1e-3, 0.99
    k0h = 2 * math.pi / 20
    _, (d_yee, _, _), _ = dsp.analyse("yee", (4, 4, 4), h, cfl, k0h, 0.0, 0.0)
    excess = []
    for n in (4, 8, 16):
        _, (d, x, _), _ = dsp.analyse_axis(n, h, cfl, k0h)
        assert x < 1e-10
        excess.append(d - d_yee)
    assert all(e > 0 for e in excess)
    assert 1.8 < excess[0] / excess[1] < 2.2 and 1.8 < excess[1] / excess[2] < 2.2
