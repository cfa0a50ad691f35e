"""Pins of the oracle's leapfrog, sources, probes and energy monitor."""
import math

import numpy as np
import pytest

import oracle
from oracle import PEC, PMC, ABSORBING, EX, EY, EZ, HX, HY, HZ
from paper_2206_00638_gb300 import workloads as wl
from tests import ref1d


def _block_from(spec, dt):
    blk = oracle.Block(spec.n, spec.h, dt, spec.faces, eps_r=spec.eps_r, mu_r=spec.mu_r)
    if spec.fields is not None:
        for c in range(6):
            blk.set_field(c, spec.fields[c])
    for s in spec.sources:
        blk.add_source(s.comp, s.i, s.j, s.k, s.kind, s.amp, s.tw, s.t0, s.f)
    for p in spec.probes:
        blk.add_probe(p.comp, p.i, p.j, p.k)
    return blk


def test_dt_matches_paper_example():
    """Sec. VI-A: dt_max = 76.98 ps for a 4 cm cubic mesh (the paper's c = 3e8)."""
    assert oracle.dt_cfl(1.0, 0.04, 0.04, 0.04, 3e8) * 1e12 == pytest.approx(76.98, abs=0.005)


def test_waveforms_closed_forms():
    tw, t0 = 80e-12, 80e-12
    assert oracle.waveform(oracle.GAUSS, t0, tw, t0) == 1.0
    assert oracle.waveform(oracle.GAUSS, t0 + tw / 2, tw, t0) == pytest.approx(math.exp(-math.pi))
    xs = tw / math.sqrt(8 * math.pi)
    assert oracle.waveform(oracle.GAUSS_DERIV, t0 - xs, tw, t0) == pytest.approx(1.0, rel=1e-14)
    assert oracle.waveform(oracle.GAUSS_DERIV, t0 + xs, tw, t0) == pytest.approx(-1.0, rel=1e-14)
    f = 36e9
    t = 0.9e-9
    assert oracle.waveform(oracle.MOD_GAUSS, t, 0.11e-9, 0.85e-9, f) == pytest.approx(
        math.sin(2 * math.pi * f * t) * math.exp(-4 * math.pi * (0.05e-9) ** 2 / (0.11e-9) ** 2))


@pytest.mark.parametrize("faces", [(PEC,) * 6, (PMC,) * 6, (PEC, PMC, PMC, PEC, PMC, PEC)])
def test_leapfrog_energy_conserved(faces):
    """Energy-neutral SATs: the leapfrog energy W^n is constant to round-off (dt = 0.99 CFL)."""
    n, h = (6, 5, 7), (0.01, 0.012, 0.009)
    dt = oracle.dt_cfl(0.99, *h)
    eps = np.random.default_rng(7).uniform(1, 4, size=(n[2], n[1], n[0]))
    blk = oracle.Block(n, h, dt, faces, eps_r=eps)
    for c, f in enumerate(wl.random_fields(n, 11)):
        blk.set_field(c, f if c < 3 else f / 377.0)
    W0 = oracle.energy([blk])
    Ws = []
    for _ in range(20):
        oracle.step([blk], 25)
        Ws.append(oracle.energy([blk]))
    assert W0 > 0
    assert max(abs(w - W0) for w in Ws) / W0 < 1e-12


def test_leapfrog_energy_conserved_two_blocks():
    n, h = (5, 6, 4), (0.01, 0.01, 0.01)
    dt = oracle.dt_cfl(0.95, *h)
    A = oracle.Block(n, h, dt, (PEC,) * 6)
    B = oracle.Block((5, 6, 7), h, dt, (PMC,) * 6, eps_r=np.full((7, 6, 5), 2.0))
    oracle.connect(A, 5, B, 4)
    for blk, seed in ((A, 3), (B, 4)):
        for c, f in enumerate(wl.random_fields(blk.n, seed)):
            blk.set_field(c, f if c < 3 else f / 377.0)
    W0 = oracle.energy([A, B])
    oracle.step([A, B], 300)
    assert abs(oracle.energy([A, B]) - W0) / W0 < 1e-12


def test_absorbing_energy_decays():
    n, h = (6, 5, 7), (0.01, 0.01, 0.01)
    dt = oracle.dt_cfl(0.95, *h)
    blk = oracle.Block(n, h, dt, (ABSORBING, PEC, PMC, ABSORBING, ABSORBING, ABSORBING))
    for c, f in enumerate(wl.random_fields(n, 5)):
        blk.set_field(c, f if c < 3 else f / 377.0)
    prev = oracle.energy([blk])
    W0 = prev
    for _ in range(40):
        oracle.step([blk], 5)
        w = oracle.energy([blk])
        assert w <= prev * (1 + 1e-13)
        prev = w
    assert prev < 0.5 * W0


def _fit_frequency(sig, dt, f_lo, f_hi):
    t = np.arange(len(sig)) * dt
    def resid(f):
        A = np.stack([np.cos(2 * np.pi * f * t), np.sin(2 * np.pi * f * t), np.ones_like(t)], 1)
        coef, *_ = np.linalg.lstsq(A, sig, rcond=None)
        return np.sum((A @ coef - sig) ** 2)
    fs = np.linspace(f_lo, f_hi, 801)
    r = [resid(f) for f in fs]
    f0 = fs[int(np.argmin(r))]
    lo, hi = f0 - (fs[1] - fs[0]), f0 + (fs[1] - fs[0])
    for _ in range(60):        # golden-section refinement
        m1, m2 = lo + 0.382 * (hi - lo), lo + 0.618 * (hi - lo)
        if resid(m1) < resid(m2):
            hi = m2
        else:
            lo = m1
    return 0.5 * (lo + hi)


def test_cavity_resonance_and_energy():
    """PEC cavity 1.0 x 0.8 x 0.6 m (20x16x12 cells), TE101-type mode + 1e-3 noise, 500 steps
    at 0.9 CFL: the Ez probe oscillates at the analytic (c/2) sqrt(1/a^2 + 1/b^2) = 239.95 MHz
    within 0.5 %, and the leapfrog energy is conserved to 1e-12 (Sec. VI-A)."""
    w = wl.cavity()
    spec = w.blocks[0]
    dt = oracle.dt_cfl(w.cfl, *spec.h)
    blk = _block_from(spec, dt)
    blk.reserve_probes(w.steps)
    W0 = oracle.energy([blk])
    oracle.step([blk], w.steps)
    W1 = oracle.energy([blk])
    assert abs(W1 - W0) / W0 < 1e-12
    sig = blk.probes()[0]
    f = _fit_frequency(sig, dt, 200e6, 280e6)
    f_exact = wl.cavity_resonance_hz()
    assert f_exact == pytest.approx(239.95e6, rel=1e-4)
    assert abs(f - f_exact) / f_exact < 5e-3


def _cavity_mode_error(m):
    """(f - f_exact) / f_exact of the Ez mode of the 1.0 x 0.8 x 0.6 m PEC cavity on 10m x 8m x 6m
    cells, from the initial mode shape (no noise) over 12 periods at 0.9 CFL."""
    a, bw = 1.0, 0.8
    n = (10 * m, 8 * m, 6 * m)
    h = a / n[0]
    dt = oracle.dt_cfl(0.9, h, h, h)
    blk = oracle.Block(n, (h, h, h), dt, (PEC,) * 6)
    shp = blk.shape(EZ)
    x, y = np.arange(shp[2]) * h, np.arange(shp[1]) * h
    mode = np.sin(np.pi * x / a)[None, :] * np.sin(np.pi * y / bw)[:, None]
    blk.set_field(EZ, np.ascontiguousarray(np.broadcast_to(mode[None], shp)))
    blk.add_probe(EZ, n[0] // 2 - 1, n[1] // 2 - 1, n[2] // 2)
    f_exact = wl.cavity_resonance_hz()
    steps = int(12 / f_exact / dt)
    blk.reserve_probes(steps)
    oracle.step([blk], steps)
    f = _fit_frequency(blk.probes()[0], dt, 0.95 * f_exact, 1.05 * f_exact)
    return (f - f_exact) / f_exact


def test_cavity_frequency_converges_second_order():
    """The scheme is second order in space and time (dt scales with h), so the cavity mode's
    frequency error falls 4x per halving of h: at 10, 20 and 40 cells along a the errors are
    -5.0e-3, -7.4e-4, -1.7e-4 (observed orders 2.8 and 2.1; the pin asks > 1.7 and the sign of
    numerical dispersion, a slower wave)."""
    e = [_cavity_mode_error(m) for m in (1, 2, 4)]
    assert all(v < 0 for v in e), e
    orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert min(orders) > 1.7, (e, orders)
    assert abs(e[2]) < 3e-4, e


def test_mode_shape_preserved():
    """After 500 steps the Ez field is still the sin(pi x/a) sin(pi y/b) mode (correlation >= 0.999)."""
    w = wl.cavity(noise=0.0)
    spec = w.blocks[0]
    dt = oracle.dt_cfl(w.cfl, *spec.h)
    blk = _block_from(spec, dt)
    oracle.step([blk], 500)
    ez = blk.field(EZ)
    mode = spec.fields[EZ]
    c = np.sum(ez * mode) / math.sqrt(np.sum(ez * ez) * np.sum(mode * mode))
    assert abs(c) > 0.999


def test_material_factor_scales_e_equations():
    """Uniform eps_r multiplies every E right-hand side by 1/eps_r and leaves H unchanged."""
    n, h = (4, 5, 6), (0.01, 0.01, 0.01)
    b1 = oracle.Block(n, h, 1e-12, (PEC, PMC) * 3)
    b4 = oracle.Block(n, h, 1e-12, (PEC, PMC) * 3, eps_r=np.full((6, 5, 4), 4.0))
    for b in (b1, b4):
        for c, f in enumerate(wl.random_fields(n, 9)):
            b.set_field(c, f)
        oracle.rhs([b])
    for c in range(6):
        scale = 0.25 if c < 3 else 1.0
        np.testing.assert_allclose(b4.rhs(c), scale * b1.rhs(c), rtol=1e-13, atol=0)


def test_node_material_closed_box_mean():
    """Half-space eps_r = 1 | 4 split at z-cell n/2: E nodes on the split plane see 2.5,
    nodes elsewhere see their own cell; Ez (on z-) never sits on the plane."""
    n = (4, 5, 6)
    eps = np.ones((6, 5, 4))
    eps[3:] = 4.0
    b = oracle.Block(n, (0.01,) * 3, 1e-12, (PEC,) * 6, eps_r=eps)
    ex = b.node_eps(EX)            # z+ index k, plane k=3 is the split
    assert np.all(ex[:3] == 1.0) and np.all(ex[3] == 2.5) and np.all(ex[4:] == 4.0)
    ez = b.node_eps(EZ)            # z- index: 0 -> cell 0, c in 1..6 -> cell c-1, 7 -> cell 5
    assert np.all(ez[:4] == 1.0) and np.all(ez[4:] == 4.0)


@pytest.mark.parametrize("faces_z", [(PEC, PMC), (PMC, PEC), (ABSORBING, ABSORBING), (PEC, ABSORBING)])
def test_reduces_to_1d_scheme(faces_z):
    """Fields uniform in x, y in a guide with PEC x-faces and PMC y-faces evolve exactly as the
    1D SBP-SAT scheme of the pair (Ex, Hy) along z, written with dense printed matrices;
    includes a Gaussian sheet current on Ex and a layered dielectric."""
    nz, h = 40, 1e-3
    n = (4, 5, nz)
    eps_z = np.where(np.arange(nz) < nz // 2, 1.0, 3.0)
    eps = np.broadcast_to(eps_z[:, None, None], (nz, 5, 4)).copy()
    dt = oracle.dt_cfl(0.95, h, h, h)
    faces = (PEC, PEC, PMC, PMC) + tuple(faces_z)
    blk = oracle.Block(n, (h, h, h), dt, faces, eps_r=eps)
    ref = ref1d.Pair1D(nz, h, dt, faces_z[0], faces_z[1], eps_cells=eps_z)
    rng = np.random.default_rng(1)
    e0 = rng.uniform(-1, 1, nz + 1)
    h0 = rng.uniform(-1, 1, nz + 2) / 377.0
    ex = np.broadcast_to(e0[:, None, None], blk.shape(EX)).copy()
    hy = np.broadcast_to(h0[:, None, None], blk.shape(HY)).copy()
    blk.set_field(EX, ex)
    blk.set_field(HY, hy)
    ref.E, ref.H = e0.copy(), h0.copy()
    tw = 20 * dt
    blk.add_source(EX, -1, -1, 7, oracle.GAUSS, 3.0, tw, tw)
    ref.add_sheet(7, 3.0, tw, tw)
    oracle.step([blk], 150)
    ref.step(150)
    ex3 = blk.field(EX)
    hy3 = blk.field(HY)
    scale_e = np.max(np.abs(ref.E))
    scale_h = np.max(np.abs(ref.H))
    assert np.max(np.abs(ex3 - ref.E[:, None, None])) < 1e-12 * scale_e
    assert np.max(np.abs(hy3 - ref.H[:, None, None])) < 1e-12 * scale_h
    for c in (EY, EZ, HX, HZ):
        assert np.max(np.abs(blk.field(c))) < 1e-12 * scale_e


def test_absorbing_reflection_small():
    """A 20-cell Gaussian pulse leaving through the absorbing z+ face at normal incidence keeps
    < 1e-6 of its energy (measured 7.4e-8, amplitude reflection ~3e-4) in the 1D reduction."""
    nz, h = 400, 1e-3
    dt = oracle.dt_cfl(0.95, h, h, h)
    ref = ref1d.Pair1D(nz, h, dt, ref1d.PEC, ref1d.ABSORBING)
    z = np.arange(nz + 1) * h
    zc, w = 0.6 * nz * h, 20 * h
    ref.E = np.exp(-((z - zc) / w) ** 2)
    zm = np.concatenate([[0.0], (np.arange(nz) + 0.5) * h, [nz * h]])
    eta = math.sqrt(ref1d.MU0 / ref1d.EPS0)
    ref.H = np.exp(-((zm - zc + 0.5 * dt * 299792458.0) / w) ** 2) / eta
    Pp = h * np.ones(nz + 1); Pp[[0, -1]] *= 0.5
    e_in = np.sum(ref1d.EPS0 * Pp * ref.E ** 2)
    ref.step(int(1.2 * 0.4 * nz * h / (299792458.0 * dt)) + 200)
    e_out = np.sum(ref1d.EPS0 * Pp * ref.E ** 2)
    assert e_out / e_in < 1e-6


def _oblique_reflection(theta_deg, top, ppw=20, w_wl=3.0, nx=4, comp=EY):
    """|reflected| / |incident| envelope of a plane-wave packet (k in the x-z plane at theta from
    z) hitting the z+ face `top`: TE with comp = E_y (E^0 only), TM with comp = H_y (H^{-1/2}
    only); either is divergence-free and splits into an up- and a down-going half.  The packet
    is periodic in x with the phase k_x L_x (phase-shifted periodic SAT, a complex field as two
    real blocks) and uniform in y.  Envelopes of comp at a probe between the packet and the
    face, before and after the reflection; the z- face is far enough that its echo arrives
    later."""
    h = 1e-3
    lam = ppw * h
    w = w_wl * lam
    th = math.radians(theta_deg)
    gap = int(round(2.5 * w / h))
    kc = 3 * gap                                  # packet centre; probe at kc + gap; face at kc + 2 gap
    n = (nx, 4, kc + 2 * gap)
    dt = oracle.dt_cfl(0.95, h, h, h)
    faces = (PEC, PEC, PEC, PEC, PEC, top)
    re, im = oracle.Block(n, (h,) * 3, dt, faces), oracle.Block(n, (h,) * 3, dt, faces)
    k = 2 * math.pi / lam
    kx, kz = k * math.sin(th), k * math.cos(th)
    oracle.connect_phase(re, im, 0, kx * nx * h)
    oracle.connect_phase(re, im, 1, 0.0)
    shp = re.shape(comp)
    plus = ((1, 0, 1) if comp == EY else (0, 1, 0))   # Table I: E_y (x+, y-, z+), H_y (x-, y+, z-)
    z = _grid_nodes(n[2], h, plus[2])
    x = _grid_nodes(n[0], h, plus[0])
    env = np.exp(-((z - kc * h) / w) ** 2) * np.cos(kz * (z - kc * h))
    f = env[:, None, None] * np.ones(shp) * np.exp(-1j * kx * x)[None, None, :]
    re.set_field(comp, np.ascontiguousarray(f.real))
    im.set_field(comp, np.ascontiguousarray(f.imag))
    for b in (re, im):
        b.add_probe(comp, 0 if comp == EY else 1, 1, kc + gap)
    vz = 299792458.0 * dt * math.cos(th)         # packet (group) speed along z, per step
    steps = int(4.5 * gap * h / vz)
    for b in (re, im):
        b.reserve_probes(steps)
    oracle.step([re, im], steps)
    sig = np.abs(re.probes()[0] + 1j * im.probes()[0])
    mid = int(2 * gap * h / vz)
    return sig[mid:].max() / sig[:mid].max()


@pytest.mark.parametrize("theta", [45, 60])
def test_absorbing_oblique_reflection_closed_form(theta):
    """Absolute accuracy of the absorbing SAT (reading 7, not the paper's): its continuous limit
    is the first-order characteristic condition E_t - phi eta H_t = 0, which reflects an
    obliquely incident TE wave with R = (cos theta - 1) / (cos theta + 1).  Measured as the
    reflection ratio to a PEC face in the same geometry (which cancels the envelope loss of the
    measurement; |R| = 1 there), at 20 points per wavelength with a packet of 2 wavelengths:
    within 10 % of the closed form (measured 3.2 % at 45 and 2.1 % at 60 degrees; 2.0 % with 3
    wavelengths).  A wrong phi sign fails it, and so does a wrong eta at 60 degrees: a doubled
    eta is an impedance wall 2 eta, whose reflection happens to equal the correct one at 45
    degrees and vanishes at 60.  A penalty on the E equation only drives the same characteristic
    to zero and passes here; the energy pins (dissipativity, energy decay, 1D reduction) fail
    it."""
    r_abs = _oblique_reflection(theta, ABSORBING, w_wl=2.0)
    r_pec = _oblique_reflection(theta, PEC, w_wl=2.0)
    c = math.cos(math.radians(theta))
    expect = (1 - c) / (1 + c)
    assert abs(r_abs / r_pec - expect) < 0.1 * expect, (r_abs, r_pec, expect)


def test_absorbing_oblique_reflection_tm():
    """The same closed form for TM incidence (H along y): the face's other tangential pair,
    (E_x, H_y), with the opposite curl sign, and a normal E component at the face.  The
    magnitude is again (1 - cos theta) / (1 + cos theta).  This pair's discrete reflection
    converges more slowly: at 45 degrees it is 0.223 at 20 points per wavelength and 0.172 at 40,
    against 0.1716.  The pin is 40 points per wavelength, a packet of 2 wavelengths, within
    5 % (measured 1.2 %)."""
    r_abs = _oblique_reflection(45, ABSORBING, ppw=40, w_wl=2.0, comp=HY)
    r_pec = _oblique_reflection(45, PEC, ppw=40, w_wl=2.0, comp=HY)
    c = math.cos(math.radians(45))
    expect = (1 - c) / (1 + c)
    assert abs(r_abs / r_pec - expect) < 0.05 * expect, (r_abs, r_pec, expect)


def _fresnel_normal(two_blocks, er2=4.0, ppw=20, w_wl=3.0):
    """Reflected and transmitted E envelope, relative to the incident one, of a plane-wave packet
    (E_x, fields uniform in x and y through zero-phase periodic x and y faces) crossing from
    eps_r = 1 into eps_r = er2 at normal incidence: one block whose cells change at the plane
    (node material = closed-box cell mean), or two blocks joined there by the interface SAT.
    Absorbing z faces far from the packet; E^0 only, so half of the packet travels up."""
    h = 1e-3
    lam = ppw * math.sqrt(er2) * h                # ppw points per wavelength in the dense medium
    w = w_wl * lam
    gap = int(round(2.5 * w / h))
    k0 = gap + 10                                 # packet; probe at k0 + gap; step at k0 + 2 gap
    ki = k0 + 2 * gap
    nz = ki + 2 * gap
    dt = oracle.dt_cfl(0.95, h, h, h)
    if not two_blocks:
        eps = np.ones((nz, 4, 4))
        eps[ki:] = er2
        lo = hi = oracle.Block((4, 4, nz), (h,) * 3, dt, (PEC, PEC, PEC, PEC, ABSORBING, ABSORBING), eps_r=eps)
        blocks, k_hi = [lo], ki + gap
    else:
        lo = oracle.Block((4, 4, ki), (h,) * 3, dt, (PEC, PEC, PEC, PEC, ABSORBING, PEC))
        hi = oracle.Block((4, 4, nz - ki), (h,) * 3, dt, (PEC, PEC, PEC, PEC, PEC, ABSORBING),
                          eps_r=np.full((nz - ki, 4, 4), er2))
        oracle.connect(lo, 5, hi, 4)
        blocks, k_hi = [lo, hi], gap
    for b in blocks:
        oracle.connect(b, 0, b, 1)
        oracle.connect(b, 2, b, 3)
    shp = lo.shape(EX)
    z = np.arange(shp[0]) * h
    env = np.exp(-((z - k0 * h) / w) ** 2) * np.cos(2 * math.pi / lam * (z - k0 * h))
    lo.set_field(EX, np.ascontiguousarray(env[:, None, None] * np.ones(shp)))
    lo.add_probe(EX, 1, 1, k0 + gap)
    hi.add_probe(EX, 1, 1, k_hi)
    v = 299792458.0 * dt
    steps = int(4.0 * gap * h / v)
    for b in blocks:
        b.reserve_probes(steps)
    oracle.step(blocks, steps)
    below, above = lo.probes()[0], hi.probes()[-1]
    mid = int(2 * gap * h / v)
    inc = np.abs(below[:mid]).max()
    return np.abs(below[mid:]).max() / inc, np.abs(above).max() / inc


@pytest.mark.parametrize("two_blocks", [False, True])
def test_dielectric_step_fresnel(two_blocks):
    """A dielectric step eps_r 1 -> 4 reflects and transmits a normally incident wave with the
    Fresnel coefficients |R| = (n2 - n1)/(n1 + n2) = 1/3 and T = 2 n1/(n1 + n2) = 2/3 (for E):
    inside one block (node material, reading 4) and across two blocks joined by the interface
    SAT.  At 20 points per wavelength in the dense medium: R within 0.03 and T within 0.06
    (measured 0.328-0.330 and 0.641; 0.332-0.333 and 0.663 at 40 points).  An interface
    coefficient of 3/4 instead of 1/2 (a planted mistake, not committed) goes unstable."""
    R, T = _fresnel_normal(two_blocks)
    assert abs(R - 1.0 / 3.0) < 0.03, R
    assert abs(T - 2.0 / 3.0) < 0.06, T


def _oblique_te_echo(theta_deg, dielectric, er2=4.0, ppw=20, w_wl=2.0, nx=4):
    """Envelope of the echo over the incident envelope of a TE packet (E_y, k in the x-z plane at
    theta, periodic in x with phase k_x L_x: a complex field as two real blocks) that meets, at
    z = zi, either a second pair of blocks of eps_r = er2 joined by the interface SAT
    (dielectric=True) or a PEC face (dielectric=False)."""
    h = 1e-3
    lam = ppw * math.sqrt(er2) * h                # ppw points per wavelength in the dense medium
    w = w_wl * lam
    th = math.radians(theta_deg)
    k = 2 * math.pi / lam
    kx, kz = k * math.sin(th), k * math.cos(th)
    gap = int(round(2.5 * w / h))
    kc, ki = 3 * gap, 5 * gap                     # packet centre, plane of the interface / wall
    dt = oracle.dt_cfl(0.95, h, h, h)
    # z+ face of the low pair: PEC, replaced by the interface when the pair is connected
    low = [oracle.Block((nx, 4, ki), (h,) * 3, dt, (PEC, PEC, PEC, PEC, ABSORBING, PEC)) for _ in range(2)]
    blocks = [low]
    if dielectric:
        high = [oracle.Block((nx, 4, 2 * gap), (h,) * 3, dt, (PEC, PEC, PEC, PEC, PEC, ABSORBING),
                             eps_r=np.full((2 * gap, 4, nx), er2)) for _ in range(2)]
        for r in range(2):
            oracle.connect(low[r], 5, high[r], 4)
        blocks.append(high)
    for pair in blocks:
        oracle.connect_phase(pair[0], pair[1], 0, kx * nx * h)
        oracle.connect_phase(pair[0], pair[1], 1, 0.0)
    shp = low[0].shape(EY)
    z = np.arange(shp[0]) * h
    x = np.arange(shp[2]) * h
    env = np.exp(-((z - kc * h) / w) ** 2) * np.cos(kz * (z - kc * h))
    f = env[:, None, None] * np.ones(shp) * np.exp(-1j * kx * x)[None, None, :]
    low[0].set_field(EY, np.ascontiguousarray(f.real))
    low[1].set_field(EY, np.ascontiguousarray(f.imag))
    vz = 299792458.0 * dt * math.cos(th)
    steps = int(4.5 * gap * h / vz)
    for b in low:
        b.add_probe(EY, 0, 1, kc + gap)
    for pair in blocks:
        for b in pair:
            b.reserve_probes(steps)
    oracle.step([b for pair in blocks for b in pair], steps)
    sig = np.abs(low[0].probes()[0] + 1j * low[1].probes()[0])
    mid = int(2 * gap * h / vz)
    return sig[mid:].max() / sig[:mid].max()


def test_interface_oblique_fresnel_te():
    """Across two blocks joined by the interface SAT, eps_r 1 -> 4, a TE wave at 60 degrees is
    reflected with |R| = (n1 cos ti - n2 cos tt) / (n1 cos ti + n2 cos tt) = 0.5657 (Snell:
    sin tt = sin ti / 2).  This exercises the (E_y, H_x) pair of the interface together with the
    phase-shifted periodic faces.  The fixed period in x gives each spectral component of the
    packet its own angle, so the packet spreads along z.  The echo is therefore taken relative to
    a PEC wall in the same place, as in the absorbing test.  At 20 points per wavelength this
    gives 0.5646, within 2 % (measured 0.2 %; 0.1-0.5 % at 0, 30 and 45 degrees)."""
    r_die = _oblique_te_echo(60, True)
    r_pec = _oblique_te_echo(60, False)
    ti = math.radians(60)
    tt = math.asin(math.sin(ti) / 2.0)
    expect = abs((math.cos(ti) - 2.0 * math.cos(tt)) / (math.cos(ti) + 2.0 * math.cos(tt)))
    assert abs(r_die / r_pec - expect) < 0.02 * expect, (r_die, r_pec, expect)


# SI constants, typed here rather than taken from the oracle (CODATA 2018)
_C0 = 299792458.0
_MU0 = 1.25663706212e-6
_EPS0 = 1.0 / (_MU0 * _C0 * _C0)


@pytest.mark.parametrize("er", [1.0, 4.0])
def test_sheet_current_radiates_half_eta_k(er):
    """A uniform current sheet K(t) = J(t) h (the sheet current J on the E_x nodes of one plane,
    whose norm weight is h) in a medium of relative permittivity er radiates
    E_x = -(eta/2) K(t - |z - z0|/v), eta = eta0/sqrt(er), v = c/sqrt(er), to both sides: the
    jump of H_y across it is K and the outgoing waves are plane.  Checked at 0, 20 and 40
    cells for a Gaussian of width 80 sqrt(er) dt, within 0.8 % of the peak (measured
    0.16-0.40 %).  The current enters the E update at t^{n+1/2} (Eq. (12) with J); evaluated
    at t^n or t^{n+1} instead, the vacuum case gives 1.7-2.1 % and fails.  A wrong sign, scale
    or material factor fails both."""
    h = 1e-3
    nz, ks = 400, 200
    dt = oracle.dt_cfl(0.95, h, h, h)
    b = oracle.Block((4, 4, nz), (h,) * 3, dt, (PEC, PEC, PEC, PEC, ABSORBING, ABSORBING),
                     eps_r=np.full((nz, 4, 4), er))
    oracle.connect(b, 0, b, 1)                    # fields uniform in x and y
    oracle.connect(b, 2, b, 3)
    tw, amp = 80 * math.sqrt(er) * dt, 2.5
    b.add_source(EX, -1, -1, ks, oracle.GAUSS, amp, tw, tw)
    dists = (0, 20, 40)
    for d in dists:
        b.add_probe(EX, 1, 1, ks + d)
    v = _C0 / math.sqrt(er)
    steps = int((2 * tw + dists[-1] * h / v) / dt) + 5   # no echo from the far faces by then
    b.reserve_probes(steps)
    oracle.step([b], steps)
    t = (np.arange(steps) + 1) * dt               # probe slot s holds E^{s+1}
    eta = math.sqrt(_MU0 / (_EPS0 * er))
    for q, d in enumerate(dists):
        x = t - d * h / v - tw
        expect = -(eta / 2) * amp * h * np.exp(-4 * math.pi * x ** 2 / tw ** 2)
        err = np.abs(b.probes()[q] - expect).max() / np.abs(expect).max()
        assert err < 0.008, (d, err)


def test_point_current_radiates_hertzian_dipole_field():
    """A current J(t) on one E_z node is a current element I l = J h^3.  In free space its
    field on the equatorial plane is E_z = -(1/(4 pi eps0)) [p/r^3 + p'/(c r^2) + p''/(c^2 r)]
    at t - r/c, with p' = I l: static, induction and radiation terms together.  With the
    normalised Gaussian-derivative waveform, p is a Gaussian (no charge left behind).  Six
    absorbing faces 32 cells out, probes 8 and 12 cells from the source, compared before the
    first echo can arrive: within 5 % of the peak (measured 1.9-2.1 %; a source evaluated half
    a step early or late gives 8-14 %)."""
    h = 1e-3
    n = 64
    c = n // 2
    dt = oracle.dt_cfl(0.95, h, h, h)
    b = oracle.Block((n, n, n), (h,) * 3, dt, (ABSORBING,) * 6)
    tw, amp = 40 * dt, 1.0
    b.add_source(EZ, c, c, c, oracle.GAUSS_DERIV, amp, tw, tw)
    dists = (8, 12)
    for d in dists:
        b.add_probe(EZ, c + d, c, c)
    steps = int((2 * tw + dists[-1] * h / _C0) / dt) + 5
    b.reserve_probes(steps)
    oracle.step([b], steps)
    t = (np.arange(steps) + 1) * dt
    # GAUSS_DERIV = K dG/dt with G = exp(-4 pi x^2 / tw^2) and K = tw e^{1/2} / sqrt(8 pi)
    m = amp * h ** 3 * tw * math.exp(0.5) / math.sqrt(8 * math.pi)
    for q, d in enumerate(dists):
        r = d * h
        x = t - r / _C0 - tw
        a = 8 * math.pi / tw ** 2
        G = np.exp(-0.5 * a * x ** 2)
        G1 = -a * x * G
        G2 = (a * a * x * x - a) * G
        expect = -(m / (4 * math.pi * _EPS0)) * (G / r ** 3 + G1 / (_C0 * r ** 2) + G2 / (_C0 ** 2 * r))
        before_echo = t < (2 * (n - c) - d) * h / _C0     # first echo: off the x+ face
        err = np.abs(b.probes()[q][before_echo] - expect[before_echo]).max() / np.abs(expect).max()
        assert err < 0.05, (d, err)


def _grid_nodes(n, h, plus):
    """Node positions of the plus grid x_i = i h or of the minus grid
    [x_0, x_{1/2}, ..., x_{n-1/2}, x_n] (Sec. II, the two one-dimensional grids)."""
    if plus:
        return np.arange(n + 1) * h
    return np.concatenate([[0.0], (np.arange(1, n + 1) - 0.5) * h, [n * h]])


# E_x .. H_z = prod over axes of cos(k pi x / L + phase): (k, phase) per component and axis
_ENERGY_MODES = [[(1.3, 0.4), (0.7, 1.1), (2.1, 0.2)], [(0.9, 0.3), (1.7, 0.5), (0.6, 1.3)],
                 [(1.1, 0.8), (0.5, 0.1), (1.9, 0.6)], [(2.3, 0.2), (1.2, 0.9), (0.8, 0.4)],
                 [(0.6, 1.0), (2.0, 0.3), (1.4, 0.7)], [(1.5, 0.6), (0.9, 1.2), (1.0, 0.5)]]


def _energy_rel_error(m, er=2.5, mr=1.5):
    """(W - exact) / exact of the E part (H = 0) and of the H part (E = 0) of the oracle's
    energy for smooth fields on a 0.9 x 0.7 x 0.5 m box of 9m x 8m x 6m cells."""
    L = (0.9, 0.7, 0.5)
    n = (9 * m, 8 * m, 6 * m)
    h = tuple(L[a] / n[a] for a in range(3))
    on_plus = ((0, 1, 1), (1, 0, 1), (1, 1, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1))   # Table I
    xg, wg = np.polynomial.legendre.leggauss(200)

    def mode(c, a, x):
        k, ph = _ENERGY_MODES[c][a]
        return np.cos(k * math.pi * x / L[a] + ph)

    out = []
    for comps, coef in ((range(3), _EPS0 * er), (range(3, 6), _MU0 * mr)):
        b = oracle.Block(n, h, oracle.dt_cfl(0.5, *h), (PEC,) * 6, eps_r=np.full(n[::-1], er),
                         mu_r=np.full(n[::-1], mr))
        exact = 0.0
        for c in comps:
            x, y, z = (_grid_nodes(n[a], h[a], on_plus[c][a]) for a in range(3))
            f = mode(c, 2, z)[:, None, None] * mode(c, 1, y)[None, :, None] * mode(c, 0, x)[None, None, :]
            assert f.shape == tuple(b.shape(c))
            b.set_field(c, np.ascontiguousarray(f))
            term = 1.0
            for a in range(3):                     # Gauss-Legendre on [0, L_a], exact here
                xa = 0.5 * L[a] * (xg + 1)
                term *= np.sum(0.5 * L[a] * wg * mode(c, a, xa) ** 2)
            exact += term
        exact *= 0.5 * coef
        out.append((oracle.energy([b]) - exact) / exact)
    return out


def test_energy_converges_to_field_energy():
    """The discrete energy of Eq. (16) (E^T eps P E + H^{n-1/2} mu P H^{n+1/2}, halved) of
    smooth fields converges to the continuous (1/2) int eps E^2 + mu H^2 dV at second order:
    within 2.5e-3 on 9x8x6 x 4 cells and 5e-4 at twice the resolution (measured 1.2e-3 / 7e-4
    and 2.2e-4 / 2.3e-4), on a box with three different spacings, eps_r 2.5 and mu_r 1.5.
    Each field sits on its own grid pair (Table I) and takes that pair's norm weights.
    Uniform weights (closure weights dropped), the spacing of the wrong axis or a missing
    material factor (planted mistakes, not committed) fail it."""
    coarse, fine = _energy_rel_error(4), _energy_rel_error(8)
    assert max(abs(v) for v in coarse) < 2.5e-3, coarse
    assert max(abs(v) for v in fine) < 5e-4, fine


@pytest.mark.parametrize("face, expect", [(PEC, -1.0), (PMC, 1.0)])
def test_pec_pmc_reflection_sign(face, expect):
    """At normal incidence a PEC wall reflects E with coefficient -1 (tangential E vanishes
    there) and a PMC wall with +1 (tangential H vanishes, so E doubles).  A Gaussian E_x pulse of
    12 cells with H = 0 splits into two halves of amplitude 1/2; the upward half is probed
    before and after the z+ face: 1/2 within 0.5 %, ratio within 1 % (measured 0.08 % and
    0.07 %, and 0.02 % at 20 cells)."""
    h, wc = 1e-3, 12
    gap = 4 * wc
    k0 = gap + 10
    nz = k0 + 2 * gap
    dt = oracle.dt_cfl(0.95, h, h, h)
    b = oracle.Block((4, 4, nz), (h,) * 3, dt, (PEC, PEC, PEC, PEC, ABSORBING, face))
    oracle.connect(b, 0, b, 1)
    oracle.connect(b, 2, b, 3)
    shp = b.shape(EX)
    z = np.arange(shp[0]) * h
    pulse = np.exp(-((z - k0 * h) / (wc * h)) ** 2)
    b.set_field(EX, np.ascontiguousarray(pulse[:, None, None] * np.ones(shp)))
    b.add_probe(EX, 1, 1, k0 + gap)
    v = 299792458.0 * dt
    steps = int(3.0 * gap * h / v)
    b.reserve_probes(steps)
    oracle.step([b], steps)
    p = b.probes()[0]
    mid = int(2 * gap * h / v)                    # between the incident and reflected passes
    inc = p[:mid][np.argmax(np.abs(p[:mid]))]
    ref = p[mid:][np.argmax(np.abs(p[mid:]))]
    assert abs(inc - 0.5) < 0.0025, inc
    assert abs(ref / inc - expect) < 0.01, ref / inc
