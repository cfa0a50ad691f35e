"""FP16 field storage (FP32 arithmetic, one scale for E and one for H): parity with the
FP64 oracle within the FP16 bound, bit-identical one-pass and in-place paths, the FP64
energy monitor on stored values, and the field round trip.

Bound.  Every update rounds each stored value to nearest in FP16, a relative error of
at most u = 2^-11.  The leapfrog scheme with these SATs neither damps nor amplifies a
perturbation (its discrete energy is conserved or decays), so the roundings of N steps
add up like a random walk: the relative L2 error per field stays below
c * u * sqrt(N + 1), with c = 4 covering the initial rounding of the inputs, the two
half-steps per step and the spread of the walk.
"""
import math

import numpy as np
import pytest

from paper_2206_00638_gb300 import workloads as wl
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_00638_gb300 import sbpsat  # noqa: E402

FP16 = sbpsat.FP32_FP16STORE
P, M, A = wl.PEC, wl.PMC, wl.ABSORBING
U16 = 2.0 ** -11


def fp16_bound(nsteps):
    return 4.0 * U16 * math.sqrt(nsteps + 1)


def _errors(w, steps, precision, **kw):
    sims = parity.gpu_run(w, steps, precision, **kw)
    blocks = parity.oracle_run(w, steps, sims[0].dt)
    errs = parity.compare(sims, blocks)
    perr = parity.probe_error(sims, blocks)
    for s in sims:
        s.close()
    return errs, perr


@pytest.mark.parametrize("faces", [(P, P, P, P, P, P), (M, M, M, M, M, M), (P, M, M, P, A, P), (A, A, A, A, A, A)])
def test_fp16_random_box_vs_oracle(faces):
    """Ragged box, random eps_r and fields, point + sheet sources, every face type."""
    w = wl.random_box((70, 43, 37), faces=faces, seed=11, steps=150)
    errs, perr = _errors(w, 150, FP16)
    assert max(errs[0]) < fp16_bound(150), errs
    assert perr < 2 * fp16_bound(150)


@pytest.mark.parametrize("n", [(70, 43, 37), (8, 8, 8), (9, 13, 10)])
def test_fp16_fused_bitwise_equals_in_place(n, monkeypatch):
    """FP16 one-pass step + band kernels == FP16 in-place half-steps, bit for bit: both
    round H^{n+1/2} to FP16 before E reads it."""
    w = wl.random_box(n, faces=(A, P, M, A, P, M), seed=21, steps=37)
    fused = parity.gpu_run(w, 37, FP16)[0]
    monkeypatch.setenv("SBP_NO_FUSED", "1")
    plain = parity.gpu_run(w, 37, FP16)[0]
    for c in range(6):
        assert np.array_equal(fused.field(c), plain.field(c)), c
    assert np.array_equal(fused.probes(), plain.probes())
    fused.close()
    plain.close()


def test_fp16_dielectric_2000_steps():
    """Dielectric-cube workload at 64^3 over its full 2000 steps."""
    w = wl.dielectric(N=64, steps=2000)
    errs, perr = _errors(w, 2000, FP16)
    assert max(errs[0]) < fp16_bound(2000), errs


def test_fp16_mixed_faces_128_copy():
    """The 512^3 mixed-face workload scaled to 128^3 (same h, geometry x 1/4): FP16 and
    FP32 storage against the FP64 oracle while the pulse crosses the box."""
    steps = 300
    w = wl.mixed_faces(N=128, steps=steps)
    e16, _ = _errors(w, steps, FP16)
    e32, _ = _errors(w, steps, sbpsat.FP32)
    assert max(e16[0]) < fp16_bound(steps), e16
    assert max(e32[0]) < 1e-5, e32


def test_fp16_energy_monitor():
    """PEC/PMC box without sources: the FP64 energy of the stored FP16 fields stays flat
    to the FP16 bound (and is not the FP32 energy times some scale)."""
    w = wl.random_box((40, 33, 29), faces=(P, P, M, M, P, M), seed=4, steps=300, sources=False)
    sim = sbpsat.from_workload(w, precision=FP16, energy_every=10)[0]
    W0 = sim.energy()
    ref = sbpsat.from_workload(w, precision=sbpsat.FP64)[0]
    assert W0 == pytest.approx(ref.energy(), rel=4 * U16)
    sim.step(300)
    series, rc = sim.energy_series()
    assert rc == 0 and len(series) == 30
    assert np.max(np.abs(series - W0)) / W0 < fp16_bound(300)
    sim.close()
    ref.close()


def test_fp16_field_roundtrip_and_scales():
    """Values exactly representable as FP16 * scale survive set/get unchanged, host and
    device, with default and with user scales."""
    n = (12, 10, 9)
    for scales in ((0.0, 0.0), (1e3, 2.5)):
        sim = sbpsat.Sim(n, (1e-3,) * 3, (P,) * 6, precision=FP16, field_scale=scales)
        sE = scales[0] or 1.0
        sH = scales[1] or 1.0 / math.sqrt(1.25663706212e-6 / 8.8541878128e-12)   # 1 / eta0
        sH = float(np.float32(sH))
        rng = np.random.default_rng(3)
        for c in range(6):
            s = sE if c < 3 else sH
            q = rng.integers(-2048, 2048, size=sim.shape(c)).astype(np.float32) / np.float32(256.0)
            vals = (q * np.float32(s)).astype(np.float32)
            sim.set_field(c, vals)
            assert np.array_equal(sim.field(c), vals), c
            t = torch.from_numpy(vals).cuda()
            sim.set_field(c, t)
            out = torch.empty_like(t)
            sim.field(c, out=out)
            torch.cuda.synchronize()
            assert torch.equal(out, t)
        sim.close()


def test_fp16_large_fields_with_scale():
    """Fields of 1e6 V/m overflow FP16 unscaled; with field_scale = (1e5, 1e5/377) the run
    matches the oracle within the FP16 bound."""
    w = wl.random_box((30, 22, 17), faces=(P, A, M, P, A, M), seed=9, steps=80, sources=False)
    for b in w.blocks:
        b.fields = [f * 1e6 for f in b.fields]
    errs, _ = _errors(w, 80, FP16, field_scale=(1e5, 1e5 / 377.0))
    assert max(errs[0]) < fp16_bound(80), errs


@pytest.mark.parametrize("faces", [(P, P, P, P, P, P), (M, M, M, M, M, M), (A, A, A, A, A, A), (P, M, M, P, A, P),
                                   (M, A, P, A, A, M)])
@pytest.mark.parametrize("steps", [1, 10])
def test_fp16_per_node_error_short_runs(faces, steps):
    """Node by node after 1 and 10 steps: |gpu - oracle| <= 4 u (N + 1) max |F| of that field
    (E or H).  Each update rounds once (<= u |F| / 2 per stored value) and a step mixes a node
    with neighbours through coefficients of order the CFL number, so a handful of u per step
    is the worst case.  A scale slip confined to boundary nodes (a wrong scale ratio in a SAT
    coefficient, say) changes those nodes by O(1) relative and fails here, while the L2 bound
    over the whole field would hide it."""
    w = wl.random_box((70, 43, 37), faces=faces, seed=17, steps=steps)
    sims = parity.gpu_run(w, steps, FP16)
    blocks = parity.oracle_run(w, steps, sims[0].dt)
    ref = [blocks[0].field(c) for c in range(6)]
    got = [sims[0].field(c).astype(np.float64) for c in range(6)]
    sims[0].close()
    for f in (0, 1):
        comps = range(3 * f, 3 * f + 3)
        scale = max(np.abs(ref[c]).max() for c in comps)
        for c in comps:
            err = np.abs(got[c] - ref[c]).max()
            assert err <= 4 * U16 * (steps + 1) * scale, (c, err / (U16 * scale))


def test_fp16_per_node_error_interface():
    """The same per-node bound across an interface SAT (two blocks joined on z)."""
    w = wl.coupled_boxes((30, 26, 20), (30, 26, 24), axis=2, facesA=(P, A, M, P, A, P),
                         facesB=(P, A, M, P, P, A), seed=5, steps=10)
    sims = parity.gpu_run(w, 10, FP16)
    blocks = parity.oracle_run(w, 10, sims[0].dt)
    for s, b in zip(sims, blocks):
        ref = [b.field(c) for c in range(6)]
        got = [s.field(c).astype(np.float64) for c in range(6)]
        for f in (0, 1):
            comps = range(3 * f, 3 * f + 3)
            scale = max(np.abs(ref[c]).max() for c in comps)
            for c in comps:
                assert np.abs(got[c] - ref[c]).max() <= 4 * U16 * 11 * scale, c
    for s in sims:
        s.close()
