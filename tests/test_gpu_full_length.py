"""Full-length parity: every block workload against the FP64 oracle over its full step count
(or, where the oracle would take too long for the suite, at full size over part of the run
and at reduced size over the whole run).  FP32 tolerance: relative L2 error per field
(E and H, each over its three components) <= 1e-5; FP16 storage: <= 4 u sqrt(N + 1) with
u = 2^-11 (the bound of the FP16 tests).  The oracle runs on the host cores (OpenMP)."""
import math

import numpy as np
import pytest

import oracle

from paper_2206_00638_gb300 import workloads as wl
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_00638_gb300 import sbpsat  # noqa: E402

FP32_TOL = 1e-5
U16 = 2.0 ** -11


def _gpu(w, steps, precision, autotune=False):
    sims = sbpsat.from_workload(w, precision=precision)
    if autotune:
        for s in sims:
            depth, _ = s.autotune(3)
            assert depth > 0
    for s in sims:
        s.reserve_probes(steps)
    if len(sims) == 1:
        sims[0].step(steps)
    else:
        sbpsat.step_group(sims, steps)
    return sims


def _check(sims, blocks, tol, ptol):
    errs = parity.compare(sims, blocks)
    perr = parity.probe_error(sims, blocks)
    for s in sims:
        s.close()
    print("relative L2 error per field (E, H) per block:", errs, "probe error:", perr)
    for e in errs:
        assert max(e) < tol, errs
    assert perr < ptol, perr
    return errs


def test_dielectric_cube_128_full_2000_steps():
    """The 256^3 dielectric-cube workload scaled to 128^3 (same h, cube and source scaled),
    over its full 2000 steps."""
    w = wl.dielectric(N=128, steps=2000)
    sims = _gpu(w, w.steps, sbpsat.FP32)
    blocks = parity.oracle_run(w, w.steps, sims[0].dt)
    _check(sims, blocks, FP32_TOL, 1e-4)


def test_dielectric_cube_256_full_size_500_steps():
    """The 256^3 dielectric-cube workload at full size in the benchmark's launch
    configuration (autotuned z-block depth) over its first 500 steps: the pulse has left
    the source and crossed the dielectric cube's near face."""
    w = wl.dielectric(N=256, steps=500)
    sims = _gpu(w, w.steps, sbpsat.FP32, autotune=True)
    blocks = parity.oracle_run(w, w.steps, sims[0].dt)
    _check(sims, blocks, FP32_TOL, 1e-4)


def test_two_block_interface_full_size_full_3000_steps():
    """Two 192x192x96 blocks joined on z by the interface SAT, absorbing outer faces, eps_r
    patches, Ex Gaussian sheet: full size, all 3000 steps, both blocks, every field.

    The absorbing faces drain the pulse: after 3000 steps ||E|| is about 1/700 of its peak.
    The FP32 path's absolute error stops growing once the pulse has been absorbed (about
    2e-5 V/m for ||E|| of 56 V/m at its peak, measured on GB300), so its error relative to the
    remaining field grows as that field decays (2.5e-4 at step 3000).  The bound is therefore
    taken against the field's peak norm over the run: ||gpu - oracle|| <= 1e-5 max_t ||F(t)||
    per field at every checkpoint, and the absolute error may not grow once the field is
    decaying (no instability hides behind the decay)."""
    w = wl.two_block()
    assert w.steps == 3000
    sims = sbpsat.from_workload(w, precision=sbpsat.FP32)
    blocks = parity.oracle_blocks(w, sims[0].dt)
    peak = None
    abs_at = []
    done = 0
    for chunk in (250, 250, 500, 500, 500, 500, 500):
        sbpsat.step_group(sims, chunk)
        oracle.step(blocks, chunk)
        done += chunk
        errs, norms = [], []
        for s, b in zip(sims, blocks):
            for comps in ((0, 1, 2), (3, 4, 5)):
                errs.append(math.sqrt(sum(float(np.sum((s.field(c).astype(np.float64) - b.field(c)) ** 2))
                                          for c in comps)))
                norms.append(math.sqrt(sum(float(np.sum(b.field(c) ** 2)) for c in comps)))
        peak = norms if peak is None else [max(a, b) for a, b in zip(peak, norms)]
        print(f"step {done}: error {errs}, norm {norms}, peak {peak}")
        for e, pk in zip(errs, peak):
            assert e <= FP32_TOL * pk, (done, errs, peak)
        abs_at.append(errs)
    assert done == 3000
    # from step 1000 on (the pulse has left; the field decays) the absolute error does not grow
    for q in range(len(abs_at[0])):
        series = [a[q] for a in abs_at[2:]]
        assert max(series[1:]) <= 1.2 * series[0], series
    for s in sims:
        s.close()


def test_mixed_faces_128_copy_full_1000_steps_fp32_and_fp16():
    """The 512^3 mixed-faces workload's 128^3 copy (same h, geometry x 1/4) over its full
    1000 steps: FP32 within 1e-5 and FP16 storage within its bound, against one oracle run."""
    w = wl.mixed_faces(N=128, steps=1000)
    s32 = _gpu(w, w.steps, sbpsat.FP32)
    blocks = parity.oracle_run(w, w.steps, s32[0].dt)
    _check(s32, blocks, FP32_TOL, 1e-4)
    s16 = _gpu(w, w.steps, sbpsat.FP32_FP16STORE)
    bound = 4.0 * U16 * math.sqrt(w.steps + 1)
    _check(s16, blocks, bound, 2 * bound)
