"""The FP16-storage tolerance of the GPU tests, 4 u sqrt(N+1) with u = 2^-11, checked on the 1D
reduction of the scheme (dense printed matrices, tests/ref1d.py) on the CPU.

Fields stored as value/scale in FP16 and rounded after every update (E with scale 1 V/m, H with
1/eta0 A/m), arithmetic in FP64, against the same scheme in FP64.  The bound assumes that the
rounding errors of N steps add like a random walk because the scheme neither damps nor
amplifies them (energy conserved, or decreasing with absorbing faces)."""
import math

import numpy as np
import pytest

from tests import ref1d

U16 = 2.0 ** -11
ETA0 = 376.730313668


def _bound(nsteps):
    return 4.0 * U16 * math.sqrt(nsteps + 1)


def _store(x, scale):
    return np.asarray(x / scale, dtype=np.float16).astype(np.float64) * scale


def _fp16_errors(nsteps, faces, nz=200, seed=1):
    h = 1e-3
    dt = 0.95 * h / 299792458.0
    eps = np.where(np.arange(nz) < nz // 2, 1.0, 3.0)
    ref = ref1d.Pair1D(nz, h, dt, faces[0], faces[1], eps_cells=eps)
    rng = np.random.default_rng(seed)
    e0 = rng.uniform(-1, 1, nz + 1)
    h0 = rng.uniform(-1, 1, nz + 2) / ETA0
    ref.E, ref.H = e0.copy(), h0.copy()
    sE, sH = 1.0, 1.0 / ETA0
    E, H = _store(e0, sE), _store(h0, sH)
    gE, gH = ref.gE, ref.gH
    for _ in range(nsteps):
        H = _store(((1 - 0.5 * dt * gH) * H + dt * (ref.AH @ E)) / (1 + 0.5 * dt * gH), sH)
        E = _store(((1 - 0.5 * dt * gE) * E + dt * (ref.AE @ H)) / (1 + 0.5 * dt * gE), sE)
    ref.step(nsteps)
    return (np.linalg.norm(E - ref.E) / np.linalg.norm(ref.E),
            np.linalg.norm(H - ref.H) / np.linalg.norm(ref.H))


@pytest.mark.parametrize("faces", [(ref1d.PEC, ref1d.PMC), (ref1d.ABSORBING, ref1d.PEC)])
def test_fp16_storage_error_within_bound_and_grows_like_sqrt_n(faces):
    """Relative L2 errors of E and H at 150 and 2000 steps stay below the bound (measured
    0.17-0.20 of it) and grow like sqrt(N): x3.0-3.9 from 150 to 2000 steps, where linear growth
    would be x13.3."""
    short = _fp16_errors(150, faces)
    long = _fp16_errors(2000, faces)
    assert max(short) < _bound(150), short
    assert max(long) < _bound(2000), long
    assert min(short) > 0.05 * _bound(150)           # the rounding is really there
    growth = max(long) / max(short)
    assert growth < 6.0, (short, long)
