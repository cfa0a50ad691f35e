"""Phase-shifted periodic SAT on the GPU (complex pair of simulations) against the oracle,
and the GPU dispersion tool against the oracle's amplification matrix and errors."""
import math

import numpy as np
import pytest

from paper_2206_00638_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from oracle import dispersion as odsp  # noqa: E402
from paper_2206_00638_gb300 import dispersion as gdsp  # noqa: E402
from paper_2206_00638_gb300 import sbpsat  # noqa: E402

TOL = {sbpsat.FP32: 1e-5, sbpsat.FP64: 1e-11}


def _pair_run(n, h, alphas, faces, steps, precision, seed):
    rng = np.random.default_rng(seed)
    eps = rng.uniform(1, 4, (n[2], n[1], n[0])).astype(np.float32)
    fields = [[rng.uniform(-1, 1, wl.field_shape(n, c)) * (1.0 if c < 3 else 1 / 377.0) for c in range(6)]
              for _ in range(2)]
    sims = [sbpsat.Sim(n, h, faces, eps_r=eps, cfl=0.95, precision=precision) for _ in range(2)]
    dt = sims[0].dt
    blks = [oracle.Block(n, h, dt, faces, eps_r=eps) for _ in range(2)]
    for part in range(2):
        for c in range(6):
            sims[part].set_field(c, fields[part][c])
            blks[part].set_field(c, fields[part][c])
    for a, al in enumerate(alphas):
        if al is not None:
            sbpsat.connect_phase(sims[0], sims[1], a, al)
            oracle.connect_phase(blks[0], blks[1], a, al)
    sbpsat.step_group(sims, steps)
    oracle.step(blks, steps)
    worst = 0.0
    for comps in ((0, 1, 2), (3, 4, 5)):
        num = sum(np.sum(np.abs((sims[0].field(c) + 1j * sims[1].field(c)) -
                                (blks[0].field(c) + 1j * blks[1].field(c))) ** 2) for c in comps)
        den = sum(np.sum(np.abs(blks[0].field(c) + 1j * blks[1].field(c)) ** 2) for c in comps)
        worst = max(worst, math.sqrt(num / den))
    for s in sims:
        s.close()
    return worst


@pytest.mark.parametrize("precision", [sbpsat.FP64, sbpsat.FP32])
@pytest.mark.parametrize("n", [(37, 26, 19), (6, 5, 7)])
def test_phase_pbc_all_axes_vs_oracle(n, precision):
    """Phase shifts on all three axes, random eps_r and complex fields (one-pass path for
    the larger grid, in-place path for the small one)."""
    err = _pair_run(n, (1e-3, 1.2e-3, 0.9e-3), (0.7, -1.9, 2.8), (0,) * 6, 120, precision, 3)
    assert err < TOL[precision], err


@pytest.mark.parametrize("precision", [sbpsat.FP64, sbpsat.FP32])
def test_phase_pbc_one_axis_with_walls(precision):
    """Periodic with phase along y only; PEC, PMC and absorbing walls elsewhere."""
    faces = (wl.PEC, wl.ABSORBING, 0, 0, wl.PMC, wl.ABSORBING)
    err = _pair_run((30, 22, 17), (1e-3,) * 3, (None, 1.1, None), faces, 120, precision, 4)
    assert err < TOL[precision], err


def test_dispersion_tool_matches_oracle():
    """The GPU-built amplification matrix (FP64) equals the oracle's, and the numerical
    wavenumber and errors derived from it agree."""
    h, cfl, n = 1e-3, 0.99, (4, 4, 4)
    k0h, theta, phi = 2 * math.pi / 20, 0.7, 0.4
    k0 = k0h / h
    alphas = gdsp.direction_phases(k0, (h,) * 3, n, theta, phi)
    lam_g, dt = gdsp.amplification_matrix(n, (h,) * 3, cfl, alphas)
    lam_o = odsp.sbp_lambda(n, (h,) * 3, dt, alphas)
    assert np.max(np.abs(lam_g - lam_o)) < 1e-11 * np.max(np.abs(lam_o))
    res = gdsp.analyse(k0h, theta, phi, n=n, h=h, cfl=cfl)
    kt_o, (d_o, x_o, g_o), _ = odsp.analyse("sbp", n, h, cfl, k0h, theta, phi)
    assert abs(res["k_numerical"] - kt_o) < 1e-8 * k0
    assert abs(res["dispersion"] - d_o) < 1e-6 and abs(res["global"] - g_o) < 1e-6
    assert res["dissipation"] < 1e-8
