"""The FDTD comparator mode of the GPU kernels (SBP_FLAG_FDTD) against the oracle's Yee
scheme, and its restrictions."""
import math

import numpy as np
import pytest

from paper_2206_00638_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import fdtd  # noqa: E402
from paper_2206_00638_gb300 import sbpsat  # noqa: E402

P = wl.PEC


def _run(n, steps, precision, seed):
    w = wl.random_box(n, faces=(P,) * 6, seed=seed, steps=steps)
    b = w.blocks[0]
    sim = sbpsat.Sim(b.n, b.h, b.faces, eps_r=b.eps_r, cfl=w.cfl, precision=precision, flags=sbpsat.FLAG_FDTD)
    ref = fdtd.Yee(b.n, b.h, sim.dt, eps_r=b.eps_r)
    for c in range(6):
        sim.set_field(c, b.fields[c])
        ref.F[c][...] = b.fields[c]
    for s in b.sources:
        sim.add_source(s.comp, s.i, s.j, s.k, s.kind, s.amp, s.tw, s.t0, s.f)
        ref.add_source(s.comp, s.i, s.j, s.k, s.kind, s.amp, s.tw, s.t0, s.f)
    probes = [(p.comp, p.i, p.j, p.k) for p in b.probes]
    for p in b.probes:
        sim.add_probe(p.comp, p.i, p.j, p.k)
    sim.reserve_probes(steps)
    sim.step(steps)
    rp = ref.step(steps, probes)
    errs = []
    for comps in ((0, 1, 2), (3, 4, 5)):
        num = sum(np.sum((sim.field(c).astype(np.float64) - ref.F[c]) ** 2) for c in comps)
        den = sum(np.sum(ref.F[c] ** 2) for c in comps)
        errs.append(math.sqrt(num / den))
    gp = sim.probes()
    perr = np.max(np.abs(gp - rp.T)) / np.max(np.abs(rp))
    sim.close()
    return errs, perr


@pytest.mark.parametrize("n", [(70, 43, 37), (8, 9, 8)])
def test_fdtd_mode_vs_oracle_yee(n):
    errs, perr = _run(n, 150, sbpsat.FP32, 11)
    assert max(errs) < 1e-5, errs
    assert perr < 1e-4


def test_fdtd_mode_fp16_storage():
    errs, _ = _run((40, 33, 29), 150, sbpsat.FP32_FP16STORE, 12)
    assert max(errs) < 4 * 2 ** -11 * math.sqrt(151), errs


def test_fdtd_mode_restrictions():
    n, h = (12, 10, 9), (1e-3,) * 3
    with pytest.raises(sbpsat.SbpError):
        sbpsat.Sim(n, h, (P, P, P, P, P, wl.ABSORBING), flags=sbpsat.FLAG_FDTD)
    with pytest.raises(sbpsat.SbpError):
        sbpsat.Sim(n, h, (P,) * 6, precision=sbpsat.FP64, flags=sbpsat.FLAG_FDTD)
    s = sbpsat.Sim(n, h, (P,) * 6, flags=sbpsat.FLAG_FDTD)
    with pytest.raises(sbpsat.SbpError):
        s.energy()
    s.close()
