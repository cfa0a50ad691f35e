"""sbp_energy_noalloc: the energy entry point for callers that must not allocate device memory.

It must give the same W^n as sbp_energy (same kernels, same fixed reduction order) while
keeping its partial sums in the library's fixed array.  Two calls in a row check that the
array's leftover contents from one call do not leak into the next.  This file is collected
last so that a run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

from paper_2206_00638_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_00638_gb300 import sbpsat  # noqa: E402

P, M, A = wl.PEC, wl.PMC, wl.ABSORBING


@pytest.mark.parametrize("precision", [sbpsat.FP64, sbpsat.FP32])
def test_noalloc_energy_matches_energy_twice(precision):
    w = wl.random_box((41, 30, 27), faces=(P, M, A, P, M, A), seed=13, steps=40)
    sim = sbpsat.from_workload(w, precision=precision)[0]
    sim.step(40)
    ref = sim.energy()
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        sim.energy_noalloc(out)
        sim.sync()
        got = float(out.item())
        assert got == pytest.approx(ref, rel=1e-12)
    # a different grid between the two calls reuses the same array
    w2 = wl.random_box((20, 18, 25), faces=(P,) * 6, seed=3, steps=5, sources=False)
    other = sbpsat.from_workload(w2, precision=precision)[0]
    ref2 = other.energy()
    other.energy_noalloc(out)
    other.sync()
    assert float(out.item()) == pytest.approx(ref2, rel=1e-12)
    sim.energy_noalloc(out)
    sim.sync()
    assert float(out.item()) == pytest.approx(ref, rel=1e-12)
    other.close()
    sim.close()


def test_noalloc_checks_arguments():
    w = wl.random_box((12, 10, 9), seed=1, sources=False)
    sim = sbpsat.from_workload(w)[0]
    assert sbpsat.lib().sbp_energy_noalloc(sim.handle, None) == -1
    sim.close()
