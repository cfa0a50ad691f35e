"""sbp_energy_noalloc: the energy entry point for callers that must not allocate device memory.

It must give the same W^n as sbp_energy, bit for bit (same kernels, same fixed reduction
order), while keeping its partial sums in the library's fixed array.  Two calls in a row
check that the array's leftover contents from one call do not leak into the next.  This file
is collected last so that a run stopping at the first failure has already run every other
test."""

import numpy as np
import pytest

from paper_2206_00638_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_00638_gb300 import sbpsat  # noqa: E402

P, M, A = wl.PEC, wl.PMC, wl.ABSORBING
EINVAL, ECAPACITY = -1, -8


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
        assert float(out.item()) == ref
    # a different grid between the two calls reuses the same array
    w2 = wl.random_box((20, 18, 25), faces=(P,) * 6, seed=3, steps=5, sources=False)
    other = sbpsat.from_workload(w2, precision=precision)[0]
    ref2 = other.energy()
    other.energy_noalloc(out)
    other.sync()
    assert float(out.item()) == ref2
    sim.energy_noalloc(out)
    sim.sync()
    assert float(out.item()) == ref
    other.close()
    sim.close()


def test_noalloc_checks_arguments():
    w = wl.random_box((12, 10, 9), seed=1, sources=False)
    sim = sbpsat.from_workload(w)[0]
    L = sbpsat.lib()
    assert L.sbp_energy_noalloc(sim.handle, None) == EINVAL
    # a host pointer is refused and left untouched
    host = np.full(1, 7.0)
    assert L.sbp_energy_noalloc(sim.handle, host.ctypes.data) == EINVAL
    assert host[0] == 7.0
    # a misaligned device pointer is refused
    buf = torch.zeros(4, dtype=torch.float64, device="cuda")
    assert L.sbp_energy_noalloc(sim.handle, buf.data_ptr() + 4) == EINVAL
    for bad in (torch.zeros(1, dtype=torch.int64, device="cuda"), torch.zeros(0, dtype=torch.float64, device="cuda"),
                torch.zeros(1, dtype=torch.float64)):
        with pytest.raises(ValueError):
            sim.energy_noalloc(bad)
    sim.close()


def test_noalloc_refuses_grids_beyond_the_array(monkeypatch):
    """A thin grid split into 2-plane z-chunks (SBP_KCHUNK=2) needs 1 x 2 x 32769 = 65538
    partial sums, two more than the array holds: SBP_ECAPACITY, nothing written."""
    monkeypatch.setenv("SBP_KCHUNK", "2")
    sim = sbpsat.Sim((4, 8, 65536), (1e-3,) * 3, (P,) * 6)
    monkeypatch.delenv("SBP_KCHUNK")
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    assert sbpsat.lib().sbp_energy_noalloc(sim.handle, out.data_ptr()) == ECAPACITY
    sim.sync()
    assert torch.isnan(out).all()
    sim.close()
