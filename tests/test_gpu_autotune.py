"""The z-block depth autotuner: trial steps leave the simulation unchanged, and the
chosen depth changes only which CTA computes a node, not the arithmetic."""
import numpy as np
import pytest

from paper_2206_00638_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_00638_gb300 import sbpsat  # noqa: E402

P, M, A = wl.PEC, wl.PMC, wl.ABSORBING


@pytest.mark.parametrize("precision", [sbpsat.FP32, sbpsat.FP32_FP16STORE])
def test_autotune_state_unchanged_and_results_identical(precision):
    w = wl.random_box((70, 43, 61), faces=(A, P, M, A, P, M), seed=13, steps=40)
    tuned = sbpsat.from_workload(w, precision=precision)[0]
    plain = sbpsat.from_workload(w, precision=precision)[0]
    for s in (tuned, plain):
        s.reserve_probes(40)
        s.step(3)
    before = [tuned.field(c) for c in range(6)]
    depth, ms = tuned.autotune(2)
    assert depth >= 8 and ms > 0
    assert tuned.step_index == 3
    for c in range(6):
        assert np.array_equal(tuned.field(c), before[c]), c
    tuned.step(37)
    plain.step(37)
    for c in range(6):
        assert np.array_equal(tuned.field(c), plain.field(c)), c
    assert np.array_equal(tuned.probes(), plain.probes())
    tuned.close()
    plain.close()


def test_autotune_rejects_ineligible():
    w = wl.random_box((12, 10, 9), seed=1, sources=False)
    s = sbpsat.from_workload(w, precision=sbpsat.FP64)[0]
    with pytest.raises(sbpsat.SbpError):
        s.autotune(1)
    s.close()
