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


@pytest.mark.parametrize("precision", [sbpsat.FP32, sbpsat.FP32_FP16STORE])
@pytest.mark.parametrize("n", [(70, 43, 37), (33, 20, 17), (65, 100, 24)])
def test_sixteen_row_tiles_bitwise_equal_eight_rows(precision, n, monkeypatch):
    """The 16-row tile (512 threads, one CTA per SM) computes every node with the same
    formula as the 8-row tile: fields and probes bit-identical, ragged last rows included."""
    w = wl.random_box(n, faces=(A, P, M, A, P, M), seed=19, steps=29)
    monkeypatch.setenv("SBP_FUSED_WIDTH", "64")
    monkeypatch.setenv("SBP_FUSED_ROWS", "16")
    big = sbpsat.from_workload(w, precision=precision)[0]
    monkeypatch.setenv("SBP_FUSED_ROWS", "8")
    small = sbpsat.from_workload(w, precision=precision)[0]
    assert big.tile()[0] == 16 and small.tile()[0] == 8
    for s in (big, small):
        s.reserve_probes(29)
        s.step(29)
    for c in range(6):
        assert np.array_equal(big.field(c), small.field(c)), c
    assert np.array_equal(big.probes(), small.probes())
    big.close()
    small.close()


@pytest.mark.parametrize("precision", [sbpsat.FP32, sbpsat.FP32_FP16STORE])
@pytest.mark.parametrize("rows", [8, 12])
@pytest.mark.parametrize("n", [(70, 43, 37), (140, 30, 21), (300, 26, 13), (8, 9, 10)])
def test_wide_tiles_bitwise_equal_narrow_tiles(precision, rows, n, monkeypatch):
    """128-column tiles (two warps per row) compute every node with the same formula as
    the 64-column tile: fields and probes bit-identical, with ragged last columns and rows,
    tiles wider than the grid, and a grid three tiles wide."""
    w = wl.random_box(n, faces=(A, P, M, A, P, M), seed=23, steps=31)
    monkeypatch.setenv("SBP_FUSED_WIDTH", "128")
    monkeypatch.setenv("SBP_FUSED_ROWS", str(rows))
    wide = sbpsat.from_workload(w, precision=precision)[0]
    monkeypatch.setenv("SBP_FUSED_WIDTH", "64")
    monkeypatch.setenv("SBP_FUSED_ROWS", "8")
    narrow = sbpsat.from_workload(w, precision=precision)[0]
    assert wide.tile()[2] == 128 and wide.tile()[0] == rows and narrow.tile()[2] == 64
    for s in (wide, narrow):
        s.reserve_probes(31)
        s.step(31)
    for c in range(6):
        assert np.array_equal(wide.field(c), narrow.field(c)), c
    assert np.array_equal(wide.probes(), narrow.probes())
    wide.close()
    narrow.close()


def test_autotune_reports_tile():
    w = wl.random_box((140, 48, 44), seed=3, steps=4)
    s = sbpsat.from_workload(w)[0]
    depth, _ = s.autotune(2)
    rows, d2, width = s.tile()
    assert (width, rows) in ((64, 8), (64, 16), (128, 8), (128, 12)) and d2 == depth
    s.close()


def test_autotune_of_joined_blocks_changes_nothing():
    """Blocks joined by the interface SAT can be tuned: the tuned group steps bit-identically
    to an untuned copy, and the partner's fields are untouched by the trials."""
    w = wl.two_block(nxy=40, nz=24, steps=30)
    tuned = sbpsat.from_workload(w)
    plain = sbpsat.from_workload(w)
    for g in (tuned, plain):
        for s in g:
            s.reserve_probes(30)
        sbpsat.step_group(g, 5)
    before = [tuned[1].field(c) for c in range(6)]
    depth, ms = tuned[0].autotune(2)
    assert depth >= 8 and ms > 0 and tuned[0].step_index == 5
    for c in range(6):
        assert np.array_equal(tuned[1].field(c), before[c]), c
    for g in (tuned, plain):
        sbpsat.step_group(g, 25)
    for a, b in zip(tuned, plain):
        for c in range(6):
            assert np.array_equal(a.field(c), b.field(c)), c
        assert np.array_equal(a.probes(), b.probes())
    for s in tuned + plain:
        s.close()
