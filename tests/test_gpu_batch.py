"""Batched stepping (continuous batching): every grid gives the same result alone and in the mix."""
import numpy as np
import pytest

from paper_2206_00638_gb300 import workloads as wl
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_00638_gb300 import sbpsat  # noqa: E402

P, M, A = wl.PEC, wl.PMC, wl.ABSORBING
SIZES = [(33, 20, 17), (8, 8, 8), (64, 48, 40), (19, 41, 23), (70, 12, 9)]
FACES = [(P,) * 6, (A, P, M, A, P, M), (A,) * 6, (M, M, P, P, A, A), (P, A, P, A, P, A)]
STEPS = [61, 40, 77, 52, 33]


def _workloads():
    return [wl.random_box(n, faces=f, seed=30 + q, steps=st) for q, (n, f, st) in enumerate(zip(SIZES, FACES, STEPS))]


@pytest.mark.parametrize("use_graphs, persistent", [(True, True), (False, True), (True, False), (False, False)])
def test_batch_equals_alone_bitwise(use_graphs, persistent):
    ws = _workloads()
    alone = []
    for w in ws:
        s = parity.gpu_run(w, w.steps, sbpsat.FP32)[0]
        alone.append(([s.field(c) for c in range(6)], s.probes()))
        s.close()
    stream = torch.cuda.current_stream()
    batch = sbpsat.Batch(stream=stream, use_graphs=use_graphs, persistent=persistent)
    sims = []
    for w in ws:
        s = sbpsat.from_workload(w, stream=stream)[0]
        s.reserve_probes(w.steps)
        batch.add(s, w.steps)
        sims.append(s)
    # uneven chunks, members finish inside chunks; a member joins late
    late = sims.pop()
    batch.remove(late)
    batch.step(16)
    batch.add(late, ws[-1].steps)
    sims.append(late)
    for k in (16, 16, 10, 16, 16, 16):
        batch.step(k)
    for s, w in zip(sims, ws):
        assert batch.remaining(s) == 0, (s.n, batch.remaining(s))
        assert s.step_index == w.steps
    for (fields, probes), s in zip(alone, sims):
        for c in range(6):
            assert np.array_equal(fields[c], s.field(c)), (s.n, c)
        assert np.array_equal(probes, s.probes())
    batch.close()
    for s in sims:
        s.close()


def test_batch_matches_oracle():
    ws = _workloads()[:3]
    stream = torch.cuda.current_stream()
    batch = sbpsat.Batch(stream=stream)
    sims = []
    for w in ws:
        s = sbpsat.from_workload(w, stream=stream)[0]
        batch.add(s, w.steps)
        sims.append(s)
    batch.step(max(w.steps for w in ws))
    for s, w in zip(sims, ws):
        blocks = parity.oracle_run(w, w.steps, s.dt)
        err = parity.compare([s], blocks)[0]
        assert max(err) < 1e-5, (w.name, err)
    batch.close()


def test_batch_energy_monitor_matches_alone():
    """Members with the FP64 energy monitor: sampled at the chunk boundaries whose step is a
    multiple of energy_every (here every chunk of 16 steps), the series is the one the member
    gives alone (every 16th step), bit for bit, and the fields stay bit-identical."""
    ws = _workloads()[:3]
    steps = 64
    alone = []
    for w in ws:
        s = parity.gpu_run(w, steps, sbpsat.FP32, energy_every=16)[0]
        series, rc = s.energy_series()
        alone.append(([s.field(c) for c in range(6)], series))
        s.close()
    stream = torch.cuda.current_stream()
    batch = sbpsat.Batch(stream=stream, use_graphs=True)
    sims = []
    for w in ws:
        s = sbpsat.from_workload(w, stream=stream, energy_every=16)[0]
        s.reserve_probes(steps)
        batch.add(s, steps)
        sims.append(s)
    for _ in range(steps // 16):
        batch.step(16)
    torch.cuda.synchronize()
    for s, (fields, series) in zip(sims, alone):
        got, rc = s.energy_series()
        # alone samples at the monitored steps 0, 16, 32, 48; the batch also at its last
        # chunk boundary, step 64
        assert len(series) == steps // 16 and len(got) == steps // 16 + 1
        assert np.array_equal(got[:-1], series)
        for c in range(6):
            assert np.array_equal(s.field(c), fields[c]), c
    batch.close()
    for s in sims:
        s.close()
