"""Checkpoint / resume, failure detection without a GPU fault, and the autotuner's
result file."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2206_00638_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_00638_gb300 import sbpsat  # noqa: E402
from tests import parity  # noqa: E402

P, M, A = wl.PEC, wl.PMC, wl.ABSORBING
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("precision", [sbpsat.FP32, sbpsat.FP32_FP16STORE, sbpsat.FP64])
def test_checkpoint_resume_bitwise(precision):
    """N steps equal k steps, save, load into a fresh simulation, N - k steps: fields,
    probe series and (FP64) the energy series bit for bit."""
    w = wl.random_box((40, 33, 29), faces=(A, P, M, A, P, M), seed=17, steps=60)
    ev = 5 if precision == sbpsat.FP64 else 0
    ref = sbpsat.from_workload(w, precision=precision, energy_every=ev)[0]
    ref.reserve_probes(60)
    ref.step(60)
    a = sbpsat.from_workload(w, precision=precision, energy_every=ev)[0]
    a.reserve_probes(60)
    a.step(25)
    blob = a.save()
    a.close()
    b = sbpsat.from_workload(w, precision=precision, energy_every=ev)[0]
    b.reserve_probes(60)
    b.load(blob)
    assert b.step_index == 25
    b.step(35)
    for c in range(6):
        assert np.array_equal(b.field(c), ref.field(c)), c
    assert np.array_equal(b.probes(), ref.probes())
    if ev:
        sr, _ = ref.energy_series()
        sb, _ = b.energy_series()
        assert np.array_equal(sr, sb)
    ref.close()
    b.close()


def test_load_rejects_other_grid():
    w1 = wl.random_box((20, 18, 16), seed=1, sources=False)
    w2 = wl.random_box((20, 18, 17), seed=1, sources=False)
    s1 = sbpsat.from_workload(w1)[0]
    s2 = sbpsat.from_workload(w2)[0]
    blob = s1.save()
    with pytest.raises(sbpsat.SbpError):
        s2.load(blob)
    s1.close()
    s2.close()


def test_pipeline_wait_timeout_is_reported_and_context_survives():
    """Bounded waits: with the test hook the one-pass step loads no planes, every wait
    gives up after its limit, and the host sees SBP_ETIMEOUT; the context stays usable."""
    w = wl.random_box((40, 33, 29), faces=(P,) * 6, seed=2, steps=3, sources=False)
    b = w.blocks[0]
    s = sbpsat.Sim(b.n, b.h, b.faces, eps_r=b.eps_r, flags=sbpsat.FLAG_TEST_WAIT_TIMEOUT)
    s.step(3)
    with pytest.raises(sbpsat.SbpError) as err:
        s.sync()
    assert err.value.code == -5
    s.close()
    # the device still works: a normal run matches the oracle
    w2 = wl.random_box((30, 22, 17), faces=(P, A, M, P, A, M), seed=3, steps=40)
    sims = parity.gpu_run(w2, 40, sbpsat.FP32)
    blocks = parity.oracle_run(w2, 40, sims[0].dt)
    assert max(parity.compare(sims, blocks)[0]) < 1e-5


def test_autotune_result_file(tmp_path):
    """SBP_TUNE_CACHE: a tuning appends its choice as a JSON line keyed by shape and
    precision, and a later process reads it back."""
    path = tmp_path / "tune.jsonl"
    env = dict(os.environ, SBP_TUNE_CACHE=str(path))
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2206_00638_gb300 import sbpsat, workloads as wl\n"
            "s = sbpsat.from_workload(wl.random_box((70, 43, 61), seed=5, sources=False))[0]\n"
            "d, ms = s.autotune(2)\n"
            "print(*s.tile())\n" % ROOT)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    tile_rows, depth, width = (int(v) for v in out.stdout.strip().splitlines()[-1].split())
    lines = [json.loads(l) for l in path.read_text().splitlines() if l.strip()]
    assert {"nx": 70, "ny": 43, "nz": 61, "precision": 0, "depth": depth, "rows": tile_rows,
            "width": width} in lines
    # a later process creates the same shape with the tuned tile
    code2 = ("import sys; sys.path.insert(0, %r)\n"
             "from paper_2206_00638_gb300 import sbpsat, workloads as wl\n"
             "s = sbpsat.from_workload(wl.random_box((70, 43, 61), seed=5, sources=False))[0]\n"
             "print(*s.tile())\n" % ROOT)
    out2 = subprocess.run([sys.executable, "-c", code2], env=env, capture_output=True, text=True, timeout=300)
    assert out2.returncode == 0, out2.stderr
    assert out2.stdout.strip().splitlines()[-1].split() == [str(tile_rows), str(depth), str(width)]
