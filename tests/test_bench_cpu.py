"""The multi-process side of bench.py on CPU: two gloo ranks reduce their step times to the
slowest one, and the reference arm runs on rank 0 alone under a two-rank launch."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _launch(cmd, world):
    port = _free_port()
    procs = []
    for rank in range(world):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                   LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
        procs.append(subprocess.Popen(cmd, env=env, cwd=ROOT, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=240)
        except subprocess.TimeoutExpired:
            p.kill()
            raise
        outs.append((p.returncode, out, err))
    return outs


_RANK_SCRIPT = """
import json, sys
import torch.distributed as dist
sys.path.insert(0, %r)
import bench
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
ms = (12.5, 20.0)[rank]
m = bench.max_over_ranks(ms, world, "cpu")
print(json.dumps({"rank": rank, "max": m, "value": bench.job_throughput(1000000, 10, world, m)}))
dist.destroy_process_group()
"""


def test_two_ranks_reduce_to_slowest_time():
    pytest.importorskip("torch")
    outs = _launch([sys.executable, "-c", _RANK_SCRIPT % ROOT], 2)
    for rc, out, err in outs:
        assert rc == 0, err[-2000:]
    got = [json.loads(out.strip().splitlines()[-1]) for _, out, _ in outs]
    for g in got:
        assert g["max"] == 20.0
        # 2 replicas x 1e6 cells x 10 steps in 20 ms
        assert g["value"] == pytest.approx(2 * 1e6 * 10 / 20e-3 / 1e9)


def test_reference_arm_runs_on_rank_zero_only():
    outs = _launch([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--N", "16",
                    "--steps", "3", "--warmup", "1"], 2)
    for rc, out, err in outs:
        assert rc == 0, err[-2000:]
    lines = [o.strip().splitlines() for _, o, _ in outs]
    assert lines[1] == []
    line = json.loads(lines[0][-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 3
    # the default block workload, the one the GPU arm measures
    assert line["config"]["workload"] == "mixed_faces_16^3"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_clock_summary_brackets_a_short_region():
    """A timed region shorter than the sampling period is reported through the nearest sample
    before and after it; samples far outside it are left out."""
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    row = lambda mhz, cap: ["0", str(mhz), "2070", "900", "0x0", "Not Active", "Not Active", "Not Active", cap]
    c.rows = [(0.0, row(1000, "Active")), (1.0, row(2000, "Not Active")), (1.05, row(2070, "Not Active")),
              (2.0, row(900, "Active"))]
    s = c.summary(1.01, 1.02)
    assert s["samples"] == 2 and s["sm_mhz"] == 2035 and s["reasons"] == []
    assert bench.ClockSampler(0).summary(0, 1)["reasons"] == ["unsampled"]
