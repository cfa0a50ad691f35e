"""Serving loop (continuous batching): results identical alone and in the mix; admission by HBM."""
import time

import numpy as np
import pytest

from paper_2206_00638_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_00638_gb300 import sbpsat  # noqa: E402


def _alone(spec, steps, stream):
    s = sbpsat.Sim(spec.n, spec.h, spec.faces, eps_r=spec.eps_r, cfl=0.95, stream=stream)
    for src in spec.sources:
        s.add_source(src.comp, src.i, src.j, src.k, src.kind, src.amp, src.tw, src.t0, src.f)
    for p in spec.probes:
        s.add_probe(p.comp, p.i, p.j, p.k)
    s.reserve_probes(steps)
    s.step(steps)
    out = s.probes()
    s.close()
    return out


def test_server_results_equal_alone():
    reqs = wl.serving_stream(nreq=7, seed=11, n_range=(12, 48), steps_range=(40, 160))
    stream = torch.cuda.current_stream()
    ref = [_alone(spec, steps, stream) for spec, steps in reqs]
    srv = sbpsat.Server(stream=torch.cuda.Stream(), max_slots=4, chunk=16)
    tickets = []
    for q, (spec, steps) in enumerate(reqs):
        tickets.append(srv.submit(spec, steps))
        if q == 3:
            time.sleep(0.05)          # later requests arrive while earlier ones run
    srv.drain()
    for t, r, (spec, steps) in zip(tickets, ref, reqs):
        res = srv.poll(t)
        assert res is not None and res.status == 0 and res.steps == steps
        assert res.submit_s <= res.admit_s <= res.done_s
        assert np.array_equal(srv.probes(t), r), spec.n
        srv.release(t)
    cu, span = srv.stats()
    assert cu == sum(int(np.prod(s.n)) * st for s, st in reqs) and span > 0
    srv.close()


def test_server_admission_waits_for_memory():
    reqs = wl.serving_stream(nreq=5, seed=3, n_range=(40, 40), steps_range=(60, 60))
    one = sbpsat.lib().sbp_workspace_bytes  # noqa: F841 (symbol present)
    spec0 = reqs[0][0]
    # budget for about two requests at a time
    d = sbpsat.GridDesc()
    d.nx, d.ny, d.nz = spec0.n
    d.dx = d.dy = d.dz = 1e-3
    d.cfl_fraction = 0.95
    for f in range(6):
        d.face[f] = 0
    per = sbpsat.lib().sbp_workspace_bytes(sbpsat.C.byref(d)) + 8 * 60 * 4
    srv = sbpsat.Server(stream=torch.cuda.Stream(), budget_bytes=int(2.5 * per), max_slots=8, chunk=8)
    tickets = [srv.submit(spec, steps) for spec, steps in reqs]
    srv.drain()
    res = [srv.poll(t) for t in tickets]
    assert all(r.status == 0 for r in res)
    # the later requests were admitted only after earlier ones finished
    assert res[4].admit_s >= min(r.done_s for r in res[:2]) - 1e-3
    srv.close()


def test_server_rejects_ineligible_requests():
    srv = sbpsat.Server(stream=torch.cuda.Stream(), max_slots=2, chunk=8)
    spec, steps = wl.serving_stream(nreq=1, seed=1, n_range=(16, 16), steps_range=(10, 10))[0]
    small = wl.BlockSpec(n=(6, 16, 16), h=spec.h, faces=spec.faces)
    with pytest.raises(sbpsat.SbpError):
        srv.submit(small, 10)
    srv.close()


def test_server_unstable_request_fails_alone():
    """A request stepped beyond the stability limit (CFL 1.2, allowed by its flags) blows up:
    its FP64 energy monitor reports SBP_EUNSTABLE and it leaves the batch early, while the
    requests sharing the batch with it finish with probe samples bit-identical to running
    alone."""
    reqs = wl.serving_stream(nreq=4, seed=21, n_range=(16, 40), steps_range=(600, 600))
    stream = torch.cuda.current_stream()
    ref = [_alone(spec, steps, stream) for spec, steps in reqs]
    srv = sbpsat.Server(stream=torch.cuda.Stream(), max_slots=8, chunk=16)
    bad_spec, _ = wl.serving_stream(nreq=1, seed=5, n_range=(24, 24), steps_range=(600, 600))[0]
    tickets = [srv.submit(spec, steps, energy_every=16) for spec, steps in reqs[:2]]
    bad = srv.submit(bad_spec, 4000, cfl=1.2, energy_every=16, flags=sbpsat.FLAG_ALLOW_UNSTABLE)
    tickets += [srv.submit(spec, steps, energy_every=16) for spec, steps in reqs[2:]]
    srv.drain()
    res_bad = srv.poll(bad)
    assert res_bad.status == -4                     # SBP_EUNSTABLE
    assert 0 < res_bad.steps < 4000                 # stopped early
    for t, r, (spec, steps) in zip(tickets, ref, reqs):
        res = srv.poll(t)
        assert res.status == 0 and res.steps == steps
        assert np.array_equal(srv.probes(t), r), spec.n
    srv.close()
