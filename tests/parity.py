"""Run a workload on the CUDA path and on the FP64 oracle and compare them."""
import numpy as np

import oracle
from paper_2206_00638_gb300 import sbpsat


def oracle_blocks(w, dt):
    blocks = []
    for b in w.blocks:
        blk = oracle.Block(b.n, b.h, dt, b.faces, eps_r=b.eps_r, mu_r=b.mu_r)
        if b.fields is not None:
            for c in range(6):
                blk.set_field(c, b.fields[c])
        for s in b.sources:
            blk.add_source(s.comp, s.i, s.j, s.k, s.kind, s.amp, s.tw, s.t0, s.f)
        for p in b.probes:
            blk.add_probe(p.comp, p.i, p.j, p.k)
        blocks.append(blk)
    for a, fa, b, fb in w.links:
        oracle.connect(blocks[a], fa, blocks[b], fb)
    return blocks


def gpu_run(w, steps, precision=sbpsat.FP32, **kw):
    sims = sbpsat.from_workload(w, precision=precision, **kw)
    for s in sims:
        s.reserve_probes(steps)
    if len(sims) == 1:
        sims[0].step(steps)
    else:
        sbpsat.step_group(sims, steps)
    return sims


def oracle_run(w, steps, dt):
    blocks = oracle_blocks(w, dt)
    for b in blocks:
        b.reserve_probes(steps)
    oracle.step(blocks, steps)
    return blocks


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


def compare(sims, blocks):
    """Per-block, per-component relative L2 error, and max relative probe error."""
    errs = []
    for s, b in zip(sims, blocks):
        errs.append([rel_l2(s.field(c).astype(np.float64), b.field(c)) for c in range(6)])
    return errs


def probe_error(sims, blocks):
    worst = 0.0
    for s, b in zip(sims, blocks):
        if b.nprobes == 0:
            continue
        g, r = s.probes(), b.probes()
        scale = np.max(np.abs(r), axis=1, keepdims=True)
        scale[scale == 0] = 1.0
        worst = max(worst, float(np.max(np.abs(g - r[:, : g.shape[1]]) / scale)))
    return worst
