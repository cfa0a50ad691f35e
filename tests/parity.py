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
        blk.probe_specs = list(b.probes)
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
    """Per block: relative L2 error of the E field and of the H field (all three components
    together), the reading of "relative L2 error per field" used throughout."""
    errs = []
    for s, b in zip(sims, blocks):
        row = []
        for comps in ((0, 1, 2), (3, 4, 5)):
            num = sum(np.sum((s.field(c).astype(np.float64) - b.field(c)) ** 2) for c in comps)
            den = sum(np.sum(b.field(c) ** 2) for c in comps)
            row.append(float(np.sqrt(num / den)) if den > 0 else float(np.sqrt(num)))
        errs.append(row)
    return errs


def component_errors(sims, blocks):
    """Per block, per component: ||gpu - ref|| / ||ref field|| (E or H norm)."""
    out = []
    for s, b in zip(sims, blocks):
        ref = [b.field(c) for c in range(6)]
        nE = np.sqrt(sum(np.sum(r ** 2) for r in ref[:3]))
        nH = np.sqrt(sum(np.sum(r ** 2) for r in ref[3:]))
        out.append([float(np.linalg.norm(s.field(c).astype(np.float64) - ref[c]) / (nE if c < 3 else nH))
                    for c in range(6)])
    return out


def probe_error(sims, blocks):
    """Max probe error, each probe scaled by the peak of all probes of its field (E or H)
    over every block (a probe the wave has not reached yet is measured against the
    field's peak elsewhere, not against its own near-zero values)."""
    pairs = []
    for s, b in zip(sims, blocks):
        if b.nprobes == 0:
            continue
        g, r = s.probes(), b.probes()[:, : s.probes().shape[1]]
        comps = np.array([p.comp for p in b.probe_specs]) if hasattr(b, "probe_specs") else None
        pairs.append((g, r, comps))
    if not pairs:
        return 0.0
    fpeak = {}
    for isH in (False, True):
        vals = [np.abs(r[(c >= 3) == isH]).max() for g, r, c in pairs if c is not None and ((c >= 3) == isH).any()]
        fpeak[isH] = max(vals) if vals else 0.0
    worst = 0.0
    for g, r, comps in pairs:
        peak = np.max(np.abs(r), axis=1)
        if comps is not None:
            for isH in (False, True):
                sel = (comps >= 3) == isH
                if sel.any():
                    peak[sel] = max(fpeak[isH], 1e-300)
        peak[peak == 0] = 1.0
        worst = max(worst, float(np.max(np.abs(g - r) / peak[:, None])))
    return worst
