"""Seeded synthetic inputs for the SBP-SAT FDTD workloads.

This module holds no arithmetic of the method: it only draws seeded material
maps, initial fields, source and probe placements, and names the boundary
types.  Both the CUDA path and the FP64 oracle are fed from it, so the two
sides see bit-identical inputs.  Importing it loads no native code.

Workloads (cells, spacing, faces, materials, sources, steps):
  cavity        20x16x12 PEC box 1.0x0.8x0.6 m, TE101-type mode (E along z)
                plus seeded U(-1e-3, 1e-3) noise on every node, dt = 0.9 CFL,
                500 steps.
  dielectric    N^3 PEC box, h = 1 mm, centred (N/4)^3 cube with eps_r = 4,
                z-directed Gaussian-derivative dipole (10 GHz), dt = 0.95 CFL,
                8 seeded probes.  N = 256 is the full-size case.
  two_block     two conforming blocks joined on z by an interface, absorbing
                outer faces, eps_r ~ U[1, 4] per 8^3 patch, Gaussian sheet.
  mixed_faces   PMC x faces, PEC y faces, absorbing z faces, dielectric
                spheres, Gaussian sheet on Ey.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

PEC, PMC, ABSORBING, INTERFACE = 0, 1, 2, 3
EX, EY, EZ, HX, HY, HZ = range(6)
GAUSS, GAUSS_DERIV, MOD_GAUSS = 0, 1, 2
C0 = 299792458.0

# Table I of the paper: 1 if the component lives on the plus grid along x, y, z.
ON_PLUS = ((0, 1, 1), (1, 0, 1), (1, 1, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1))


def extents(n: Sequence[int], comp: int) -> Tuple[int, int, int]:
    """(x, y, z) node counts of a component on an n = (nx, ny, nz) block."""
    return tuple(int(n[a]) + (1 if ON_PLUS[comp][a] else 2) for a in range(3))


def field_shape(n: Sequence[int], comp: int) -> Tuple[int, int, int]:
    e = extents(n, comp)
    return (e[2], e[1], e[0])


@dataclass
class Source:
    comp: int
    i: int
    j: int
    k: int           # -1 on an index = every node along that axis (sheet)
    kind: int
    amp: float
    tw: float
    t0: float
    f: float = 0.0


@dataclass
class Probe:
    comp: int
    i: int
    j: int
    k: int


@dataclass
class BlockSpec:
    n: Tuple[int, int, int]
    h: Tuple[float, float, float]
    faces: Tuple[int, int, int, int, int, int]
    eps_r: Optional[np.ndarray] = None          # (nz, ny, nx) float32 or None
    mu_r: Optional[np.ndarray] = None
    fields: Optional[List[np.ndarray]] = None   # six arrays in natural extents (float64) or None
    sources: List[Source] = field(default_factory=list)
    probes: List[Probe] = field(default_factory=list)


@dataclass
class Workload:
    name: str
    blocks: List[BlockSpec]
    links: List[Tuple[int, int, int, int]]      # (block a, face a, block b, face b)
    cfl: float
    steps: int

    def cells(self) -> int:
        return sum(b.n[0] * b.n[1] * b.n[2] for b in self.blocks)


def gaussian_deriv_tw(f_center: float) -> float:
    """Pulse width t_w whose Gaussian-derivative spectrum peaks at f_center."""
    return math.sqrt(2.0) / (math.sqrt(math.pi) * f_center)


def random_fields(n, seed: int, amp: float = 1.0) -> List[np.ndarray]:
    rng = np.random.default_rng(seed)
    return [rng.uniform(-amp, amp, size=field_shape(n, c)) for c in range(6)]


def cavity(seed: int = 1, noise: float = 1e-3, steps: int = 500) -> Workload:
    """PEC cavity 1.0 x 0.8 x 0.6 m on 20x16x12 cells of 5 cm: Ez = sin(pi x/a) sin(pi y/b)
    on the Ez nodes (x+, y+, z-), H^{-1/2} = 0, plus uniform noise on every node."""
    n = (20, 16, 12)
    h = 0.05
    a, b = n[0] * h, n[1] * h
    rng = np.random.default_rng(seed)
    fields = [rng.uniform(-noise, noise, size=field_shape(n, c)) for c in range(6)]
    ez = field_shape(n, EZ)
    x = np.arange(ez[2]) * h
    y = np.arange(ez[1]) * h
    mode = np.sin(np.pi * x / a)[None, :] * np.sin(np.pi * y / b)[:, None]
    fields[EZ] = fields[EZ] + mode[None, :, :]
    blk = BlockSpec(n=n, h=(h, h, h), faces=(PEC,) * 6, fields=fields,
                    probes=[Probe(EZ, 10, 8, 6)])
    return Workload("pec_cavity_20x16x12", [blk], [], 0.9, steps)


def cavity_resonance_hz() -> float:
    """Analytic frequency of the cavity mode with E along z: (c/2) sqrt(1/a^2 + 1/b^2)."""
    return 0.5 * C0 * math.sqrt(1.0 / 1.0 ** 2 + 1.0 / 0.8 ** 2)


def dielectric(N: int = 256, seed: int = 2, steps: int = 2000, nprobes: int = 8) -> Workload:
    """N^3 PEC box, h = 1 mm, eps_r = 4 on the centred cube of N/4 cells per side,
    z-directed Gaussian-derivative dipole centred at 10 GHz on the Ez node
    (N/4, N/2, N/2), dt = 0.95 CFL, probes at seeded interior nodes."""
    n = (N, N, N)
    eps = np.ones((N, N, N), dtype=np.float32)
    lo, hi = 3 * N // 8, 5 * N // 8
    eps[lo:hi, lo:hi, lo:hi] = 4.0
    tw = gaussian_deriv_tw(10e9)
    src = Source(EZ, N // 4, N // 2, N // 2, GAUSS_DERIV, 1.0, tw, tw)
    rng = np.random.default_rng(seed)
    probes = []
    for p in range(nprobes):
        comp = p % 3
        e = extents(n, comp)
        probes.append(Probe(comp, *[int(rng.integers(3, e[a] - 3)) for a in range(3)]))
    blk = BlockSpec(n=n, h=(1e-3,) * 3, faces=(PEC,) * 6, eps_r=eps, sources=[src], probes=probes)
    return Workload(f"dielectric_cube_{N}^3", [blk], [], 0.95, steps)


def two_block(nxy: int = 192, nz: int = 96, patch: int = 8, seed: int = 3, steps: int = 3000) -> Workload:
    """Two nxy x nxy x nz blocks joined z+ of A to z- of B, absorbing outer faces,
    eps_r ~ U[1, 4] per patch^3 cells over the combined box, Ex Gaussian sheet on
    the z-plane k = nz/6 of block A."""
    rng = np.random.default_rng(seed)
    pz = 2 * nz // patch
    pxy = nxy // patch
    patches = rng.uniform(1.0, 4.0, size=(pz, pxy, pxy)).astype(np.float32)
    full = np.repeat(np.repeat(np.repeat(patches, patch, 0), patch, 1), patch, 2)
    tw = 80e-12
    A = BlockSpec(n=(nxy, nxy, nz), h=(1e-3,) * 3,
                  faces=(ABSORBING, ABSORBING, ABSORBING, ABSORBING, ABSORBING, INTERFACE),
                  eps_r=np.ascontiguousarray(full[:nz]),
                  sources=[Source(EX, -1, -1, nz // 6, GAUSS, 1.0, tw, tw)],
                  probes=[Probe(EX, nxy // 2, nxy // 2, nz // 2)])
    B = BlockSpec(n=(nxy, nxy, nz), h=(1e-3,) * 3,
                  faces=(ABSORBING, ABSORBING, ABSORBING, ABSORBING, INTERFACE, ABSORBING),
                  eps_r=np.ascontiguousarray(full[nz:]),
                  probes=[Probe(EX, nxy // 2, nxy // 2, nz // 2)])
    return Workload(f"two_block_{nxy}x{nxy}x{nz}x2", [A, B], [(0, 5, 1, 4)], 0.95, steps)


def mixed_faces(N: int = 512, seed: int = 5, steps: int = 1000, h: float = 1e-3) -> Workload:
    """N^3 block, PMC on x faces, PEC on y faces, absorbing z faces, four seeded
    dielectric spheres eps_r ~ U[2, 8] with radii ~ U[N/16, 3N/16], Ey Gaussian
    sheet on the z-plane k = N/16."""
    rng = np.random.default_rng(seed)
    eps = np.ones((N, N, N), dtype=np.float32)
    zc = (np.arange(N) + 0.5)
    for _ in range(4):
        r = rng.uniform(N / 16, 3 * N / 16)
        c = [rng.uniform(r, N - r) for _ in range(3)]
        er = np.float32(rng.uniform(2.0, 8.0))
        d2 = ((zc[:, None, None] - c[2]) ** 2 + (zc[None, :, None] - c[1]) ** 2
              + (zc[None, None, :] - c[0]) ** 2)
        eps[d2 <= r * r] = er
    tw = 80e-12
    blk = BlockSpec(n=(N, N, N), h=(h,) * 3, faces=(PMC, PMC, PEC, PEC, ABSORBING, ABSORBING),
                    eps_r=eps, sources=[Source(EY, -1, -1, N // 16, GAUSS, 1.0, tw, tw)],
                    probes=[Probe(EY, N // 2, N // 2, N // 2)])
    return Workload(f"mixed_faces_{N}^3", [blk], [], 0.95, steps)


def random_box(n, h=(1e-3, 1e-3, 1e-3), faces=(PEC,) * 6, seed: int = 0, eps_range=(1.0, 4.0),
               mu_range=None, cfl: float = 0.95, steps: int = 100, nprobes: int = 12,
               sources: bool = True) -> Workload:
    """Parity workload: seeded per-cell eps_r ~ U[eps_range] (and mu_r if given), random
    initial fields on every node (E ~ U(-1, 1) V/m, H ~ U(-1, 1)/377 A/m), a
    Gaussian-derivative point source on Ez, a Gaussian sheet on Ex, and probes of
    all six components at seeded nodes (boundary nodes included)."""
    n = tuple(int(v) for v in n)
    rng = np.random.default_rng(seed)
    eps = rng.uniform(*eps_range, size=(n[2], n[1], n[0])).astype(np.float32)
    mu = None if mu_range is None else rng.uniform(*mu_range, size=(n[2], n[1], n[0])).astype(np.float32)
    fields = [rng.uniform(-1.0, 1.0, size=field_shape(n, c)) * (1.0 if c < 3 else 1.0 / 377.0)
              for c in range(6)]
    srcs = []
    if sources:
        tw = gaussian_deriv_tw(20e9)
        ez = extents(n, EZ)
        srcs.append(Source(EZ, int(rng.integers(0, ez[0])), int(rng.integers(0, ez[1])),
                           int(rng.integers(0, ez[2])), GAUSS_DERIV, 2.0, tw, tw))
        srcs.append(Source(EX, -1, -1, int(rng.integers(0, extents(n, EX)[2])), GAUSS, 1.0, 2 * tw, 2 * tw))
    probes = []
    for p in range(nprobes):
        comp = p % 6
        e = extents(n, comp)
        probes.append(Probe(comp, *[int(rng.integers(0, e[a])) for a in range(3)]))
    blk = BlockSpec(n=n, h=tuple(h), faces=tuple(faces), eps_r=eps, mu_r=mu, fields=fields,
                    sources=srcs, probes=probes)
    return Workload(f"random_box_{n[0]}x{n[1]}x{n[2]}", [blk], [], cfl, steps)


def coupled_boxes(nA, nB, axis: int, h=(1e-3, 1e-3, 1e-3), facesA=(PEC,) * 6, facesB=(PEC,) * 6,
                  seed: int = 0, cfl: float = 0.95, steps: int = 100) -> Workload:
    """Two random boxes joined high face of A to low face of B along axis (conforming)."""
    wa = random_box(nA, h, facesA, seed=seed, cfl=cfl, steps=steps)
    wb = random_box(nB, h, facesB, seed=seed + 1, cfl=cfl, steps=steps, sources=False)
    return Workload(f"coupled_{axis}", wa.blocks + wb.blocks, [(0, 2 * axis + 1, 1, 2 * axis)], cfl, steps)


def serving_requests(nreq: int = 512, seed: int = 4, n_range=(32, 192), steps_range=(500, 4000),
                     eps_range=(1.0, 6.0), sub: int = 16):
    """Compact descriptors of the serving workload's requests (materialise with serving_spec):
    per-axis cells ~ U{n_range}, steps ~ U{steps_range}, each face PEC or absorbing with
    probability 1/2, eps_r ~ U[eps_range] per sub^3-cell sub-box, a 10 GHz Gaussian-derivative
    Ez dipole at a uniformly random interior node and one Ez probe two nodes above it."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nreq):
        n = tuple(int(rng.integers(n_range[0], n_range[1] + 1)) for _ in range(3))
        faces = tuple(int(PEC if rng.random() < 0.5 else ABSORBING) for _ in range(6))
        nb = [(n[a] + sub - 1) // sub for a in range(3)]
        boxes = rng.uniform(*eps_range, size=(nb[2], nb[1], nb[0])).astype(np.float32)
        e = extents(n, EZ)
        pos = tuple(int(rng.integers(3, e[a] - 3)) for a in range(3))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        out.append({"n": n, "faces": faces, "boxes": boxes, "sub": sub, "pos": pos, "steps": steps})
    return out


def serving_spec(r, h: float = 1e-3) -> BlockSpec:
    n, sub, pos = r["n"], r["sub"], r["pos"]
    eps = np.repeat(np.repeat(np.repeat(r["boxes"], sub, 0), sub, 1), sub, 2)[: n[2], : n[1], : n[0]]
    tw = gaussian_deriv_tw(10e9)
    e = extents(n, EZ)
    return BlockSpec(n=n, h=(h,) * 3, faces=r["faces"], eps_r=np.ascontiguousarray(eps),
                     sources=[Source(EZ, *pos, GAUSS_DERIV, 1.0, tw, tw)],
                     probes=[Probe(EZ, pos[0], pos[1], min(pos[2] + 2, e[2] - 1))])


def serving_stream(nreq: int = 512, seed: int = 4, n_range=(32, 192), steps_range=(500, 4000),
                   eps_range=(1.0, 6.0), sub: int = 16, h: float = 1e-3):
    """The serving workload materialised: a list of (BlockSpec, nsteps)."""
    return [(serving_spec(r, h), r["steps"])
            for r in serving_requests(nreq, seed, n_range, steps_range, eps_range, sub)]
