"""FP64 CPU oracle of the 3D SBP-SAT FDTD method (arXiv 2206.00638).

TEST INFRASTRUCTURE ONLY.  The arithmetic lives in ``sbpsat_oracle.c`` (plain
C loops, OpenMP over z-planes, no blocking or fusion); this module compiles
it with gcc on first use and wraps it with ctypes.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg
may import it.  It shares no code with the CUDA library.

Every function of the C file cites the passage it follows.  Pins (tests under
``tests/test_oracle_*.py``) tie it to the paper's exact SBP identities, to the
Kronecker construction of Eqs. (ED_1)-(ED_3) built from the printed Q
matrices, to energy conservation, to the analytic cavity resonance and to a
1D reduction.  The absorbing penalty (not the paper's) is pinned to the
closed-form oblique reflection of the first-order characteristic condition;
the interface penalty to the printed periodic-SAT matrices (1D complex pair)
and to the Fresnel coefficients of a dielectric step.  The current sources are
pinned to the field a current sheet radiates (-eta K / 2) and to the full
Hertzian-dipole field of a point current element.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbpsat_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

PEC, PMC, ABSORBING, INTERFACE = 0, 1, 2, 3
EX, EY, EZ, HX, HY, HZ = range(6)
GAUSS, GAUSS_DERIV, MOD_GAUSS = 0, 1, 2
C0 = 299792458.0
EPS0 = 8.8541878128e-12
MU0 = 1.25663706212e-6

# Table I: 1 if the component lives on the plus grid along x, y, z.
ON_PLUS = ((0, 1, 1), (1, 0, 1), (1, 1, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1))


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_liboracle.so`` (gcc, -O3, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P, D, I, V = C.c_void_p, C.c_double, C.c_int, None
            dp = C.POINTER(C.c_double)
            sig = {
                "ob_dplus": (V, [I, dp]), "ob_dminus": (V, [I, dp]),
                "ob_pplus": (V, [I, dp]), "ob_pminus": (V, [I, dp]),
                "ob_create": (P, [I, I, I, D, D, D, D, C.POINTER(C.c_int), dp, dp]),
                "ob_destroy": (V, [P]), "ob_count": (C.c_long, [P, I]),
                "ob_set_field": (V, [P, I, dp]), "ob_get_field": (V, [P, I, dp]),
                "ob_get_rhs": (V, [P, I, dp]), "ob_get_node_eps": (V, [P, I, dp]),
                "ob_get_step": (C.c_long, [P]), "ob_set_step": (V, [P, C.c_long]),
                "ob_connect": (I, [P, I, P, I]),
                "ob_connect_phase": (I, [P, P, I, D]),
                "ob_add_source": (I, [P, I, I, I, I, I, D, D, D, D]),
                "ob_add_probe": (I, [P, I, I, I, I]),
                "ob_probe_reserve": (V, [P, C.c_long]), "ob_get_probes": (V, [P, dp]),
                "ob_waveform": (D, [I, D, D, D, D]), "ob_dt": (D, [D, D, D, D, D]),
                "ob_rhs": (V, [C.POINTER(P), I]), "ob_step": (V, [C.POINTER(P), I, C.c_long]),
                "ob_energy": (D, [C.POINTER(P), I]),
                "ob_set_threads": (V, [I]), "ob_get_threads": (I, []),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def extents(n, comp):
    """Natural extents (x, y, z) of a component on an (nx, ny, nz)-cell block: Table I."""
    return tuple(n[a] + (1 if ON_PLUS[comp][a] else 2) for a in range(3))


def dplus(n: int) -> np.ndarray:
    """D+ of the Appendix at unit spacing, shape (n+1, n+2)."""
    out = np.zeros((n + 1, n + 2))
    lib().ob_dplus(n, _dp(out))
    return out


def dminus(n: int) -> np.ndarray:
    """D- of the Appendix at unit spacing, shape (n+2, n+1)."""
    out = np.zeros((n + 2, n + 1))
    lib().ob_dminus(n, _dp(out))
    return out


def pplus(n: int) -> np.ndarray:
    out = np.zeros(n + 1)
    lib().ob_pplus(n, _dp(out))
    return out


def pminus(n: int) -> np.ndarray:
    out = np.zeros(n + 2)
    lib().ob_pminus(n, _dp(out))
    return out


def waveform(kind: int, t: float, tw: float, t0: float, f: float = 0.0) -> float:
    return lib().ob_waveform(kind, t, tw, t0, f)


def dt_cfl(cfl: float, dx: float, dy: float, dz: float, c: float = C0) -> float:
    return lib().ob_dt(cfl, dx, dy, dz, c)


def set_threads(n: int) -> None:
    lib().ob_set_threads(int(n))


def get_threads() -> int:
    return lib().ob_get_threads()


class Block:
    """One rectangular block of nx*ny*nz cells (oracle side).

    ``faces`` lists the boundary type of x-, x+, y-, y+, z-, z+.  ``eps_r`` and
    ``mu_r`` are per-cell arrays of shape (nz, ny, nx) or None (vacuum).
    Fields use natural extents, arrays of shape (ext_z, ext_y, ext_x).
    """

    def __init__(self, n, h, dt, faces, eps_r=None, mu_r=None):
        self.n = tuple(int(v) for v in n)
        self.h = tuple(float(v) for v in h)
        self.dt = float(dt)
        L = lib()
        fa = (C.c_int * 6)(*[int(f) for f in faces])
        self._eps = None if eps_r is None else np.ascontiguousarray(eps_r, dtype=np.float64).reshape(-1)
        self._mu = None if mu_r is None else np.ascontiguousarray(mu_r, dtype=np.float64).reshape(-1)
        ncell = self.n[0] * self.n[1] * self.n[2]
        for arr in (self._eps, self._mu):
            if arr is not None and arr.size != ncell:
                raise ValueError("material array must have nx*ny*nz entries")
        self._h = L.ob_create(*self.n, *self.h, self.dt, fa,
                              None if self._eps is None else _dp(self._eps),
                              None if self._mu is None else _dp(self._mu))
        if not self._h:
            raise ValueError("oracle block needs at least 4 cells per axis")
        self.nprobes = 0
        self.probe_cap = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().ob_destroy(h)
            self._h = None

    def shape(self, comp):
        e = extents(self.n, comp)
        return (e[2], e[1], e[0])

    def set_field(self, comp, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64)
        if a.shape != self.shape(comp):
            raise ValueError(f"component {comp}: expected {self.shape(comp)}, got {a.shape}")
        lib().ob_set_field(self._h, comp, _dp(a))

    def field(self, comp):
        out = np.zeros(self.shape(comp))
        lib().ob_get_field(self._h, comp, _dp(out))
        return out

    def rhs(self, comp):
        out = np.zeros(self.shape(comp))
        lib().ob_get_rhs(self._h, comp, _dp(out))
        return out

    def node_eps(self, comp):
        out = np.zeros(self.shape(comp))
        lib().ob_get_node_eps(self._h, comp, _dp(out))
        return out

    @property
    def step_index(self):
        return lib().ob_get_step(self._h)

    def add_source(self, comp, i, j, k, kind, amp, tw, t0, f=0.0):
        return lib().ob_add_source(self._h, comp, i, j, k, kind, amp, tw, t0, f)

    def add_probe(self, comp, i, j, k):
        self.nprobes += 1
        return lib().ob_add_probe(self._h, comp, i, j, k)

    def reserve_probes(self, nsteps):
        self.probe_cap = int(nsteps)
        lib().ob_probe_reserve(self._h, self.probe_cap)

    def probes(self):
        out = np.zeros((max(self.nprobes, 1), self.probe_cap))
        lib().ob_get_probes(self._h, _dp(out))
        return out[: self.nprobes]


def _handles(blocks):
    arr = (C.c_void_p * len(blocks))(*[b._h for b in blocks])
    return arr, len(blocks)


def connect(a: Block, face_a: int, b: Block, face_b: int) -> None:
    """Conforming interface SAT between face_a of a and face_b of b."""
    rc = lib().ob_connect(a._h, face_a, b._h, face_b)
    if rc != 0:
        raise ValueError(f"faces do not conform (code {rc})")


def connect_phase(re: Block, im: Block, axis: int, alpha: float) -> None:
    """Periodic faces along ``axis`` with phase shift ``alpha`` (radians per period,
    Eqs. (EPBC1-6)) for the complex field re + j im; both blocks are stepped together."""
    rc = lib().ob_connect_phase(re._h, im._h, int(axis), float(alpha))
    if rc != 0:
        raise ValueError(f"blocks do not form a complex pair (code {rc})")


def step(blocks, nsteps: int) -> None:
    arr, nb = _handles(blocks)
    lib().ob_step(arr, nb, int(nsteps))


def rhs(blocks) -> None:
    arr, nb = _handles(blocks)
    lib().ob_rhs(arr, nb)


def energy(blocks) -> float:
    arr, nb = _handles(blocks)
    return lib().ob_energy(arr, nb)
