"""Python binding of the C ABI in ``include/sbpsat.h`` (argument marshalling only).

Every step of the leapfrog runs in the CUDA kernels of ``csrc/``; this module
builds ``libsbpsat.so`` in-tree with nvcc, loads it with ctypes and converts
numpy arrays / torch tensors to plain pointers.  There is no CPU fallback: if
the library cannot be built or loaded, every call raises.

PyTorch supplies device memory (the simulation workspace can be a torch
uint8 tensor, so the caching allocator owns it) and the CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
_CSRC = os.path.join(_PKG, "csrc")
_INC = os.path.join(_ROOT, "include")
_LIBDIR = os.path.join(_PKG, "_lib")
LIB_PATH = os.path.join(_LIBDIR, "libsbpsat.so")
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared"]

PEC, PMC, ABSORBING, INTERFACE = 0, 1, 2, 3
FP32, FP64, FP32_FP16STORE = 0, 1, 2
EX, EY, EZ, HX, HY, HZ = range(6)
GAUSS, GAUSS_DERIV, MOD_GAUSS = 0, 1, 2
FLAG_ALLOW_UNSTABLE = 1
FLAG_FDTD = 2          # plain Yee FDTD comparator (six PEC faces, one-pass path)
FLAG_TEST_WAIT_TIMEOUT = 4   # test hook: the one-pass pipeline waits run out (SBP_ETIMEOUT)

ON_PLUS = ((0, 1, 1), (1, 0, 1), (1, 1, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1))

_lock = threading.Lock()
_lib = None


class SbpError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = _strerror(code)
        super().__init__(f"{what}: {msg} ({code})")


def _sources():
    return [os.path.join(_CSRC, f) for f in sorted(os.listdir(_CSRC)) if f.endswith((".cu", ".cuh"))] + \
        [os.path.join(_INC, "sbpsat.h")]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/*.cu for sm_103a into _lib/libsbpsat.so (in-tree)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _sources())
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    tmp = LIB_PATH + f".{os.getpid()}.tmp"
    extra = os.environ.get("SBP_NVCC_FLAGS", "").split()   # tuning experiments only
    cmd = ["nvcc", *NVCC_FLAGS, *extra, "-I" + _INC, "-I" + _CSRC, "-o", tmp, os.path.join(_CSRC, "sbpsat.cu")]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class GridDesc(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
        ("eps_r", C.POINTER(C.c_float)), ("mu_r", C.POINTER(C.c_float)),
        ("face", C.c_int32 * 6),
        ("cfl_fraction", C.c_double),
        ("precision", C.c_int32),
        ("energy_every", C.c_int32),
        ("flags", C.c_int32),
        ("field_scale", C.c_double * 2),
    ]


def lib():
    """Load libsbpsat.so (building it first if needed).  Raises if it cannot."""
    global _lib
    with _lock:
        if _lib is None:
            path = LIB_PATH if os.path.exists(LIB_PATH) else build()
            L = C.CDLL(path)
            P, I, D, I64, SZ = C.c_void_p, C.c_int, C.c_double, C.c_int64, C.c_size_t
            pp = C.POINTER(C.c_void_p)
            sig = {
                "sbp_create": (I, [C.POINTER(GridDesc), P, pp]),
                "sbp_workspace_bytes": (SZ, [C.POINTER(GridDesc)]),
                "sbp_create_in": (I, [C.POINTER(GridDesc), P, P, SZ, pp]),
                "sbp_connect": (I, [P, I, P, I]),
                "sbp_set_field": (I, [P, I, P, I]),
                "sbp_get_field": (I, [P, I, P, I]),
                "sbp_add_source": (I, [P, I, I, I, I, I, D, D, D, D]),
                "sbp_add_probe": (I, [P, I, I, I, I, C.POINTER(C.c_int)]),
                "sbp_reserve_probes": (I, [P, I64]),
                "sbp_step": (I, [P, I64]),
                "sbp_step_group": (I, [pp, I, I64]),
                "sbp_half_step_h": (I, [pp, I]),
                "sbp_half_step_e": (I, [pp, I]),
                "sbp_autotune": (I, [P, I, C.POINTER(C.c_int), C.POINTER(D)]),
                "sbp_tile": (I, [P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
                "sbp_connect_phase": (I, [P, P, I, D]),
                "sbp_checkpoint_bytes": (SZ, [P]),
                "sbp_save": (I, [P, P, SZ]),
                "sbp_load": (I, [P, P, SZ]),
                "sbp_step_timed": (I, [P, I64, C.POINTER(C.c_double), C.POINTER(C.c_int64), I]),
                "sbp_get_probes": (I, [P, C.POINTER(C.c_double), I64, C.POINTER(C.c_int64)]),
                "sbp_energy": (I, [P, C.POINTER(C.c_double)]),
                "sbp_energy_group": (I, [pp, I, C.POINTER(C.c_double)]),
                "sbp_energy_noalloc": (I, [P, P]),
                "sbp_energy_series": (I, [P, C.POINTER(C.c_double), I64, C.POINTER(C.c_int64)]),
                "sbp_sync": (I, [P]),
                "sbp_dt": (D, [P]),
                "sbp_step_index": (I64, [P]),
                "sbp_destroy": (I, [P]),
                "sbp_strerror": (C.c_char_p, [I]),
                "sbp_batch_create": (I, [P, I, pp]),
                "sbp_batch_add": (I, [P, P, I64]),
                "sbp_batch_remove": (I, [P, P]),
                "sbp_batch_remaining": (I, [P, P, C.POINTER(C.c_int64)]),
                "sbp_batch_step": (I, [P, I64]),
                "sbp_batch_size": (I, [P]),
                "sbp_batch_destroy": (I, [P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def exported_symbols() -> Sequence[str]:
    return ["sbp_create", "sbp_workspace_bytes", "sbp_create_in", "sbp_connect", "sbp_connect_phase", "sbp_set_field",
            "sbp_get_field", "sbp_add_source", "sbp_add_probe", "sbp_reserve_probes", "sbp_step",
            "sbp_step_group", "sbp_half_step_h", "sbp_half_step_e", "sbp_step_timed", "sbp_autotune", "sbp_tile", "sbp_get_probes", "sbp_energy", "sbp_energy_group", "sbp_energy_noalloc", "sbp_energy_series",
            "sbp_sync", "sbp_checkpoint_bytes", "sbp_save", "sbp_load", "sbp_dt", "sbp_step_index", "sbp_destroy", "sbp_strerror",
            "sbp_batch_create", "sbp_batch_add", "sbp_batch_remove", "sbp_batch_remaining", "sbp_batch_step",
            "sbp_batch_size", "sbp_batch_destroy", "sbp_server_create", "sbp_server_submit", "sbp_server_poll",
            "sbp_server_probes", "sbp_server_release", "sbp_server_drain", "sbp_server_stats", "sbp_server_destroy"]


def _strerror(code: int) -> str:
    try:
        return lib().sbp_strerror(code).decode()
    except Exception:  # pragma: no cover - library missing
        return "error"


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise SbpError(rc, what)
    return rc


def extents(n, comp):
    return tuple(int(n[a]) + (1 if ON_PLUS[comp][a] else 2) for a in range(3))


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Sim:
    """One block of the SBP-SAT FDTD leapfrog on the GPU (wraps ``sbp_sim``).

    n: cells (nx, ny, nz); h: mesh steps (dx, dy, dz) in metres; faces: six
    face types (x-, x+, y-, y+, z-, z+); eps_r / mu_r: per-cell arrays of shape
    (nz, ny, nx) or None; cfl: dt as a fraction of the CFL limit.
    torch_memory=True carves the device arrays from a torch uint8 tensor.
    """

    def __init__(self, n, h, faces, eps_r=None, mu_r=None, cfl=0.95, precision=FP32,
                 energy_every=0, flags=0, stream=None, torch_memory=True, field_scale=(0.0, 0.0)):
        L = lib()
        self.n = tuple(int(v) for v in n)
        self.h = tuple(float(v) for v in h)
        self.precision = precision
        self.dtype = np.float64 if precision == FP64 else np.float32
        self._keep = []
        d = GridDesc()
        d.nx, d.ny, d.nz = self.n
        d.dx, d.dy, d.dz = self.h
        ncell = self.n[0] * self.n[1] * self.n[2]
        for name, arr in (("eps_r", eps_r), ("mu_r", mu_r)):
            if arr is None:
                setattr(d, name, None)
                continue
            a = np.ascontiguousarray(np.asarray(arr, dtype=np.float32).reshape(-1))
            if a.size != ncell:
                raise ValueError(f"{name} must have nx*ny*nz = {ncell} entries")
            self._keep.append(a)
            setattr(d, name, a.ctypes.data_as(C.POINTER(C.c_float)))
        for f in range(6):
            d.face[f] = int(faces[f])
        d.cfl_fraction = float(cfl)
        d.precision = int(precision)
        d.energy_every = int(energy_every)
        d.flags = int(flags)
        d.field_scale[0], d.field_scale[1] = float(field_scale[0]), float(field_scale[1])
        self._desc = d
        self.stream = _stream_ptr(stream)
        import torch
        self.device = torch.cuda.current_device()   # the library creates the simulation on this device
        h_out = C.c_void_p()
        self._ws = None
        if torch_memory:
            import torch
            nbytes = L.sbp_workspace_bytes(C.byref(d))
            if nbytes == 0:
                raise SbpError(-1, "sbp_workspace_bytes")
            self._ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            _check(L.sbp_create_in(C.byref(d), self.stream, self._ws.data_ptr(), nbytes, C.byref(h_out)),
                   "sbp_create_in")
        else:
            _check(L.sbp_create(C.byref(d), self.stream, C.byref(h_out)), "sbp_create")
        self._keep.clear()
        self._h = h_out.value
        self.nprobes = 0

    # --- lifetime -------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().sbp_destroy(self._h)
            self._h = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # --- problem statement ----------------------------------------------
    def shape(self, comp):
        e = extents(self.n, comp)
        return (e[2], e[1], e[0])

    def connect(self, face, other: "Sim", other_face):
        _check(lib().sbp_connect(self._h, int(face), other._h, int(other_face)), "sbp_connect")

    def add_source(self, comp, i, j, k, kind, amp, tw, t0, f=0.0):
        return _check(lib().sbp_add_source(self._h, comp, i, j, k, kind, amp, tw, t0, f), "sbp_add_source")

    def add_probe(self, comp, i, j, k):
        pid = C.c_int()
        _check(lib().sbp_add_probe(self._h, comp, i, j, k, C.byref(pid)), "sbp_add_probe")
        self.nprobes += 1
        return pid.value

    def reserve_probes(self, nsteps):
        _check(lib().sbp_reserve_probes(self._h, int(nsteps)), "sbp_reserve_probes")
        self.probe_cap = int(nsteps)

    # --- fields ---------------------------------------------------------
    def set_field(self, comp, arr):
        """arr: numpy array (host) or CUDA torch tensor of the component's shape."""
        if hasattr(arr, "data_ptr") and getattr(arr, "is_cuda", False):
            if tuple(arr.shape) != self.shape(comp) or not arr.is_contiguous():
                raise ValueError("device tensor must be contiguous with the component's shape")
            _check(lib().sbp_set_field(self._h, comp, arr.data_ptr(), 1), "sbp_set_field")
            return
        a = np.ascontiguousarray(np.asarray(arr, dtype=self.dtype))
        if a.shape != self.shape(comp):
            raise ValueError(f"component {comp}: expected {self.shape(comp)}, got {a.shape}")
        _check(lib().sbp_set_field(self._h, comp, a.ctypes.data, 0), "sbp_set_field")

    def field(self, comp, out=None):
        """Host copy (numpy) of a component, or into a CUDA torch tensor ``out``."""
        if out is not None:
            _check(lib().sbp_get_field(self._h, comp, out.data_ptr(), 1), "sbp_get_field")
            return out
        a = np.empty(self.shape(comp), dtype=self.dtype)
        _check(lib().sbp_get_field(self._h, comp, a.ctypes.data, 0), "sbp_get_field")
        return a

    # --- time stepping --------------------------------------------------
    def step(self, nsteps):
        _check(lib().sbp_step(self._h, int(nsteps)), "sbp_step")

    KERNELS = ("h_update", "e_update", "band_h", "fused_interior", "band_e")

    def step_timed(self, nsteps):
        """Step with CUDA events around each launch: {kernel: (avg ms, launches)}."""
        ms = (C.c_double * 5)()
        cnt = (C.c_int64 * 5)()
        _check(lib().sbp_step_timed(self._h, int(nsteps), ms, cnt, 5), "sbp_step_timed")
        return {k: (ms[q], cnt[q]) for q, k in enumerate(self.KERNELS) if cnt[q]}

    def autotune(self, trial_steps=5):
        """Choose the tile of the one-pass step (64 x 8 / 64 x 16 / 128 x 8 / 128 x 12 H
        nodes, z-block depth) by timing candidates (state unchanged); returns (depth, ms per
        step); ``tile`` gives the whole tile."""
        depth, ms = C.c_int(), C.c_double()
        _check(lib().sbp_autotune(self._h, int(trial_steps), C.byref(depth), C.byref(ms)), "sbp_autotune")
        return depth.value, ms.value

    def tile(self):
        """(rows, depth, width) of the one-pass step's tile."""
        rows, depth, width = C.c_int(), C.c_int(), C.c_int()
        _check(lib().sbp_tile(self._h, C.byref(rows), C.byref(depth), C.byref(width)), "sbp_tile")
        return rows.value, depth.value, width.value

    def save(self) -> bytes:
        """Checkpoint: the simulation's state as bytes (sbp_save)."""
        n = lib().sbp_checkpoint_bytes(self._h)
        buf = C.create_string_buffer(n)
        _check(lib().sbp_save(self._h, buf, n), "sbp_save")
        return buf.raw

    def load(self, blob: bytes):
        """Restore a checkpoint written by ``save`` of a simulation with the same
        descriptor, sources and probes (sbp_load)."""
        buf = C.create_string_buffer(blob, len(blob))
        _check(lib().sbp_load(self._h, buf, len(blob)), "sbp_load")

    def sync(self):
        _check(lib().sbp_sync(self._h), "sbp_sync")

    @property
    def dt(self):
        return lib().sbp_dt(self._h)

    @property
    def step_index(self):
        return lib().sbp_step_index(self._h)

    def probes(self):
        cap = getattr(self, "probe_cap", 0)
        out = np.zeros((max(self.nprobes, 1), max(cap, 1)))
        ns = C.c_int64()
        _check(lib().sbp_get_probes(self._h, out.ctypes.data_as(C.POINTER(C.c_double)), max(cap, 1),
                                    C.byref(ns)), "sbp_get_probes")
        return out[: self.nprobes, : ns.value]

    def energy(self):
        w = C.c_double()
        _check(lib().sbp_energy(self._h, C.byref(w)), "sbp_energy")
        return w.value

    def energy_noalloc(self, out):
        """Write W^n into ``out`` (a CUDA float64 tensor with one element) on the simulation's
        stream, without allocating device memory (scratch is a fixed array in the library)."""
        import torch
        if (not isinstance(out, torch.Tensor) or out.dtype != torch.float64 or not out.is_cuda
                or out.numel() < 1 or out.device.index != self.device):
            raise ValueError(f"out must be a float64 tensor of at least one element on cuda:{self.device}")
        _check(lib().sbp_energy_noalloc(self._h, out.data_ptr()), "sbp_energy_noalloc")
        return out

    def energy_series(self):
        """(samples, rc): rc is 0 or SBP_EUNSTABLE (-4) when the monitor saw growth."""
        cnt = C.c_int64()
        rc = lib().sbp_energy_series(self._h, None, 0, C.byref(cnt))
        if rc < 0 and rc != -4:
            _check(rc, "sbp_energy_series")
        out = np.zeros(max(cnt.value, 1))
        rc = lib().sbp_energy_series(self._h, out.ctypes.data_as(C.POINTER(C.c_double)), cnt.value,
                                     C.byref(cnt))
        return out[: cnt.value], rc


def _handles(sims):
    return (C.c_void_p * len(sims))(*[s._h for s in sims])


def step_group(sims, nsteps):
    _check(lib().sbp_step_group(_handles(sims), len(sims), int(nsteps)), "sbp_step_group")


def half_step_h(sims):
    _check(lib().sbp_half_step_h(_handles(sims), len(sims)), "sbp_half_step_h")


def half_step_e(sims):
    _check(lib().sbp_half_step_e(_handles(sims), len(sims)), "sbp_half_step_e")


def energy_group(sims):
    w = C.c_double()
    _check(lib().sbp_energy_group(_handles(sims), len(sims), C.byref(w)), "sbp_energy_group")
    return w.value


def connect_phase(re: "Sim", im: "Sim", axis: int, alpha: float) -> None:
    """Periodic faces along ``axis`` with phase shift ``alpha`` for the complex field
    re + j im (two simulations advanced together with ``step_group``)."""
    _check(lib().sbp_connect_phase(re.handle, im.handle, int(axis), float(alpha)), "sbp_connect_phase")


def from_workload(w, precision=FP32, stream=None, torch_memory=True, energy_every=0, field_scale=(0.0, 0.0),
                  flags=0):
    """Create the GPU blocks of a workloads.Workload (fields, sources, probes, links).
    field_scale: (E, H) scales of FP16 storage (0 = library default); flags: FLAG_*."""
    sims = []
    for b in w.blocks:
        s = Sim(b.n, b.h, b.faces, eps_r=b.eps_r, mu_r=b.mu_r, cfl=w.cfl, precision=precision,
                stream=stream, torch_memory=torch_memory, energy_every=energy_every, field_scale=field_scale,
                flags=flags)
        if b.fields is not None:
            for c in range(6):
                s.set_field(c, b.fields[c])
        for src in b.sources:
            s.add_source(src.comp, src.i, src.j, src.k, src.kind, src.amp, src.tw, src.t0, src.f)
        for p in b.probes:
            s.add_probe(p.comp, p.i, p.j, p.k)
        sims.append(s)
    for a, fa, b, fb in w.links:
        sims[a].connect(fa, sims[b], fb)
    return sims


class Batch:
    """Continuous batching of many simulations: one launch per kernel kind per step covers every
    member (wraps ``sbp_batch``).  Members must be created on the batch's stream."""

    GRAPHS, PERSISTENT = 1, 2

    def __init__(self, stream=None, use_graphs=True, persistent=False):
        """use_graphs: replay each chunk as a CUDA graph; persistent: one persistent launch per
        chunk instead of three launches per step."""
        self.stream = _stream_ptr(stream)
        h = C.c_void_p()
        flags = (self.GRAPHS if use_graphs else 0) | (self.PERSISTENT if persistent else 0)
        _check(lib().sbp_batch_create(self.stream, flags, C.byref(h)), "sbp_batch_create")
        self._h = h.value
        self.members = []

    def add(self, sim: Sim, nsteps: int):
        _check(lib().sbp_batch_add(self._h, sim.handle, int(nsteps)), "sbp_batch_add")
        self.members.append(sim)

    def remove(self, sim: Sim):
        _check(lib().sbp_batch_remove(self._h, sim.handle), "sbp_batch_remove")
        self.members.remove(sim)

    def remaining(self, sim: Sim) -> int:
        r = C.c_int64()
        _check(lib().sbp_batch_remaining(self._h, sim.handle, C.byref(r)), "sbp_batch_remaining")
        return r.value

    def step(self, nsteps: int):
        _check(lib().sbp_batch_step(self._h, int(nsteps)), "sbp_batch_step")

    def close(self):
        if getattr(self, "_h", None):
            lib().sbp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SourceDesc(C.Structure):
    _fields_ = [("comp", C.c_int32), ("i", C.c_int32), ("j", C.c_int32), ("k", C.c_int32),
                ("waveform", C.c_int32), ("amp", C.c_double), ("tw", C.c_double), ("t0", C.c_double),
                ("f", C.c_double)]


class ProbeDesc(C.Structure):
    _fields_ = [("comp", C.c_int32), ("i", C.c_int32), ("j", C.c_int32), ("k", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("grid", GridDesc), ("nsteps", C.c_int64), ("nsources", C.c_int32),
                ("sources", C.POINTER(SourceDesc)), ("nprobes", C.c_int32), ("probes", C.POINTER(ProbeDesc))]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("steps", C.c_int64), ("submit_s", C.c_double),
                ("admit_s", C.c_double), ("done_s", C.c_double), ("nprobes", C.c_int32)]


_SERVER_SIGS = {
    "sbp_server_create": (C.c_int, [C.c_void_p, C.c_size_t, C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    "sbp_server_submit": (C.c_int, [C.c_void_p, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    "sbp_server_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(Result)]),
    "sbp_server_probes": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(C.c_double), C.c_int64]),
    "sbp_server_release": (C.c_int, [C.c_void_p, C.c_uint64]),
    "sbp_server_drain": (C.c_int, [C.c_void_p]),
    "sbp_server_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "sbp_server_destroy": (C.c_int, [C.c_void_p]),
}


def _server_lib():
    L = lib()
    if not getattr(L, "_server_sigs", False):
        for name, (res, args) in _SERVER_SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        L._server_sigs = True
    return L


class Server:
    """Request loop with continuous batching (wraps ``sbp_server``).  ``submit`` copies the
    request; a scheduler thread in the library admits, batches, steps and retires requests."""

    def __init__(self, stream=None, budget_bytes=0, max_slots=64, chunk=32):
        L = _server_lib()
        self.stream = _stream_ptr(stream)
        h = C.c_void_p()
        _check(L.sbp_server_create(self.stream, int(budget_bytes), int(max_slots), int(chunk), C.byref(h)),
               "sbp_server_create")
        self._h = h.value
        self.meta = {}

    def submit(self, spec, nsteps, cfl=0.95, energy_every=0, flags=0):
        """spec: workloads.BlockSpec (FP32, uniform mu, >= 8 cells per axis, no interfaces).
        energy_every > 0 turns on the FP64 energy monitor (sampled at chunk boundaries whose
        step is a multiple of it); flags: FLAG_* of the grid descriptor."""
        d = GridDesc()
        d.nx, d.ny, d.nz = spec.n
        d.dx, d.dy, d.dz = spec.h
        eps = None
        if spec.eps_r is not None:
            eps = np.ascontiguousarray(np.asarray(spec.eps_r, dtype=np.float32).reshape(-1))
            d.eps_r = eps.ctypes.data_as(C.POINTER(C.c_float))
        d.mu_r = None
        for f in range(6):
            d.face[f] = int(spec.faces[f])
        d.cfl_fraction = float(cfl)
        d.precision = FP32
        d.energy_every = int(energy_every)
        d.flags = int(flags)
        srcs = (SourceDesc * max(len(spec.sources), 1))()
        for q, s in enumerate(spec.sources):
            srcs[q] = SourceDesc(s.comp, s.i, s.j, s.k, s.kind, s.amp, s.tw, s.t0, s.f)
        prbs = (ProbeDesc * max(len(spec.probes), 1))()
        for q, p in enumerate(spec.probes):
            prbs[q] = ProbeDesc(p.comp, p.i, p.j, p.k)
        r = Request(d, int(nsteps), len(spec.sources), srcs, len(spec.probes), prbs)
        t = C.c_uint64()
        _check(_server_lib().sbp_server_submit(self._h, C.byref(r), C.byref(t)), "sbp_server_submit")
        self.meta[t.value] = (len(spec.probes), int(nsteps), int(np.prod(spec.n)))
        return t.value

    def poll(self, ticket):
        res = Result()
        rc = _server_lib().sbp_server_poll(self._h, ticket, C.byref(res))
        if rc == -9:
            return None
        _check(rc, "sbp_server_poll")
        return res

    def probes(self, ticket):
        npr, nsteps, _ = self.meta[ticket]
        out = np.zeros((max(npr, 1), max(nsteps, 1)))
        _check(_server_lib().sbp_server_probes(self._h, ticket, out.ctypes.data_as(C.POINTER(C.c_double)),
                                               max(nsteps, 1)), "sbp_server_probes")
        return out[:npr, :nsteps]

    def release(self, ticket):
        _check(_server_lib().sbp_server_release(self._h, ticket), "sbp_server_release")
        self.meta.pop(ticket, None)

    def drain(self):
        _check(_server_lib().sbp_server_drain(self._h), "sbp_server_drain")

    def stats(self):
        cu, span = C.c_double(), C.c_double()
        _check(_server_lib().sbp_server_stats(self._h, C.byref(cu), C.byref(span)), "sbp_server_stats")
        return cu.value, span.value

    def close(self):
        if getattr(self, "_h", None):
            _server_lib().sbp_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
