"""CPU-side checks of the C ABI: the library builds, loads and exports every declared symbol.

No compute call is made here (there is no GPU on this side)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names.update(re.findall(r"\b(sbp_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_entry_points():
    names = _declared()
    for must in ("sbp_create", "sbp_step", "sbp_energy", "sbp_get_probes", "sbp_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2206_00638_gb300 import sbpsat
    path = sbpsat.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(sbpsat.exported_symbols()) <= set(_declared())


def test_strerror_and_workspace_bytes_without_gpu():
    from paper_2206_00638_gb300 import sbpsat
    L = sbpsat.lib()
    assert L.sbp_strerror(-4).decode().startswith("energy monitor")
    d = sbpsat.GridDesc()
    d.nx, d.ny, d.nz = 8, 9, 10
    d.dx = d.dy = d.dz = 1e-3
    d.cfl_fraction = 0.9
    d.precision = 0
    for f in range(6):
        d.face[f] = 0
    nbytes = L.sbp_workspace_bytes(ctypes.byref(d))
    # six padded FP32 fields + padded eps + partials: at least 7 * (nx+2)(ny+2)(nz+2) * 4 bytes
    assert nbytes >= 7 * 10 * 11 * 12 * 4
    d.nx = 3                                  # closures would overlap: rejected
    assert L.sbp_workspace_bytes(ctypes.byref(d)) == 0
    d.nx = 8
    d.cfl_fraction = 1.2                      # above the CFL limit without the flag
    assert L.sbp_workspace_bytes(ctypes.byref(d)) == 0
    d.flags = sbpsat.FLAG_ALLOW_UNSTABLE
    assert L.sbp_workspace_bytes(ctypes.byref(d)) > 0


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf"), 0.0, -2.0, 9.9e-4])
@pytest.mark.parametrize("which", ["eps_r", "mu_r"])
def test_workspace_bytes_rejects_bad_material_cells(bad, which):
    """Every eps_r / mu_r cell must be finite and >= 1e-3; one bad cell anywhere (here the
    last, and one in the middle of a run of good cells) rejects the grid."""
    import numpy as np
    from paper_2206_00638_gb300 import sbpsat
    L = sbpsat.lib()
    d = sbpsat.GridDesc()
    d.nx, d.ny, d.nz = 17, 9, 10
    d.dx = d.dy = d.dz = 1e-3
    d.cfl_fraction = 0.9
    d.precision = 0
    for f in range(6):
        d.face[f] = 0
    cells = np.full(17 * 9 * 10, 2.5, dtype=np.float32)
    cells[:5] = 1e-3                          # the smallest accepted value
    setattr(d, which, cells.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    assert L.sbp_workspace_bytes(ctypes.byref(d)) > 0
    for pos in (cells.size - 1, 777):
        c2 = cells.copy()
        c2[pos] = bad
        setattr(d, which, c2.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        assert L.sbp_workspace_bytes(ctypes.byref(d)) == 0, (bad, pos)


def test_no_cpu_fallback_in_product_path():
    """The binding never imports the oracle (the only CPU implementation)."""
    src = open(os.path.join(ROOT, "paper_2206_00638_gb300", "sbpsat.py")).read()
    assert "import oracle" not in src and "from oracle" not in src
