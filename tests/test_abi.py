"""The C-ABI library loads on a machine without a GPU and exports every
function that include/pcg.h declares; host-only entry points validate their
input."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "pcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?[\s\*]+([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if not n.startswith("void") and n not in ("if",)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("ainv_setup", "pcg_solve", "pcg_solve_batched", "solver_server_create", "solver_server_submit",
                 "solver_server_wait", "solver_server_stats", "solver_server_destroy", "pcg_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_1210_1878_b300 as pcg
    lib = ctypes.CDLL(pcg.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(pcg.EXPORTED) <= set(_declared())


def test_status_strings():
    import paper_1210_1878_b300 as pcg
    assert pcg.lib.pcg_status_string(pcg.PCG_OK) == b"ok"
    assert pcg.lib.pcg_status_string(pcg.PCG_EBREAKDOWN) == b"breakdown"


def _fields(nx=8, ny=5):
    wet = np.ones((ny, nx), np.uint8)
    return nx, ny, wet, np.ones((ny, nx)), np.ones((ny, nx)), np.ones((ny, nx))


@pytest.mark.parametrize("mutate,pattern,band_q", [
    (lambda f: f.__setitem__(0, 2), 0, 0),                              # nx < 3
    (lambda f: f.__setitem__(0, 4), 1, 0),                              # tril(A^2) with nx < 5
    (lambda f: f[3].__setitem__((1, 1), -1.0), 0, 0),                   # negative face coefficient
    (lambda f: f[4].__setitem__((2, 2), np.nan), 0, 0),                 # NaN coefficient
    (lambda f: f[5].__setitem__((0, 0), 0.0), 0, 0),                    # zero shift on a wet cell
    (lambda f: None, 2, 0),                                             # dense pattern: oracle only
    (lambda f: None, 3, 9),                                             # band_q out of range
    (lambda f: None, 7, 0),                                             # unknown pattern
])
def test_host_factor_rejects_invalid_input(mutate, pattern, band_q):
    import paper_1210_1878_b300 as pcg
    f = list(_fields())
    mutate(f)
    nx, ny = f[0], f[1]
    wet, ce, cn, sh = [np.ascontiguousarray(a[:ny, :max(nx, 1)]) for a in f[2:]]
    with pytest.raises(pcg.PCGError) as e:
        pcg.ainv_factor_host(nx, ny, wet, ce, cn, sh, pattern=pattern, band_q=band_q)
    assert e.value.status == pcg.PCG_EINVAL


def test_device_setup_refuses_grids_narrower_than_four_columns():
    """The device layout keeps one periodic copy of a column per side, so a
    device handle needs nx >= 4; the refusal comes before any device call."""
    import paper_1210_1878_b300 as pcg
    nx, ny, wet, ce, cn, sh = _fields(nx=3, ny=5)
    with pytest.raises(pcg.PCGError) as e:
        pcg.ainv_setup(nx, ny, wet, ce, cn, sh, pattern=pcg.PCG_PAT_TRIL_A)
    assert e.value.status == pcg.PCG_EINVAL
    assert "4 columns" in str(e.value)
