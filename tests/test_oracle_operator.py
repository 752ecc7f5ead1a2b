"""Pins of the oracle's operator A (Section 3, Eq. 9, SPD form, plus the mass
shift of Section 2, Eq. 2) against things other than the oracle itself: a
hand-derived fixture, structural counts taken straight from the mask, the
zero-flux row-sum identity, and the closed-form Fourier spectrum of the
constant-coefficient periodic/closed operator."""
import math

import numpy as np
import pytest

import gridgen
import oracle
from conftest import load_golden


def _fields_from_golden(name):
    g = load_golden(name)
    wet = np.array(g["wet"], dtype=np.uint8)
    return (wet, np.array(g["c_e"]), np.array(g["c_n"]), np.array(g["shift"]), np.array(g["A"]))


def test_hand_derived_operator():
    wet, ce, cn, sh, A_expected = _fields_from_golden("operator_3x2.txt")
    P = oracle.OracleProblem(3, 2, wet, ce, cn, sh)
    assert P.n == 5
    np.testing.assert_array_equal(P.dense(), A_expected)
    x = np.array([1.0, -2.0, 0.5, 3.0, -1.5])
    np.testing.assert_allclose(P.spmv(x), A_expected @ x, rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed_cfg", [(gridgen.TINY, 0), (gridgen.COARSE, 1)])
def test_symmetry_rowsums_and_nnz(seed_cfg):
    cfg, ci = seed_cfg
    g = gridgen.make_grid(seed=gridgen.seed_for(ci), **cfg)
    P = oracle.OracleProblem.from_grid(g)
    rp, col, val, pi, pj = P.csr()
    n = P.n
    assert n == int(g.wet.sum())
    # natural ordering: (j, i) lexicographic
    key = pj.astype(np.int64) * g.nx + pi
    assert np.all(np.diff(key) > 0)
    # exact symmetry of the stored entries
    rows = np.repeat(np.arange(n), np.diff(rp))
    S = {(int(r), int(c)): v for r, c, v in zip(rows, col, val)}
    for (r, c), v in S.items():
        assert S[(c, r)] == v
    # off-diagonals are non-positive, diagonal positive (an M-matrix)
    off = rows != col
    assert np.all(val[off] < 0) and np.all(val[~off] > 0)
    # zero-flux rows: A * 1 = shift on the wet points
    np.testing.assert_allclose(P.spmv(np.ones(n)), P.to_wet(g.shift), rtol=1e-12, atol=1e-9)
    # nnz = n + 2 * (# faces between two wet cells), counted from the mask alone
    w = g.wet.astype(bool)
    faces_e = int((w & np.roll(w, -1, axis=1)).sum()) if g.nx > 2 else None
    faces_n = int((w[:-1] & w[1:]).sum())
    assert len(val) == n + 2 * (faces_e + faces_n)


def _constant_fields(nx, ny, ce, cn, s):
    wet = np.ones((ny, nx), np.uint8)
    c_e = np.full((ny, nx), ce)
    c_n = np.full((ny, nx), cn)
    c_n[-1, :] = 0.0
    return wet, c_e, c_n, np.full((ny, nx), s)


def test_closed_form_spectrum():
    """Constant coefficients, all wet: A = s I + c_E (periodic 1-D Laplacian in i)
    + c_N (Neumann 1-D Laplacian in j); its eigenpairs are
    lambda_pq = s + 2 c_E (1 - cos 2 pi p / nx) + 2 c_N (1 - cos pi q / ny),
    v = cos(2 pi p i / nx + theta) cos(pi q (j + 1/2) / ny)."""
    nx, ny, ce, cn, s = 9, 6, 3.0, 5.0, 0.7
    P = oracle.OracleProblem(nx, ny, *_constant_fields(nx, ny, ce, cn, s))
    I, J = np.meshgrid(np.arange(nx), np.arange(ny))
    for p in range(nx):
        for q in range(ny):
            lam = s + 2 * ce * (1 - math.cos(2 * math.pi * p / nx)) + 2 * cn * (1 - math.cos(math.pi * q / ny))
            for theta in (0.0, 0.3):
                v = np.cos(2 * math.pi * p * I / nx + theta) * np.cos(math.pi * q * (J + 0.5) / ny)
                vw = P.to_wet(v)
                if np.linalg.norm(vw) < 1e-8:
                    continue
                np.testing.assert_allclose(P.spmv(vw), lam * vw, rtol=0, atol=1e-12 * lam * np.abs(vw).max() + 1e-13)
    ev = np.sort(np.linalg.eigvalsh(P.dense()))
    lam_all = np.sort([s + 2 * ce * (1 - math.cos(2 * math.pi * p / nx)) + 2 * cn * (1 - math.cos(math.pi * q / ny))
                       for p in range(nx) for q in range(ny)])
    np.testing.assert_allclose(ev, lam_all, rtol=1e-12)


def test_cg_on_eigenvectors_terminates():
    """On one periodic latitude row every diagonal equals s + 2 c_E, so the Jacobi
    preconditioner is a scalar and CG on a right-hand side made of m eigenmodes
    with distinct eigenvalues ends in at most m steps."""
    nx = 16
    wet, ce, cn, sh = _constant_fields(nx, 1, 2.0, 0.0, 0.5)
    P = oracle.OracleProblem(nx, 1, wet, ce, cn, sh)
    assert P.ainv(oracle.PAT_DIAG) == oracle.OK
    i = np.arange(nx)
    mode = lambda p: np.cos(2 * math.pi * p * i / nx + 0.2)
    r1 = P.pcg(mode(3), rtol=1e-12, max_replace=0)
    assert r1.iters == 1 and r1.status == oracle.OK
    b3 = mode(1) + 0.5 * mode(2) - 2.0 * mode(5)
    r3 = P.pcg(b3, rtol=1e-12, max_replace=0)
    assert r3.iters <= 3 and r3.status == oracle.OK
