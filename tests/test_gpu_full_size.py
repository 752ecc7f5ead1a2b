"""Parity at the full 4322 x 3059 size (9,254,699 wet points), in the launch
configuration the benchmark times: default strips chosen at setup, persistent
launches, the graph loop.

Element by element against the oracle: q = A v (Section 3, Eq. 9) and
s = Z D^-1 Z^T r (the preconditioning step of Algorithm 1) over every point,
with the rounding bounds of the smaller parity tests. For whole solves: the
iteration count within 2 of the oracle's count for the same grid and
right-hand side (recorded by ``oracle/record_iterations.py``), the true
relative residual of the returned x, recomputed by the oracle, at most 1e-10,
and x within 1e-8 of the tight reference solution (the oracle's own PCG run
to 1e-13, about a minute of CPU time, computed once for all four solves),
in both precisions."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import gridgen
import oracle
from oracle_checks import tight_reference

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ITERS = json.load(open(os.path.join(ROOT, "oracle", "iterations.json")))


@pytest.fixture(scope="module")
def full():
    """The 4322 x 3059 grid of the benchmark (same seed), its oracle problem and
    the library handles of both patterns the benchmark runs."""
    import paper_1210_1878_b300 as pcg
    g = gridgen.make_grid(seed=gridgen.seed_for(4), **gridgen.ORCA12)
    P = oracle.OracleProblem.from_grid(g)
    hs = {1: pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A2, drop_tol=0.05),
          0: pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A)}
    yield pcg, g, P, hs
    for h in hs.values():
        h.close()


@pytest.fixture(scope="module")
def x_ref(full):
    """A x_ref = b for the benchmark's right-hand side, by the oracle alone."""
    pcg, g, P, hs = full
    return tight_reference(P, P.to_wet(g.b))


def _csr(P):
    rp, col, val, _, _ = P.csr()
    return sp.csr_matrix((val, col, rp), shape=(P.n, P.n))


def test_full_size_spmv(full):
    pcg, g, P, hs = full
    rng = np.random.default_rng(31)
    v = rng.standard_normal((g.ny, g.nx))
    q = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
    pcg.pcg_spmv(hs[1], torch.from_numpy(v).cuda(), q)
    vw = P.to_wet(v)
    qo = P.spmv(vw)
    mag = abs(_csr(P)) @ np.abs(vw)
    qg = q.cpu().numpy()
    err = np.abs(P.to_wet(qg) - qo)
    assert np.all(err <= 1e-13 * mag + 1e-300), float((err / (mag + 1e-300)).max())
    assert np.all(qg[g.wet == 0] == 0)


def test_full_size_precond(full):
    pcg, g, P, hs = full
    assert P.ainv(oracle.PAT_TRIL_A2, 0.05, 0) == oracle.OK
    rng = np.random.default_rng(32)
    r = rng.standard_normal((g.ny, g.nx))
    s = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
    pcg.pcg_precond_apply(hs[1], torch.from_numpy(r).cuda(), s)
    rw = P.to_wet(r)
    so = P.apply(rw)
    cp, row, val, d = P.z()
    Z = sp.csc_matrix((np.abs(val), row, cp), shape=(P.n, P.n))
    mag = Z @ ((Z.T @ np.abs(rw)) / d)
    sg = s.cpu().numpy()
    err = np.abs(P.to_wet(sg) - so)
    assert np.all(err <= 1e-13 * mag + 1e-300), float((err / (mag + 1e-300)).max())
    assert np.all(sg[g.wet == 0] == 0)


@pytest.mark.parametrize("pattern,prec,key", [(1, 0, "orca12-fp64"), (0, 0, "orca12-fp64-trilA"),
                                              (1, 1, None), (0, 1, None)],
                         ids=["trilA2-fp64", "trilA-fp64", "trilA2-mixed", "trilA-mixed"])
def test_full_size_solve(full, x_ref, pattern, prec, key):
    pcg, g, P, hs = full
    b = torch.from_numpy(g.b).cuda()
    x = torch.zeros_like(b)
    st = pcg.pcg_solve(hs[pattern], b, x, pcg.make_opts(rtol=1e-10, max_iter=5000, prec=prec))
    assert st.status == pcg.PCG_OK
    if key is not None:                          # binary64: the oracle's iteration count
        assert abs(st.iters - ITERS[key]) <= 2, (st.iters, ITERS[key])
    xg = x.cpu().numpy()
    assert np.all(xg[g.wet == 0] == 0)
    bw = P.to_wet(g.b)
    xw = P.to_wet(xg)
    true_rel = np.linalg.norm(bw - P.spmv(xw)) / np.linalg.norm(bw)
    assert true_rel <= 1e-10 * (1 + 1e-3), true_rel
    assert abs(st.true_relres - true_rel) <= 1e-3 * 1e-10 + 1e-3 * true_rel
    err = np.linalg.norm(xw - x_ref) / np.linalg.norm(x_ref)
    assert err <= 1e-8, err


def test_full_size_f32_kernels(full):
    """The binary32 kernels of the mixed mode (its default strips) at full size,
    element by element: bound 32 u (u = 2^-24) of the absolute-value products,
    as in the smaller binary32 parity tests."""
    pcg, g, P, hs = full
    assert P.ainv(oracle.PAT_TRIL_A2, 0.05, 0) == oracle.OK
    tol = 32 * 2.0 ** -24
    rng = np.random.default_rng(33)
    v = rng.standard_normal((g.ny, g.nx))
    out = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
    pcg.pcg_apply_f32(hs[1], 0, torch.from_numpy(v).cuda(), out)
    vw = P.to_wet(v)
    err = np.abs(P.to_wet(out.cpu().numpy()) - P.spmv(vw))
    assert np.all(err <= tol * (abs(_csr(P)) @ np.abs(vw)) + 1e-300)
    pcg.pcg_apply_f32(hs[1], 1, torch.from_numpy(v).cuda(), out)
    cp, row, val, d = P.z()
    Z = sp.csc_matrix((np.abs(val), row, cp), shape=(P.n, P.n))
    err = np.abs(P.to_wet(out.cpu().numpy()) - P.apply(vw))
    assert np.all(err <= tol * (Z @ ((Z.T @ np.abs(vw)) / d)) + 1e-300)
    assert pcg.pcg_tiles(hs[1], 1)[0] == 124
