"""The narrowest device grids, 4 and 5 columns (the periodic copies of the
strip layout need at least 4): every column has a periodic copy on both
sides. Operator, preconditioner apply and whole solves (binary64 and mixed)
against the FP64 CPU oracle, with the tolerances of the other parity tests
(Section 3, Eq. 9; the preconditioning step and stopping rule of Algorithm 1)."""
import numpy as np
import pytest
import scipy.sparse as sp

import gridgen
import oracle
from oracle_checks import judge

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# (name, grid, seed offset, pattern, drop tolerance, band q)
CASES = [
    ("nx4-trilA", dict(nx=4, ny=33, land=0.0), 21, 0, 0.0, 0),
    ("nx4-jacobi", dict(nx=4, ny=33, land=0.0), 21, 4, 0.0, 0),
    ("nx4-bandT3", dict(nx=4, ny=33, land=0.0), 21, 3, 0.0, 3),
    ("nx5-trilA2", dict(nx=5, ny=47, land=0.2), 22, 1, 0.0, 0),
    ("nx5-trilA2-drop", dict(nx=5, ny=47, land=0.2), 22, 1, 0.05, 0),
]


def _pcg():
    import paper_1210_1878_b300 as pcg
    return pcg


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _case(cfg, off):
    return gridgen.make_grid(seed=gridgen.seed_for(0) + 100 * off, **cfg)


@pytest.mark.parametrize("name,cfg,off,pattern,tau,q", CASES, ids=[c[0] for c in CASES])
def test_narrow_operator_and_preconditioner(name, cfg, off, pattern, tau, q):
    pcg = _pcg()
    g = _case(cfg, off)
    P = oracle.OracleProblem.from_grid(g)
    assert P.ainv(pattern, tau, q) == oracle.OK
    h = pcg.ainv_setup_grid(g, pattern=pattern, drop_tol=tau, band_q=q)
    rng = np.random.default_rng(31)
    v = rng.standard_normal((g.ny, g.nx))
    out = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
    # A v, element by element within binary64 rounding of |A| |v|
    pcg.pcg_spmv(h, _dev(v), out)
    rp, col, val, _, _ = P.csr()
    A = sp.csr_matrix((val, col, rp), shape=(P.n, P.n))
    qo = P.to_grid(P.spmv(P.to_wet(v)))
    mag = P.to_grid(abs(A) @ np.abs(P.to_wet(v)))
    assert np.all(np.abs(out.cpu().numpy() - qo) <= 1e-13 * mag + 1e-300)
    # M^-1 v = Z D^-1 Z^T v, within binary64 rounding of |Z| D^-1 |Z|^T |v|
    pcg.pcg_precond_apply(h, _dev(v), out)
    so = P.to_grid(P.apply(P.to_wet(v)))
    cp, row, zv, d = P.z()
    Z = sp.csc_matrix((np.abs(zv), row, cp), shape=(P.n, P.n))
    mag = P.to_grid(Z @ ((Z.T @ np.abs(P.to_wet(v))) / d))
    assert np.all(np.abs(out.cpu().numpy() - so) <= 1e-13 * mag + 1e-300)
    assert np.all(out.cpu().numpy()[g.wet == 0] == 0)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name,cfg,off,pattern,tau,q", CASES, ids=[c[0] for c in CASES])
def test_narrow_solve_matches_oracle(name, cfg, off, pattern, tau, q, prec):
    pcg = _pcg()
    g = _case(cfg, off)
    P = oracle.OracleProblem.from_grid(g)
    assert P.ainv(pattern, tau, q) == oracle.OK
    b = P.to_wet(g.b)
    ref = P.pcg(b, rtol=1e-10)
    assert ref.status == oracle.OK
    h = pcg.ainv_setup_grid(g, pattern=pattern, drop_tol=tau, band_q=q)
    x = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
    st = pcg.pcg_solve(h, _dev(g.b), x, pcg.make_opts(rtol=1e-10, prec=prec))
    assert st.status == pcg.PCG_OK
    if prec == 0:
        assert abs(st.iters - ref.iters) <= 2, (st.iters, ref.iters)
    judge(P, g, b, x.cpu().numpy(), rtol=1e-10, stats=st)
