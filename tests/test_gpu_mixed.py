"""Mixed precision (binary32 inner PCG inside binary64 iterative refinement):
the result must meet the same acceptance as the binary64 solve -- the true
residual ||b - A x|| / ||b||, recomputed by the FP64 oracle from the returned
x, at most rtol, and x within 1e-8 of the tight reference solution -- and a
grid's result must not depend on the other members of a batch."""
import numpy as np
import pytest

import gridgen
import oracle
from oracle_checks import judge

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


CASES = [
    ("tiny-trilA", dict(gridgen.TINY), 0, 0, 0.0),
    ("coarse-trilA2", dict(gridgen.COARSE), 1, 1, 0.05),
    ("ragged-trilA", dict(nx=203, ny=77, land=0.3), 7, 0, 0.0),
    ("orca025-trilA2", dict(gridgen.ORCA025), 2, 1, 0.05),
]


@pytest.mark.parametrize("name,cfg,ci,pattern,tau", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("inner_rtol", [1e-5, 1e-3])
def test_mixed_meets_fp64_acceptance(name, cfg, ci, pattern, tau, inner_rtol):
    import paper_1210_1878_b300 as pcg
    g = gridgen.make_grid(seed=gridgen.seed_for(ci), **cfg)
    P = oracle.OracleProblem.from_grid(g)
    b = P.to_wet(g.b)
    h = pcg.ainv_setup_grid(g, pattern=pattern, drop_tol=tau)
    x = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
    st = pcg.pcg_solve(h, _dev(g.b), x, pcg.make_opts(rtol=1e-10, prec=pcg.PCG_MIXED, inner_rtol=inner_rtol))
    assert st.status == pcg.PCG_OK and st.outer_iters >= 1
    judge(P, g, b, x.cpu().numpy(), rtol=1e-10, stats=st)


def test_mixed_batched_matches_oracle_and_alone():
    """Each member of a mixed-precision batch meets the oracle's acceptance
    (binary64 true residual recomputed by the oracle, distance to the tight
    reference) and equals the same solve alone, bit for bit."""
    import paper_1210_1878_b300 as pcg
    specs = [(dict(gridgen.COARSE), 1), (dict(gridgen.ORCA1), 3), (dict(gridgen.TINY), 0)]
    grids = [gridgen.make_grid(seed=gridgen.seed_for(ci), **cfg) for cfg, ci in specs]
    hs = [pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A2, drop_tol=0.05) for g in grids]
    opts = pcg.make_opts(rtol=1e-10, prec=pcg.PCG_MIXED)
    alone = []
    for h, g in zip(hs, grids):
        x = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
        st = pcg.pcg_solve(h, _dev(g.b), x, opts)
        alone.append((x.cpu().numpy(), st.iters, st.outer_iters))
    xs = [torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda") for g in grids]
    rc, stats = pcg.pcg_solve_batched(hs, [_dev(g.b) for g in grids], xs, opts)
    assert rc == pcg.PCG_OK
    for (xa, ia, oa), xb, st, g in zip(alone, xs, stats, grids):
        assert st.status == pcg.PCG_OK and (st.iters, st.outer_iters) == (ia, oa)
        xbn = xb.cpu().numpy()
        np.testing.assert_array_equal(xbn, xa)
        P = oracle.OracleProblem.from_grid(g)
        judge(P, g, P.to_wet(g.b), xbn, rtol=1e-10, stats=st)


def test_mixed_zero_rhs_and_warm_start():
    import paper_1210_1878_b300 as pcg
    g = gridgen.make_grid(seed=gridgen.seed_for(1), **gridgen.COARSE)
    h = pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A2, drop_tol=0.05)
    opts = pcg.make_opts(rtol=1e-10, prec=pcg.PCG_MIXED)
    x = torch.full((g.ny, g.nx), 3.0, dtype=torch.float64, device="cuda")
    st = pcg.pcg_solve(h, torch.zeros_like(x), x, opts)
    assert st.status == pcg.PCG_OK and st.iters == 0 and float(x.abs().max()) == 0.0
    st = pcg.pcg_solve(h, _dev(g.b), x, opts)
    assert st.status == pcg.PCG_OK
    st2 = pcg.pcg_solve(h, _dev(g.b), x, pcg.make_opts(rtol=1e-10, prec=pcg.PCG_MIXED, use_x0=True))
    assert st2.status == pcg.PCG_OK and st2.iters == 0
