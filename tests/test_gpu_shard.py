"""Row-band sharded solve of one grid (pcg_shard_*), on one GPU: the grid's
rows split into 2 or 3 bands of about equal wet count, each band with its own
planes and halo rows, the band-edge rows exchanged after every kernel, one
reduction over all bands. Algorithm 1 is unchanged, so the result must meet
the same acceptance as the whole-grid solve: true residual recomputed by the
FP64 oracle at most rtol, x within 1e-8 of the oracle's tight reference, and
the iteration count within 2 of the oracle's."""
import numpy as np
import pytest

import gridgen
import oracle
from oracle_checks import judge

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [
    ("coarse-trilA2", dict(gridgen.COARSE), 1, 1, 0.05),
    ("coarse-trilA", dict(gridgen.COARSE), 1, 0, 0.0),
    ("ragged-trilA2", dict(nx=203, ny=77, land=0.3), 7, 1, 0.05),
    ("orca1-trilA2", dict(gridgen.ORCA1), 3, 1, 0.05),
    ("orca1-jacobi", dict(gridgen.ORCA1), 3, 4, 0.0),
    ("orca025-trilA2", dict(gridgen.ORCA025), 2, 1, 0.05),
]


@pytest.mark.parametrize("name,cfg,ci,pattern,tau", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("nbands", [2, 3])
def test_shard_solve_matches_oracle(name, cfg, ci, pattern, tau, nbands):
    import paper_1210_1878_b300 as pcg
    g = gridgen.make_grid(seed=gridgen.seed_for(ci), **cfg)
    P = oracle.OracleProblem.from_grid(g)
    assert P.ainv(pattern, tau) == oracle.OK
    b = P.to_wet(g.b)
    ref = P.pcg(b, rtol=1e-10)
    h = pcg.ainv_setup_grid(g, pattern=pattern, drop_tol=tau)
    sh = pcg.Shard(h, nbands)
    row0, halo = sh.bands()
    plan, halo2 = pcg.pcg_band_plan(g.wet, pattern, nbands)
    np.testing.assert_array_equal(row0, plan)
    assert halo == halo2 == max(1, {1: 2, 0: 1}.get(pattern, 0))
    x = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
    st = sh.solve(torch.from_numpy(g.b).cuda(), x, pcg.make_opts(rtol=1e-10))
    assert st.status == pcg.PCG_OK
    assert abs(st.iters - ref.iters) <= 2, (st.iters, ref.iters)
    judge(P, g, b, x.cpu().numpy(), rtol=1e-10, stats=st)
    # warm start from the solution: nothing left to do
    st2 = sh.solve(torch.from_numpy(g.b).cuda(), x, pcg.make_opts(rtol=1e-10, use_x0=True))
    assert st2.status == pcg.PCG_OK and st2.iters == 0
    sh.close()


def test_shard_agrees_with_whole_grid_solve():
    """The same solve as bands and as one grid: the same kernels on the same
    rows, only the order of the reductions' additions differs (per unit, units
    numbered band after band), so the iterates stay within rounding of each
    other: iteration counts within 1 and solutions within 1e-8."""
    import paper_1210_1878_b300 as pcg
    g = gridgen.make_grid(seed=gridgen.seed_for(1), **gridgen.COARSE)
    h = pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A2, drop_tol=0.05)
    b = torch.from_numpy(g.b).cuda()
    x1 = torch.zeros_like(b)
    x2 = torch.zeros_like(b)
    st1 = pcg.pcg_solve(h, b, x1)
    sh = pcg.Shard(h, 2)
    st2 = sh.solve(b, x2)
    assert abs(st1.iters - st2.iters) <= 1
    d = (x1 - x2).norm().item() / x1.norm().item()
    assert d <= 1e-8, d
    sh.close()
