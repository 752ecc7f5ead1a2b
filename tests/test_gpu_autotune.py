"""Strip-shape autotuner (batching row: tile shapes chosen by measurement):
the tuned shape is one of the candidates, is applied to the handle, is
remembered for later handles of the same grid shape, and solves on retiled
planes still meet the acceptance test (true relative residual <= 1e-10,
recomputed by the oracle)."""
import numpy as np
import pytest

import gridgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# a grid shape used by no other test (the tuned shapes are kept per process)
CFG = dict(nx=150, ny=97, land=0.3)


def _check_solve(pcg, h, g, prec):
    P = oracle.OracleProblem.from_grid(g)
    b = P.to_wet(g.b)
    x = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
    st = pcg.pcg_solve(h, torch.from_numpy(g.b).cuda(), x, pcg.make_opts(rtol=1e-10, prec=prec))
    assert st.status == pcg.PCG_OK
    xw = P.to_wet(x.cpu().numpy())
    assert np.linalg.norm(b - P.spmv(xw)) / np.linalg.norm(b) <= 1e-10 * (1 + 1e-3)


@pytest.mark.parametrize("prec", [1, 0])
def test_autotune_applies_and_remembers(prec):
    """Objective 0 (alone): later handles of the shape start with it."""
    import paper_1210_1878_b300 as pcg
    g = gridgen.make_grid(seed=gridgen.seed_for(5), **CFG)
    h = pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A2, drop_tol=0.05)
    tx, ty = pcg.pcg_autotune(h, prec)
    # candidates: 64, 128 and the whole-warp widths of tril(A^2) (60 and 92 binary64, 124 binary32)
    assert tx in ((64, 128, 60, 92) if prec == 0 else (64, 128, 124)) and ty in (8, 16, 32, 64)
    assert pcg.pcg_tiles(h, prec) == (tx, ty)
    _check_solve(pcg, h, g, prec)
    # a later handle of the same grid shape starts with the tuned strips
    g2 = gridgen.make_grid(seed=gridgen.seed_for(6), **CFG)
    h2 = pcg.ainv_setup_grid(g2, pattern=pcg.PCG_PAT_TRIL_A2, drop_tol=0.05)
    if prec == 1:
        pcg.pcg_apply_f32(h2, 0, torch.zeros((g2.ny, g2.nx), dtype=torch.float64, device="cuda"),
                          torch.zeros((g2.ny, g2.nx), dtype=torch.float64, device="cuda"))
    assert pcg.pcg_tiles(h2, prec) == (tx, ty)
    _check_solve(pcg, h2, g2, prec)
    # a second call is a cache hit: same answer
    assert pcg.pcg_autotune(h2, prec) == (tx, ty)


def test_autotune_throughput_objective():
    """Objective 1 (as a batch member) is kept apart from objective 0 and
    applied on request; the retiled handle still solves correctly."""
    import paper_1210_1878_b300 as pcg
    cfg = dict(nx=170, ny=61, land=0.3)
    g = gridgen.make_grid(seed=gridgen.seed_for(7), **cfg)
    h = pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A2, drop_tol=0.05)
    tx, ty = pcg.pcg_autotune(h, 1, objective=1)
    assert tx in (64, 124, 128) and ty in (8, 16, 32, 64)
    assert pcg.pcg_tiles(h, 1) == (tx, ty)
    _check_solve(pcg, h, g, 1)
    with pytest.raises(pcg.PCGError) as e:
        pcg.pcg_autotune(h, 1, objective=2)
    assert e.value.status == pcg.PCG_EINVAL


def test_autotune_fp64_trilA_offers_both_whole_warp_widths():
    """binary64 tril(A) has two whole-warp strips (62 and 124 columns) besides
    64 and 128; the tuned one is among them and solves correctly."""
    import paper_1210_1878_b300 as pcg
    cfg = dict(nx=260, ny=53, land=0.3)
    g = gridgen.make_grid(seed=gridgen.seed_for(8), **cfg)
    h = pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A)
    assert pcg.pcg_tiles(h, 0)[0] == 62            # narrow grid: the 62-column strip by default
    tx, ty = pcg.pcg_autotune(h, 0)
    assert tx in (62, 64, 124, 128) and ty in (8, 16, 32, 64)
    assert pcg.pcg_tiles(h, 0) == (tx, ty)
    _check_solve(pcg, h, g, 0)
