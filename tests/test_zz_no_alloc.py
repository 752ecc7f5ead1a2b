"""The allocation-free operator apply (pcg_spmv_noalloc) gives the same q = A v
as pcg_spmv. It serves callers that cannot allocate device memory at the point
of the call (their own memory manager owns the device, or an allocation there
would break a capture or a budget), so its scratch is a fixed device array
that every call reuses: two calls in a row on different grids must each match
the allocating entry point. Grids beyond the array's limit are refused."""
import numpy as np
import pytest

import gridgen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _spmv_both(pcg, h, g, seed):
    rng = np.random.default_rng(seed)
    v = torch.from_numpy(rng.standard_normal((g.ny, g.nx))).cuda()
    q_ref = torch.zeros_like(v)
    pcg.pcg_spmv(h, v, q_ref)
    q = torch.full_like(v, float("nan"))
    assert pcg.pcg_spmv_noalloc(h, v, q) == pcg.PCG_OK
    return q.cpu().numpy(), q_ref.cpu().numpy()


def test_noalloc_spmv_matches_spmv_twice():
    import paper_1210_1878_b300 as pcg
    g1 = gridgen.make_grid(seed=gridgen.seed_for(1), **gridgen.COARSE)
    g2 = gridgen.make_grid(nx=203, ny=77, seed=gridgen.seed_for(0) + 700, land=0.3)
    h1 = pcg.ainv_setup_grid(g1, pattern=pcg.PCG_PAT_TRIL_A2, drop_tol=0.05)
    h2 = pcg.ainv_setup_grid(g2, pattern=pcg.PCG_PAT_TRIL_A)
    for h, g, seed in ((h1, g1, 1), (h2, g2, 2), (h1, g1, 3)):
        q, q_ref = _spmv_both(pcg, h, g, seed)
        scale = np.abs(q_ref).max()
        np.testing.assert_allclose(q, q_ref, rtol=0, atol=1e-13 * scale)
        assert np.all(q[g.wet == 0] == 0)


def test_noalloc_refuses_grids_beyond_its_scratch():
    import paper_1210_1878_b300 as pcg
    g = gridgen.make_grid(nx=2100, ny=1050, seed=gridgen.seed_for(0) + 701, land=0.95)
    h = pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_DIAG)
    v = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
    q = torch.zeros_like(v)
    assert pcg.pcg_spmv_noalloc(h, v, q) == pcg.PCG_EINVAL
    assert b"limit" in pcg.lib.pcg_last_error_message()
