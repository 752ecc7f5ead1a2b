"""Second handles of one grid (pcg_clone), and solves with host buffers kept in
flight on two handles at once.

A clone holds the same A, Z, D^-1 and strips as its source, so the same solve
(Algorithm 1) on either gives the same iterates, bit for bit, and the clone
keeps working after its source is freed. Solves alternating between a handle
and its clone with pinned host buffers, each synchronised only when its
handle is used again, give exactly the results of the same solves done one at
a time, and those results meet the oracle's acceptance (true residual at most
rtol, x within 1e-8 of the oracle's tight solution in binary64)."""
import numpy as np
import pytest

import gridgen
import oracle
from oracle_checks import judge

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _pcg():
    import paper_1210_1878_b300 as pcg
    return pcg


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_clone_solves_like_its_source(prec):
    pcg = _pcg()
    g = gridgen.make_grid(seed=gridgen.seed_for(3), **gridgen.ORCA1)
    h = pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A2, drop_tol=0.05)
    c = pcg.pcg_clone(h)
    assert c.n_wet == h.n_wet and c.resident_bytes == h.resident_bytes
    assert pcg.pcg_tiles(c, prec) == pcg.pcg_tiles(h, prec)
    o = pcg.make_opts(rtol=1e-10, prec=prec)
    b = _dev(g.b)
    x1 = torch.zeros_like(b)
    x2 = torch.zeros_like(b)
    s1 = pcg.pcg_solve(h, b, x1, o)
    s2 = pcg.pcg_solve(c, b, x2, o)
    assert (s1.iters, s1.outer_iters) == (s2.iters, s2.outer_iters)
    assert torch.equal(x1, x2)
    h.close()                                   # the clone owns its device memory
    x3 = torch.zeros_like(b)
    s3 = pcg.pcg_solve(c, b, x3, o)
    assert torch.equal(x3, x1)
    P = oracle.OracleProblem.from_grid(g)
    judge(P, g, P.to_wet(g.b), x3.cpu().numpy(), rtol=1e-10, stats=s3)
    c.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_pipelined_host_solves_on_two_handles(prec):
    pcg = _pcg()
    g = gridgen.make_grid(seed=gridgen.seed_for(2), **gridgen.ORCA025)
    h = pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A2, drop_tol=0.05)
    c = pcg.pcg_clone(h)
    o = pcg.make_opts(rtol=1e-10, prec=prec)
    wet = g.wet.astype(bool)
    rhs = []
    for k in range(6):
        rng = np.random.default_rng(100 + k)
        rhs.append(np.where(wet, g.b + 0.1 * np.abs(g.b).max() * rng.standard_normal(g.b.shape), 0.0))
    # the same solves one at a time, on device buffers
    ref = []
    for bk in rhs:
        x = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
        assert pcg.pcg_solve(h, _dev(bk), x, o).status == pcg.PCG_OK
        ref.append(x.cpu().numpy())
    bh = [torch.from_numpy(bk.copy()).pin_memory() for bk in rhs]
    xh = [torch.zeros((g.ny, g.nx), dtype=torch.float64).pin_memory() for _ in rhs]
    handles = [h, c]
    torch.cuda.synchronize()
    stats = [pcg.pcg_solve(handles[k % 2], bh[k], xh[k], o, sync=False) for k in range(len(rhs))]
    for hh in handles:
        assert pcg.pcg_sync(hh) == pcg.PCG_OK
    for k in range(len(rhs)):
        assert stats[k].status == pcg.PCG_OK and stats[k].iters > 0, k
        np.testing.assert_array_equal(xh[k].numpy(), ref[k])
    P = oracle.OracleProblem.from_grid(g)
    for k in (0, len(rhs) - 1):
        judge(P, g, P.to_wet(rhs[k]), xh[k].numpy(), rtol=1e-10, stats=stats[k])
    h.close()
    c.close()
