"""GPU parity of the CUDA path against the FP64 CPU oracle, through the C ABI.

Element by element on seeded grids that span several strips and a ragged
last strip; tolerances follow from binary64 rounding of the stated
operations (Section 3, Eq. 9 for A; the preconditioning step of Algorithm 1 for M^-1 = Z D^-1 Z^T;
Algorithm 1 for the solve, whose result is judged by the residual and by the
distance to a tight reference solution)."""
import numpy as np
import pytest
import scipy.sparse as sp

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


GRIDS = [
    ("tiny", dict(gridgen.TINY), 0),
    ("coarse", dict(gridgen.COARSE), 1),
    ("ragged", dict(nx=203, ny=77, land=0.3), 7),       # last strip partial in i and j
    ("row", dict(nx=150, ny=1, land=0.1), 8),            # one latitude row
    ("channel", dict(nx=6, ny=40, land=0.0), 9),         # narrow periodic channel
]


def _grid(spec):
    name, cfg, seed = spec
    return gridgen.make_grid(seed=gridgen.seed_for(0) + 100 * seed, **cfg)


def _csr(P):
    rp, col, val, _, _ = P.csr()
    return sp.csr_matrix((val, col, rp), shape=(P.n, P.n))


@pytest.mark.parametrize("spec", GRIDS, ids=[g[0] for g in GRIDS])
@pytest.mark.parametrize("tiles", [(0, 0), (64, 8), (128, 32), (62, 16), (124, 16)])
def test_spmv_matches_oracle(spec, tiles):
    pcg = _pcg()
    g = _grid(spec)
    P = oracle.OracleProblem.from_grid(g)
    h = pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A, tile_x=tiles[0], tile_y=tiles[1])
    rng = np.random.default_rng(11)
    v = rng.standard_normal((g.ny, g.nx))
    q = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
    pcg.pcg_spmv(h, _dev(v), q)
    qo = P.to_grid(P.spmv(P.to_wet(v)))
    mag = P.to_grid(abs(_csr(P)) @ np.abs(P.to_wet(v)))
    err = np.abs(q.cpu().numpy() - qo)
    assert np.all(err <= 1e-13 * mag + 1e-300)
    assert np.all(q.cpu().numpy()[g.wet == 0] == 0)


PRECONDS = [(0, 0.0, 0), (1, 0.0, 0), (1, 0.05, 0), (4, 0.0, 0), (3, 0.0, 1), (3, 0.0, 4), (3, 0.0, 8)]


@pytest.mark.parametrize("spec", GRIDS, ids=[g[0] for g in GRIDS])
@pytest.mark.parametrize("pattern,tau,q", PRECONDS)
@pytest.mark.parametrize("tile_x", [0, 64, 124, 92])
def test_precond_matches_oracle(spec, pattern, tau, q, tile_x):
    """tile_x 0: the default strips (60/62 columns for tril(A^2)/tril(A), whose
    t phase fills whole warps); 64: strips with a halo pass; 124 and 92: the wide
    binary64 strips of tril(A) and tril(A^2)."""
    pcg = _pcg()
    g = _grid(spec)
    if tile_x == 124 and pattern != pcg.PCG_PAT_TRIL_A:
        pytest.skip("124-column binary64 strips exist for tril(A) only")
    if tile_x == 92 and pattern != pcg.PCG_PAT_TRIL_A2:
        pytest.skip("92-column binary64 strips exist for tril(A^2) only")
    if pattern == 3 and q >= g.nx:
        pytest.skip("band wider than the row")
    P = oracle.OracleProblem.from_grid(g)
    assert P.ainv(pattern, tau, q) == oracle.OK
    h = pcg.ainv_setup_grid(g, pattern=pattern, drop_tol=tau, band_q=q, tile_x=tile_x)
    rng = np.random.default_rng(12)
    r = rng.standard_normal((g.ny, g.nx))
    s = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
    pcg.pcg_precond_apply(h, _dev(r), s)
    so = P.to_grid(P.apply(P.to_wet(r)))
    cp, row, val, d = P.z()
    Z = sp.csc_matrix((np.abs(val), row, cp), shape=(P.n, P.n))
    mag = P.to_grid(Z @ ((Z.T @ np.abs(P.to_wet(r))) / d))
    err = np.abs(s.cpu().numpy() - so)
    assert np.all(err <= 1e-13 * mag + 1e-300), float((err / (mag + 1e-300)).max())


SOLVES = [
    ("tiny-trilA", dict(gridgen.TINY), 0, 0, 0.0, 0, 0),
    ("tiny-trilA2", dict(gridgen.TINY), 0, 1, 0.0, 0, 0),
    ("tiny-trilA2-drop", dict(gridgen.TINY), 0, 1, 0.05, 0, 0),
    ("coarse-trilA2", dict(gridgen.COARSE), 1, 1, 0.05, 0, 0),
    ("coarse-jacobi", dict(gridgen.COARSE), 1, 4, 0.0, 0, 0),
    ("coarse-bandT4", dict(gridgen.COARSE), 1, 3, 0.0, 4, 0),
    ("ragged-trilA", dict(nx=203, ny=77, land=0.3), 7, 0, 0.0, 0, 0),
    ("ragged-trilA2", dict(nx=203, ny=77, land=0.3), 7, 1, 0.05, 0, 0),
    ("ragged-trilA-wide", dict(nx=203, ny=77, land=0.3), 7, 0, 0.0, 0, 124),   # 124-column strips
    ("ragged-trilA2-wide", dict(nx=203, ny=77, land=0.3), 7, 1, 0.05, 0, 92),   # 92-column strips
    ("orca1-trilA2", dict(gridgen.ORCA1), 3, 1, 0.05, 0, 0),
    ("orca025-trilA2", dict(gridgen.ORCA025), 2, 1, 0.05, 0, 0),
]


@pytest.mark.parametrize("name,cfg,ci,pattern,tau,q,tile_x", SOLVES, ids=[s[0] for s in SOLVES])
def test_solve_matches_oracle(name, cfg, ci, pattern, tau, q, tile_x):
    pcg = _pcg()
    g = gridgen.make_grid(seed=gridgen.seed_for(ci), **cfg)
    P = oracle.OracleProblem.from_grid(g)
    assert P.ainv(pattern, tau, q) == oracle.OK
    b = P.to_wet(g.b)
    ref = P.pcg(b, rtol=1e-10)
    assert ref.status == oracle.OK
    h = pcg.ainv_setup_grid(g, pattern=pattern, drop_tol=tau, band_q=q, tile_x=tile_x, tile_y=8 if tile_x else 0)
    if tile_x:
        assert pcg.pcg_tiles(h) == (tile_x, 8)
    x = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
    st = pcg.pcg_solve(h, _dev(g.b), x, pcg.make_opts(rtol=1e-10))
    assert st.status == pcg.PCG_OK
    assert abs(st.iters - ref.iters) <= 2, (st.iters, ref.iters)
    judge(P, g, b, x.cpu().numpy(), rtol=1e-10, stats=st)


def test_batched_matches_oracle_and_alone():
    """Every member of a batch meets the oracle's acceptance (true residual
    recomputed by the oracle, distance to the tight reference), and equals the
    same solve run alone, bit for bit (same kernels, same per-grid reduction
    order)."""
    pcg = _pcg()
    specs = [(dict(gridgen.COARSE), 1), (dict(nx=203, ny=77, land=0.3), 7), (dict(gridgen.TINY), 0),
             (dict(gridgen.ORCA1), 3)]
    grids = [gridgen.make_grid(seed=gridgen.seed_for(ci), **cfg) for cfg, ci in specs]
    hs = [pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A2, drop_tol=0.05) for g in grids]
    alone = []
    for h, g in zip(hs, grids):
        x = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
        st = pcg.pcg_solve(h, _dev(g.b), x)
        alone.append((x.cpu().numpy(), st.iters))
    xs = [torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda") for g in grids]
    rc, stats = pcg.pcg_solve_batched(hs, [_dev(g.b) for g in grids], xs)
    assert rc == pcg.PCG_OK
    for (xa, ia), xb, st, g in zip(alone, xs, stats, grids):
        assert st.status == pcg.PCG_OK and st.iters == ia
        xbn = xb.cpu().numpy()
        np.testing.assert_array_equal(xbn, xa)
        P = oracle.OracleProblem.from_grid(g)
        assert P.ainv(oracle.PAT_TRIL_A2, 0.05) == oracle.OK
        b = P.to_wet(g.b)
        ref = P.pcg(b, rtol=1e-10)
        assert abs(st.iters - ref.iters) <= 2, (st.iters, ref.iters)
        judge(P, g, b, xbn, rtol=1e-10, stats=st)


def test_true_residual_restart_path():
    """The stop-and-verify step (the loop condition of Algorithm 1 plus the
    true-residual check on exit): near the attainable accuracy the recursive
    residual runs ahead of the true one, the check fails and the solve restarts
    from the true residual. (a) An unreachable tolerance: both the oracle and
    the GPU restart max_replace times and report ENOTCONV, and the GPU's final
    true residual (recomputed by the oracle) is as small as the oracle's own.
    (b) Tolerances at which the oracle needs a restart and then succeeds: the
    GPU meets the tolerance (by the oracle's residual), and at least one of them
    took the restart path on the GPU too."""
    pcg = _pcg()
    g = gridgen.make_grid(seed=gridgen.seed_for(1), **gridgen.COARSE)
    P = oracle.OracleProblem.from_grid(g)
    assert P.ainv(oracle.PAT_TRIL_A2, 0.05) == oracle.OK
    b = P.to_wet(g.b)
    h = pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A2, drop_tol=0.05)
    x = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
    ref = P.pcg(b, rtol=5e-16, max_iter=5000, max_replace=3)
    assert ref.status == oracle.ENOTCONV and ref.replacements == 3
    st = pcg.pcg_solve(h, _dev(g.b), x, pcg.make_opts(rtol=5e-16, max_iter=5000, max_replace=3), check=False)
    assert st.status == pcg.PCG_ENOTCONV and st.replacements == 3 and st.outer_iters == 4, st.as_dict()
    rp, col, val, _, _ = P.csr()
    A_abs = sp.csr_matrix((np.abs(val), col, rp), shape=(P.n, P.n))

    def residual_and_floor():
        # at this level both sides' residuals are rounding: each entry of
        # b - A x carries at most gamma_6 (|b| + |A||x|) of binary64 error
        xw = P.to_wet(x.cpu().numpy())
        rel = float(np.linalg.norm(b - P.spmv(xw)) / np.linalg.norm(b))
        floor = 2 * 6 * 2.0 ** -53 * np.linalg.norm(np.abs(b) + A_abs @ np.abs(xw)) / np.linalg.norm(b)
        return rel, floor

    rel, floor = residual_and_floor()
    assert rel <= 4 * ref.true_relres and rel <= 3e-15, (rel, ref.true_relres)
    assert abs(st.true_relres - rel) <= floor, (st.true_relres, rel, floor)
    restarted = 0
    for rtol in (5e-15, 3e-15, 2e-15, 1e-15):
        ref = P.pcg(b, rtol=rtol, max_iter=5000, max_replace=3)
        if not (ref.status == oracle.OK and ref.replacements >= 1):
            continue
        st = pcg.pcg_solve(h, _dev(g.b), x, pcg.make_opts(rtol=rtol, max_iter=5000, max_replace=3), check=False)
        assert st.status == pcg.PCG_OK, (rtol, st.as_dict())
        rel, floor = residual_and_floor()
        # the device accepted on its own true residual, within rounding of the oracle's
        assert st.true_relres <= rtol and rel <= rtol + floor, (rtol, st.true_relres, rel, floor)
        assert abs(st.replacements - ref.replacements) <= 1, (rtol, st.replacements, ref.replacements)
        restarted += st.replacements >= 1
    assert restarted >= 1


def test_host_buffers_and_warm_start():
    pcg = _pcg()
    g = gridgen.make_grid(seed=gridgen.seed_for(1), **gridgen.COARSE)
    h = pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A2, drop_tol=0.05)
    x_host = np.zeros((g.ny, g.nx))
    st = pcg.pcg_solve(h, np.ascontiguousarray(g.b), x_host)
    x_dev = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
    st2 = pcg.pcg_solve(h, _dev(g.b), x_dev)
    np.testing.assert_array_equal(x_host, x_dev.cpu().numpy())
    assert st.iters == st2.iters
    # warm start from the solution: converged before the first iteration
    st3 = pcg.pcg_solve(h, _dev(g.b), x_dev, pcg.make_opts(use_x0=True))
    assert st3.status == pcg.PCG_OK and st3.iters == 0


def test_degenerate_cases():
    pcg = _pcg()
    g = gridgen.make_grid(seed=gridgen.seed_for(1), **gridgen.COARSE)
    h = pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A)
    x = torch.full((g.ny, g.nx), 7.0, dtype=torch.float64, device="cuda")
    st = pcg.pcg_solve(h, torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda"), x)
    assert st.status == pcg.PCG_OK and st.iters == 0 and float(x.abs().max()) == 0.0
    st = pcg.pcg_solve(h, _dev(g.b), x, pcg.make_opts(rtol=1e-14, max_iter=5, max_replace=0), check=False)
    assert st.status == pcg.PCG_ENOTCONV and st.iters == 5
    # a single wet cell: A = shift, one step
    wet = np.zeros((9, 12), np.uint8)
    wet[4, 11] = 1
    sh = np.where(wet > 0, 3.0, 0.0)
    h1 = pcg.ainv_setup(12, 9, wet, np.ones((9, 12)), np.ones((9, 12)), sh, pattern=pcg.PCG_PAT_TRIL_A2)
    b = np.zeros((9, 12))
    b[4, 11] = 6.0
    x1 = torch.zeros((9, 12), dtype=torch.float64, device="cuda")
    st = pcg.pcg_solve(h1, _dev(b), x1)
    assert st.status == pcg.PCG_OK and float(x1[4, 11]) == pytest.approx(2.0, rel=1e-15)
    # all land
    h0 = pcg.ainv_setup(12, 9, np.zeros((9, 12), np.uint8), np.ones((9, 12)), np.ones((9, 12)), np.ones((9, 12)),
                        pattern=pcg.PCG_PAT_TRIL_A)
    st = pcg.pcg_solve(h0, _dev(np.ones((9, 12))), x1)
    assert st.status == pcg.PCG_OK and float(x1.abs().max()) == 0.0


def test_bounded_wait_reports_timeout():
    """A device wait that can never complete gives up after its limit and the
    kernel returns PCG_ETIMEOUT through the grid state; the handle keeps working."""
    pcg = _pcg()
    g = gridgen.make_grid(seed=gridgen.seed_for(1), **gridgen.COARSE)
    h = pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A2)
    assert pcg.pcg_debug_wait_timeout(h, unit=1, timeout_ms=20.0) == pcg.PCG_ETIMEOUT
    x = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
    st = pcg.pcg_solve(h, _dev(g.b), x)
    assert st.status == pcg.PCG_OK and st.true_relres <= 1e-10


def test_strip_counts_beyond_16_bits_are_refused():
    """Strip coordinates are 16-bit: a grid 140000 rows tall cannot take 4-row
    strips (35000 of them); the default height keeps the count in range and the
    solve still passes the acceptance test."""
    pcg = _pcg()
    g = gridgen.make_grid(seed=gridgen.seed_for(0) + 900, nx=5, ny=140000, land=0.2)
    with pytest.raises(pcg.PCGError) as e:
        pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A, tile_y=4)
    assert e.value.status == pcg.PCG_EINVAL
    h = pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A)
    assert (g.ny + pcg.pcg_tiles(h)[1] - 1) // pcg.pcg_tiles(h)[1] <= 32767
    P = oracle.OracleProblem.from_grid(g)
    x = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
    st = pcg.pcg_solve(h, _dev(g.b), x, pcg.make_opts(rtol=1e-10, max_iter=5000))
    assert st.status == pcg.PCG_OK
    bw = P.to_wet(g.b)
    assert np.linalg.norm(bw - P.spmv(P.to_wet(x.cpu().numpy()))) / np.linalg.norm(bw) <= 1e-10 * (1 + 1e-3)


def test_async_solves_on_two_streams():
    """The solve entry points enqueue the whole solve and return: two solves on
    two streams (one binary64 restart-checked solve, one mixed-precision solve)
    are issued back to back with no synchronisation in between, then pcg_sync
    makes each result and its statistics valid; both meet the oracle's
    acceptance. The first call returns while its solve is still running on the
    device (the stopping test, the true-residual check and any restart are
    decided there)."""
    pcg = _pcg()
    g1 = gridgen.make_grid(seed=gridgen.seed_for(2), **gridgen.ORCA025)
    g2 = gridgen.make_grid(seed=gridgen.seed_for(1), **gridgen.COARSE)
    h1 = pcg.ainv_setup_grid(g1, pattern=pcg.PCG_PAT_TRIL_A2, drop_tol=0.05)
    h2 = pcg.ainv_setup_grid(g2, pattern=pcg.PCG_PAT_TRIL_A)
    o1 = pcg.make_opts(rtol=1e-10)
    o2 = pcg.make_opts(rtol=1e-10, prec=pcg.PCG_MIXED)
    b1, b2 = _dev(g1.b), _dev(g2.b)
    x1 = torch.zeros_like(b1)
    x2 = torch.zeros_like(b2)
    # first use builds the plans and graphs; the timed behaviour is the second
    pcg.pcg_solve(h1, b1, x1, o1)
    pcg.pcg_solve(h2, b2, x2, o2)
    x1.zero_()
    x2.zero_()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    st1 = pcg.pcg_solve(h1, b1, x1, o1, stream=s1, sync=False)
    running = not s1.query()
    st2 = pcg.pcg_solve(h2, b2, x2, o2, stream=s2, sync=False)
    assert st1.rc == pcg.PCG_OK and st2.rc == pcg.PCG_OK
    assert running, "pcg_solve waited for its solve"
    assert pcg.pcg_sync(h2) == pcg.PCG_OK
    assert pcg.pcg_sync(h1) == pcg.PCG_OK
    assert pcg.pcg_sync(h1) == pcg.PCG_OK          # nothing in flight: the last status again
    assert st1.status == pcg.PCG_OK and st1.iters > 0 and st2.status == pcg.PCG_OK and st2.outer_iters >= 1
    for g, x, st in ((g1, x1, st1), (g2, x2, st2)):
        P = oracle.OracleProblem.from_grid(g)
        judge(P, g, P.to_wet(g.b), x.cpu().numpy(), rtol=1e-10, stats=st)
