"""GPU parity of the binary32 kernels (the inner iterations of the mixed
precision mode) against the binary64 CPU oracle, element by element, through
the C ABI (pcg_apply_f32).

Tolerance from binary32 rounding (u = 2^-24), to first order in u:
  q = A v (Section 3, Eq. 9): v and the coefficients are rounded once each and
  the 5-term FMA chain adds at most 5 roundings: |q32 - q| <= 7u (|A| |v|).
  s = Z D^-1 Z^T r (the preconditioning step of Algorithm 1): r, Z, D^-1
  rounded, k_t + 1 roundings in t = D^-1 Z^T r and k_s in s = Z t (k_t, k_s
  <= 9 terms for the patterns here): |s32 - s| <= (k_t + k_s + 5)u
  (|Z| |D^-1| |Z|^T |r|) <= 23u (...).
Both tests use 32u."""
import numpy as np
import pytest
import scipy.sparse as sp

import gridgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

U32 = 2.0 ** -24
TOL = 32 * U32

GRIDS = [
    ("tiny", dict(gridgen.TINY), 0),
    ("coarse", dict(gridgen.COARSE), 1),
    ("ragged", dict(nx=203, ny=77, land=0.3), 7),       # last strip partial in i and j
    ("row", dict(nx=150, ny=1, land=0.1), 8),            # one latitude row
    ("channel", dict(nx=6, ny=40, land=0.0), 9),         # narrow periodic channel
    ("orca1", dict(gridgen.ORCA1), 3),                   # several strips and row groups
]


def _grid(spec):
    name, cfg, seed = spec
    return gridgen.make_grid(seed=gridgen.seed_for(0) + 100 * seed, **cfg)


def _csr(P):
    rp, col, val, _, _ = P.csr()
    return sp.csr_matrix((val, col, rp), shape=(P.n, P.n))


@pytest.mark.parametrize("spec", GRIDS, ids=[g[0] for g in GRIDS])
@pytest.mark.parametrize("tiles", [(0, 0), (64, 8), (128, 32), (0, 4)])
def test_spmv_f32_matches_oracle(spec, tiles):
    import paper_1210_1878_b300 as pcg
    g = _grid(spec)
    P = oracle.OracleProblem.from_grid(g)
    h = pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A, tile_x=tiles[0], tile_y=tiles[1])
    rng = np.random.default_rng(21)
    v = rng.standard_normal((g.ny, g.nx))
    q = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
    pcg.pcg_apply_f32(h, 0, torch.from_numpy(v).cuda(), q)
    qo = P.to_grid(P.spmv(P.to_wet(v)))
    mag = P.to_grid(abs(_csr(P)) @ np.abs(P.to_wet(v)))
    qg = q.cpu().numpy()
    err = np.abs(qg - qo)
    assert np.all(err <= TOL * mag + 1e-300), float((err / (mag + 1e-300)).max())
    assert np.all(qg[g.wet == 0] == 0)
    # the binary32 result is not the binary64 one: the test does see rounding
    assert np.any(err > 0)


PRECONDS = [(0, 0.0, 0), (1, 0.0, 0), (1, 0.05, 0), (4, 0.0, 0), (3, 0.0, 1), (3, 0.0, 4), (3, 0.0, 8)]


@pytest.mark.parametrize("spec", GRIDS, ids=[g[0] for g in GRIDS])
@pytest.mark.parametrize("pattern,tau,q", PRECONDS)
@pytest.mark.parametrize("ty", [0, 4])
def test_precond_f32_matches_oracle(spec, pattern, tau, q, ty):
    import paper_1210_1878_b300 as pcg
    g = _grid(spec)
    if pattern == 3 and q >= g.nx:
        pytest.skip("band wider than the row")
    P = oracle.OracleProblem.from_grid(g)
    assert P.ainv(pattern, tau, q) == oracle.OK
    h = pcg.ainv_setup_grid(g, pattern=pattern, drop_tol=tau, band_q=q, tile_y=ty)
    rng = np.random.default_rng(22)
    r = rng.standard_normal((g.ny, g.nx))
    s = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
    pcg.pcg_apply_f32(h, 1, torch.from_numpy(r).cuda(), s)
    so = P.to_grid(P.apply(P.to_wet(r)))
    cp, row, val, d = P.z()
    Z = sp.csc_matrix((np.abs(val), row, cp), shape=(P.n, P.n))
    mag = P.to_grid(Z @ ((Z.T @ np.abs(P.to_wet(r))) / d))
    sg = s.cpu().numpy()
    err = np.abs(sg - so)
    assert np.all(err <= TOL * mag + 1e-300), float((err / (mag + 1e-300)).max())
    assert np.all(sg[g.wet == 0] == 0)


def test_apply_f32_rejects_bad_op():
    import paper_1210_1878_b300 as pcg
    g = _grid(GRIDS[0])
    h = pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A)
    v = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
    with pytest.raises(pcg.PCGError) as e:
        pcg.pcg_apply_f32(h, 2, v, v)
    assert e.value.status == pcg.PCG_EINVAL


def test_explicit_width_applies_to_the_precisions_that_have_it():
    """tile_x = 124 with tril(A^2): binary32 kernels exist for it, binary64 ones
    do not (binary64 keeps its default 60-column strips); both paths solve."""
    import paper_1210_1878_b300 as pcg
    g = _grid(GRIDS[2])
    P = oracle.OracleProblem.from_grid(g)
    h = pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A2, drop_tol=0.05, tile_x=124, tile_y=16)
    assert pcg.pcg_tiles(h, 0) == (60, 16)
    for prec in (0, 1):
        x = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
        st = pcg.pcg_solve(h, torch.from_numpy(g.b).cuda(), x, pcg.make_opts(rtol=1e-10, prec=prec))
        assert st.status == pcg.PCG_OK
        bw = P.to_wet(g.b)
        assert np.linalg.norm(bw - P.spmv(P.to_wet(x.cpu().numpy()))) / np.linalg.norm(bw) <= 1e-10 * (1 + 1e-3)
    assert pcg.pcg_tiles(h, 1) == (124, 16)
    with pytest.raises(pcg.PCGError) as e:
        pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A2, tile_x=100)
    assert e.value.status == pcg.PCG_EINVAL
