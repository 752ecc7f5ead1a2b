"""The library builds its factor by LEFT-looking conjugate orthogonalisation
(an independent implementation); the oracle builds it right-looking. Both
apply the same updates to each column in the same order (Section 3: pattern
and drop after every update), so Z and D must agree entry by entry."""
import numpy as np
import pytest

import gridgen
import oracle


CASES = [
    ("tiny", gridgen.TINY, 0),
    ("coarse", gridgen.COARSE, 1),
]
PATTERNS = [
    (0, 0.0, 0), (1, 0.0, 0), (1, 0.05, 0), (1, 0.3, 0), (3, 0.0, 1), (3, 0.0, 4), (3, 0.0, 8), (4, 0.0, 0),
]


def _oracle_entries(P):
    cp, row, val, d = P.z()
    ent = {}
    for j in range(P.n):
        for t in range(cp[j], cp[j + 1]):
            if row[t] != j and val[t] != 0.0:
                ent[(int(row[t]), j)] = float(val[t])
    return ent, d


@pytest.mark.parametrize("name,cfg,ci", CASES)
@pytest.mark.parametrize("pattern,tau,q", PATTERNS)
def test_factor_matches_oracle(name, cfg, ci, pattern, tau, q):
    import paper_1210_1878_b300 as pcg
    g = gridgen.make_grid(seed=gridgen.seed_for(ci), **cfg)
    P = oracle.OracleProblem.from_grid(g)
    assert P.ainv(pattern, tau, q) == oracle.OK
    ent_o, d_o = _oracle_entries(P)
    D, rows, vals = pcg.ainv_factor_host(g.nx, g.ny, g.wet, g.c_e, g.c_n, g.shift, pattern=pattern,
                                         drop_tol=tau, band_q=q)
    np.testing.assert_allclose(D, d_o, rtol=1e-14, atol=0)
    ent_l = {}
    for k in range(len(D)):
        for e in range(8):
            if rows[k, e] >= 0:
                ent_l[(int(rows[k, e]), k)] = float(vals[k, e])
    assert set(ent_l) == set(ent_o)
    for key, v in ent_o.items():
        assert ent_l[key] == pytest.approx(v, rel=1e-14, abs=0)


def test_factor_on_wrap_heavy_grid():
    """A narrow periodic channel (nx = 6, all wet rows) exercises every periodic
    side-table entry of tril(A^2)."""
    import paper_1210_1878_b300 as pcg
    g = gridgen.make_grid(nx=6, ny=7, seed=5, land=0.0)
    for pattern, tau in ((0, 0.0), (1, 0.0)):
        P = oracle.OracleProblem.from_grid(g)
        assert P.ainv(pattern, tau) == oracle.OK
        ent_o, d_o = _oracle_entries(P)
        D, rows, vals = pcg.ainv_factor_host(g.nx, g.ny, g.wet, g.c_e, g.c_n, g.shift, pattern=pattern)
        np.testing.assert_allclose(D, d_o, rtol=1e-14)
        ent_l = {(int(rows[k, e]), k): float(vals[k, e]) for k in range(len(D)) for e in range(8) if rows[k, e] >= 0}
        assert set(ent_l) == set(ent_o)
        for key, v in ent_o.items():
            assert ent_l[key] == pytest.approx(v, rel=1e-14)
