"""Acceptance of a GPU solve, judged by the FP64 CPU oracle alone.

A solve of Algorithm 1 has many correct results (any x whose relative residual
meets rtol), so a returned x is judged by two numbers the oracle computes from
it: the true relative residual ||b - A x|| / ||b|| (A assembled by the oracle,
Section 3, Eq. 9 in SPD form), and its distance to a tight reference solution
x_ref of A x = b (a dense solve up to 2000 unknowns, otherwise the oracle's own
PCG run to 1e-13). Nothing here reads a value the CUDA path produced except
the x being judged.
"""
import numpy as np

import oracle

DENSE_MAX = 2000
SOLUTION_TOL = 1e-8


def tight_reference(P, b, pattern=oracle.PAT_TRIL_A2, tau=0.05):
    """x_ref with A x_ref = b: a dense solve for small systems,
    otherwise oracle PCG at rtol 1e-13 (its preconditioner is rebuilt with the
    given pattern; x_ref does not depend on the preconditioner)."""
    if P.n <= DENSE_MAX:
        return np.linalg.solve(P.dense(), b)
    assert P.ainv(pattern, tau) == oracle.OK
    res = P.pcg(b, rtol=1e-13, max_iter=20 * P.n)
    assert res.status in (oracle.OK, oracle.ENOTCONV)
    return res.x


def true_relres(P, b, xw):
    """||b - A x|| / ||b|| in binary64, from the oracle's operator."""
    return float(np.linalg.norm(b - P.spmv(xw)) / np.linalg.norm(b))


def judge(P, g, b, x_grid, rtol=1e-10, x_ref=None, stats=None):
    """Assert that x_grid ([ny][nx], land zero) meets the acceptance: true
    residual (by the oracle) <= rtol, within 1e-8 of the tight reference, and
    the device-reported true residual (if given) agrees with the oracle's.
    Returns (true relative residual, relative solution error)."""
    x_grid = np.asarray(x_grid)
    assert np.all(x_grid[g.wet == 0] == 0)
    xw = P.to_wet(x_grid)
    rel = true_relres(P, b, xw)
    assert rel <= rtol * (1 + 1e-3), rel
    if x_ref is None:
        x_ref = tight_reference(P, b)
    err = float(np.linalg.norm(xw - x_ref) / np.linalg.norm(x_ref))
    assert err <= SOLUTION_TOL, err
    if stats is not None:
        assert abs(stats.true_relres - rel) <= 1e-3 * rtol + 1e-3 * rel, (stats.true_relres, rel)
    return rel, err
