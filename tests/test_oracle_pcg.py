"""Pins of the oracle's PCG (Algorithm 1 with d = s + beta d, true-residual
check on exit) against a dense solve, the convergence bound of Section 3
Eq. 10, exact special cases and an exact scaling symmetry; plus the paper's
qualitative Table 2 result (the AINV preconditioner needs fewer iterations
than the diagonal one)."""
import math

import numpy as np
import pytest

import gridgen
import oracle


def _tiny():
    g = gridgen.make_grid(seed=gridgen.seed_for(0), **gridgen.TINY)
    P = oracle.OracleProblem.from_grid(g)
    return g, P, P.to_wet(g.b)


@pytest.mark.parametrize("pattern,tau", [(oracle.PAT_TRIL_A, 0.0), (oracle.PAT_TRIL_A2, 0.05),
                                         (oracle.PAT_DIAG, 0.0), (oracle.PAT_BAND_T, 0.0)])
def test_matches_dense_solve(pattern, tau):
    g, P, b = _tiny()
    assert P.ainv(pattern, tau, 4) == oracle.OK
    res = P.pcg(b, rtol=1e-13, hist=True)
    assert res.status == oracle.OK and res.true_relres <= 1e-13
    x_ref = np.linalg.solve(P.dense(), b)
    assert np.linalg.norm(res.x - x_ref) / np.linalg.norm(x_ref) < 1e-12
    # the recursive residual history is what the stopping test saw
    assert res.res[-1] <= 1e-13 and np.all(res.res[:-1] > 1e-13)


def test_convergence_bound_eq10():
    """||x - x_m||_A < 2 ((sqrt(mu)-1)/(sqrt(mu)+1))^(m-1) ||x - x_0||_A with mu the
    condition number of the preconditioned operator (Section 3, Eq. 10)."""
    g, P, b = _tiny()
    assert P.ainv(oracle.PAT_TRIL_A) == oracle.OK
    A = P.dense()
    Z, d = P.z_dense()
    Lm = Z @ np.diag(1 / np.sqrt(d))                  # M^-1 = Lm Lm^T
    ev = np.linalg.eigvalsh(Lm.T @ A @ Lm)
    mu = ev[-1] / ev[0]
    x = np.linalg.solve(A, b)
    anorm = lambda e: math.sqrt(e @ A @ e)
    e0 = anorm(x)
    rate = (math.sqrt(mu) - 1) / (math.sqrt(mu) + 1)
    for m in (1, 5, 10, 20, 40):
        xm = P.pcg(b, rtol=0.0, max_iter=m, max_replace=0).x
        assert anorm(x - xm) < 2 * rate ** (m - 1) * e0
    # the Lanczos estimate from the CG coefficients approaches mu from below
    full = P.pcg(b, rtol=1e-12, hist=True)
    kap = oracle.lanczos_condition(full.alpha, full.beta)
    assert 0.9 * mu <= kap <= mu * (1 + 1e-8)


def test_special_cases():
    g, P, b = _tiny()
    assert P.ainv(oracle.PAT_TRIL_A2, 0.05) == oracle.OK
    x_star = np.linalg.solve(P.dense(), b)
    warm = P.pcg(b, x0=x_star, rtol=1e-10)
    assert warm.iters == 0 and warm.status == oracle.OK
    zero = P.pcg(np.zeros(P.n), rtol=1e-10)
    assert zero.iters == 0 and zero.status == oracle.OK and np.all(zero.x == 0)
    capped = P.pcg(b, rtol=1e-14, max_iter=3, max_replace=0)
    assert capped.status == oracle.ENOTCONV and capped.iters == 3


def test_power_of_two_scaling_is_exact():
    """Scaling A and b by 4 leaves every iterate bit-identical (Z unchanged, D x4,
    and every ratio in the recurrence is exact under power-of-two scaling)."""
    g, P, b = _tiny()
    P4 = oracle.OracleProblem(g.nx, g.ny, g.wet, 4 * g.c_e, 4 * g.c_n, 4 * g.shift)
    for Q in (P, P4):
        assert Q.ainv(oracle.PAT_TRIL_A2, 0.05) == oracle.OK
    r1 = P.pcg(b, rtol=1e-10)
    r4 = P4.pcg(4 * b, rtol=1e-10)
    assert r1.iters == r4.iters
    np.testing.assert_array_equal(r1.x, r4.x)


def test_ainv_beats_jacobi_on_coarse_grid():
    """Table 2's direction: the approximate-inverse preconditioner needs fewer
    iterations than NEMO's diagonal one; the wider pattern is not worse."""
    g = gridgen.make_grid(seed=gridgen.seed_for(1), **gridgen.COARSE)
    P = oracle.OracleProblem.from_grid(g)
    b = P.to_wet(g.b)
    it = {}
    for name, pat, tau in [("jacobi", oracle.PAT_DIAG, 0.0), ("trilA", oracle.PAT_TRIL_A, 0.0),
                           ("trilA2", oracle.PAT_TRIL_A2, 0.05)]:
        assert P.ainv(pat, tau) == oracle.OK
        r = P.pcg(b, rtol=1e-10)
        assert r.status == oracle.OK and r.true_relres <= 1e-10
        it[name] = r.iters
    assert it["trilA2"] < it["trilA"] < it["jacobi"]
    assert it["trilA2"] <= 1.05 * it["trilA"]


def test_pole_anisotropy_banded_t_vs_jacobi():
    """Proposition 1 and the pattern-selection scheme of Section 3 in practice:
    shrinking e1 towards the pole (alpha >> beta) makes the east-west
    tridiagonal part T dominate A. The diagonal preconditioner then degrades
    (its iteration count grows several-fold) while the banded inverse factor of
    T barely changes and beats both the diagonal and the tril(A^2) factor."""
    counts = {}
    for tag, an in (("base", 0.0), ("pole", 0.99)):
        g = gridgen.make_grid(seed=gridgen.seed_for(1), pole_anisotropy=an, **gridgen.COARSE)
        P = oracle.OracleProblem.from_grid(g)
        b = P.to_wet(g.b)
        for name, pat, tau, q in (("jacobi", oracle.PAT_DIAG, 0.0, 0), ("trilA2", oracle.PAT_TRIL_A2, 0.05, 0),
                                  ("bandT", oracle.PAT_BAND_T, 0.0, 64)):
            assert P.ainv(pat, tau, q) == oracle.OK
            r = P.pcg(b, rtol=1e-10)
            assert r.status == oracle.OK
            counts[(tag, name)] = r.iters
    assert counts[("pole", "jacobi")] > 2.5 * counts[("base", "jacobi")]
    assert counts[("pole", "bandT")] < 1.2 * counts[("base", "bandT")]
    assert counts[("pole", "bandT")] < counts[("pole", "trilA2")] < counts[("pole", "jacobi")]
