"""Pins of the oracle's factored approximate inverse M^-1 = Z D^-1 Z^T
(Section 3: conjugate orthogonalisation on a sparsity pattern, Propositions
2 and 3, pattern-selection steps 1-6) against dense factorisations written in
the tests, the closed form of Proposition 3, and invariants."""
import math

import numpy as np
import pytest

import gridgen
import oracle


def _tiny():
    g = gridgen.make_grid(seed=gridgen.seed_for(0), **gridgen.TINY)
    return g, oracle.OracleProblem.from_grid(g)


def _ldlt(A):
    """Textbook LDL^T of an SPD matrix: A = L D L^T, L unit lower triangular."""
    n = A.shape[0]
    L = np.eye(n)
    D = np.zeros(n)
    for j in range(n):
        D[j] = A[j, j] - np.sum(L[j, :j] ** 2 * D[:j])
        for i in range(j + 1, n):
            L[i, j] = (A[i, j] - np.sum(L[i, :j] * L[j, :j] * D[:j])) / D[j]
    return L, D


def test_full_pattern_is_exact_inverse():
    g, P = _tiny()
    assert P.ainv(oracle.PAT_FULL) == oracle.OK
    Z, d = P.z_dense()
    A = P.dense()
    Ainv = np.linalg.inv(A)
    np.testing.assert_allclose(Z @ np.diag(1 / d) @ Z.T, Ainv, rtol=0, atol=1e-12 * np.abs(Ainv).max())
    L, D = _ldlt(A)
    np.testing.assert_allclose(d, D, rtol=1e-12)
    np.testing.assert_allclose(Z, np.linalg.inv(L).T, rtol=0, atol=1e-12)
    # Z^T A Z = D (A-orthogonal columns)
    np.testing.assert_allclose(Z.T @ A @ Z, np.diag(d), rtol=0, atol=1e-9 * d.max())


def _lower_structure(A, q):
    S = (A != 0).astype(np.int64)
    R = np.eye(A.shape[0], dtype=np.int64)
    for _ in range(q):
        R = np.minimum(R @ S, 1)
    return np.triu(R.T) > 0          # Z[m, k] allowed iff m <= k and (A^q)[m, k] != 0


@pytest.mark.parametrize("pattern,q,tau", [(oracle.PAT_TRIL_A, 1, 0.0), (oracle.PAT_TRIL_A2, 2, 0.0),
                                           (oracle.PAT_TRIL_A2, 2, 0.05), (oracle.PAT_TRIL_A2, 2, 0.3)])
def test_pattern_invariants(pattern, q, tau):
    g, P = _tiny()
    assert P.ainv(pattern, tau) == oracle.OK
    Z, d = P.z_dense()
    A = P.dense()
    allowed = _lower_structure(A, q)
    assert np.all(Z[~allowed] == 0)
    assert np.all(np.diag(Z) == 1.0)
    assert np.all(d > 0)
    # M-matrix: the approximate inverse factor stays entrywise non-negative
    assert np.all(Z >= 0)
    M = Z @ np.diag(1 / d) @ Z.T
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0
    # the drop rule: every surviving off-diagonal passes the scaled threshold
    if tau > 0:
        a = np.diag(A)
        m_idx, k_idx = np.nonzero(np.triu(Z, 1))
        assert np.all(np.abs(Z[m_idx, k_idx]) * np.sqrt(a[m_idx] / a[k_idx]) >= tau)
    if pattern == oracle.PAT_TRIL_A2 and tau == 0.3:
        assert np.count_nonzero(np.triu(Z, 1)) < np.count_nonzero(np.triu(allowed, 1))
    if tau == 0 and pattern == oracle.PAT_TRIL_A:
        # M-matrix, connected rows: with nothing dropped Z fills the structure of tril(A)
        assert np.array_equal(Z != 0, allowed)
    if tau == 0 and pattern == oracle.PAT_TRIL_A2:
        # two-step couplings (WW, SS, SW, SE) are filled, beyond tril(A)
        assert np.count_nonzero((Z != 0) & ~_lower_structure(A, 1)) > Z.shape[0]


def _path_grid(n, c=1.0, s_end=1.0, s_mid=0.0, cvar=None):
    """One latitude row of n wet cells closed by one land cell (no periodic face):
    A is tridiagonal. With s_end = c on the two end cells every diagonal is 2c."""
    nx = n + 1
    wet = np.ones((1, nx), np.uint8)
    wet[0, -1] = 0
    ce = np.full((1, nx), c) if cvar is None else np.asarray(cvar, float).reshape(1, nx)
    ce[0, -2:] = 0.0
    cn = np.zeros((1, nx))
    sh = np.full((1, nx), s_mid)
    sh[0, 0] = sh[0, n - 1] = s_end
    return oracle.OracleProblem(nx, 1, wet, ce, cn, sh)


def test_drop_rule_hand_computed():
    """Right-looking construction with drops after each update (Section 3),
    worked by hand on three wet cells in a row, A = tridiag(-1; 2, 5, 2):
    i = 1 gives z_12 = 1/2 with scaled size (1/2) sqrt(2/5) = 0.316; i = 2 then
    has d_2 = 5 - 1/2 (or 5 if z_12 was dropped) and z_23 = 1/d_2 with scaled
    size z_23 sqrt(5/2); d_3 = 2 - z_23. At tau = 0.4 both entries drop; at
    tau = 0.3 both stay (0.316 and 0.351), so Z and D are the values below.
    An unscaled or inversely scaled test keeps z_12 at 0.4 or drops z_23 at 0.3."""
    P = _path_grid(3, c=1.0, s_end=1.0, s_mid=3.0)
    assert np.array_equal(np.diag(P.dense()), [2.0, 5.0, 2.0])
    assert P.ainv(oracle.PAT_TRIL_A, 0.4) == oracle.OK
    Z, d = P.z_dense()
    assert np.array_equal(Z, np.eye(3)) and np.array_equal(d, [2.0, 5.0, 2.0])
    assert P.ainv(oracle.PAT_TRIL_A, 0.3) == oracle.OK
    Z, d = P.z_dense()
    Zh = np.array([[1.0, 0.5, 0.0], [0.0, 1.0, 2.0 / 9.0], [0.0, 0.0, 1.0]])
    assert np.allclose(Z, Zh, rtol=1e-15, atol=0) and np.allclose(d, [2.0, 4.5, 16.0 / 9.0], rtol=1e-15, atol=0)


def _cholesky_upper_tridiag(T):
    """Textbook Cholesky T = U^T U of a tridiagonal SPD matrix (U upper bidiagonal)."""
    n = T.shape[0]
    U = np.zeros((n, n))
    for k in range(n):
        U[k, k] = math.sqrt(T[k, k] - (U[k - 1, k] ** 2 if k > 0 else 0.0))
        if k + 1 < n:
            U[k, k + 1] = T[k, k + 1] / U[k, k]
    return U


def test_proposition3_closed_form_and_decay():
    """Proposition 3: for T = U^T U tridiagonal and diagonally dominant, the
    columns of U^-1 follow z_{k-i,k} = (-1)^i / u_kk prod_{r=1..i} u_{k-r,k-r+1}/u_{k-r,k-r}.
    The oracle's unit factor is Z = U^-1 diag(u_kk), D = diag(u_kk^2)."""
    n = 12
    rng = np.random.default_rng(5)
    cvar = np.concatenate([rng.uniform(0.5, 2.0, n), [0.0]])
    P = _path_grid(n, s_end=0.3, s_mid=0.3, cvar=cvar)
    assert P.ainv(oracle.PAT_FULL) == oracle.OK
    Z, d = P.z_dense()
    U = _cholesky_upper_tridiag(P.dense())
    np.testing.assert_allclose(d, np.diag(U) ** 2, rtol=1e-13)
    for k in range(n):
        for i in range(k + 1):
            closed = (-1) ** i / U[k, k] * np.prod([U[k - r, k - r + 1] / U[k - r, k - r] for r in range(1, i + 1)])
            assert Z[k - i, k] == pytest.approx(closed * U[k, k], rel=1e-12)
        # Proposition 2 (U diagonally dominant) and the strict decay of Proposition 3
        if k + 1 < n:
            assert abs(U[k, k]) > abs(U[k, k + 1])
        col = Z[:k + 1, k][::-1]
        assert np.all(col > 0) and np.all(np.diff(col) < 0)


@pytest.mark.parametrize("q", [1, 2, 4])
def test_banded_pattern_is_truncation(q):
    """Pattern-selection steps 4-6: for a tridiagonal matrix the pattern-restricted
    factor equals the exact factor truncated to the band, and D is exact."""
    n = 15
    P = _path_grid(n, c=1.3, s_end=0.2, s_mid=0.05)
    assert P.ainv(oracle.PAT_FULL) == oracle.OK
    Zf, df = P.z_dense()
    assert P.ainv(oracle.PAT_BAND_T, band_q=q) == oracle.OK
    Zb, db = P.z_dense()
    band = np.triu(np.ones((n, n), bool)) & ~np.triu(np.ones((n, n), bool), q + 1)
    np.testing.assert_allclose(Zb, np.where(band, Zf, 0.0), rtol=1e-13, atol=0)
    np.testing.assert_allclose(db, df, rtol=1e-13)
    if q == 1:
        assert P.ainv(oracle.PAT_TRIL_A) == oracle.OK
        Za, da = P.z_dense()
        np.testing.assert_array_equal(Za, Zb)


def test_band_t_on_a_grid_uses_row_blocks():
    """BAND_T builds Z from T = east-west tridiagonal part of A (no periodic face):
    Z is block diagonal over latitude runs and each block is the banded inverse
    factor of that run's T."""
    g, P = _tiny()
    q = 3
    assert P.ainv(oracle.PAT_BAND_T, band_q=q) == oracle.OK
    Z, d = P.z_dense()
    rp, col, val, pi, pj = P.csr()
    A = P.dense()
    n = P.n
    T = np.zeros_like(A)
    for k in range(n):
        for t in range(rp[k], rp[k + 1]):
            m = col[t]
            if m == k or (pj[m] == pj[k] and abs(int(pi[m]) - int(pi[k])) == 1):
                T[k, m] = val[t]
    L, D = _ldlt(T)
    Zt = np.linalg.inv(L).T
    idx = np.arange(n)
    band = (idx[None, :] - idx[:, None] >= 0) & (idx[None, :] - idx[:, None] <= q)
    np.testing.assert_allclose(Z, np.where(band, Zt, 0.0), rtol=0, atol=1e-12)
    np.testing.assert_allclose(d, D, rtol=1e-12)


def test_proposition1_limit_spectrum():
    """Proposition 1 (reading: the eigenvalues are 1 - cos(k pi/(n+1)), the same set
    as the printed 1 + cos(k pi/(n+1))): with every diagonal equal to 2c the
    Jacobi-preconditioned tridiagonal operator is tridiag(-1/2, 1, -1/2), with
    condition number cot^2(pi / (2(n+1)))."""
    n = 20
    P = _path_grid(n, c=1.0, s_end=1.0, s_mid=0.0)
    assert P.ainv(oracle.PAT_DIAG) == oracle.OK
    Z, d = P.z_dense()
    A = P.dense()
    Dm = np.diag(1 / np.sqrt(d))
    ev = np.sort(np.linalg.eigvalsh(Dm @ A @ Dm))
    k = np.arange(1, n + 1)
    np.testing.assert_allclose(ev, np.sort(1 + np.cos(k * np.pi / (n + 1))), atol=1e-13)
    np.testing.assert_allclose(ev, np.sort(1 - np.cos(k * np.pi / (n + 1))), atol=1e-13)
    assert ev[-1] / ev[0] == pytest.approx(1 / math.tan(math.pi / (2 * (n + 1))) ** 2, rel=1e-10)
