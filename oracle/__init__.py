"""FP64 CPU oracle: ctypes wrapper around ``oracle/oracle.c``.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package. The CUDA library never
does, and this package never imports the library.

What each function follows is stated in ``oracle.c``'s header: the operator is
Section 3, Eq. 9 negated to its SPD form plus the mass shift of Section 2,
Eq. 2; the preconditioner is the factored approximate inverse of Section 3
built by right-looking conjugate orthogonalisation on a pattern; the solver is
Algorithm 1 (with d = s + beta d) plus a true-residual check on exit.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(closed forms, a hand-derived operator, dense factorisations, invariants).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

PAT_TRIL_A, PAT_TRIL_A2, PAT_FULL, PAT_BAND_T, PAT_DIAG = 0, 1, 2, 3, 4
OK, EINVAL, ENOMEM, ENOTCONV, EBREAKDOWN = 0, 1, 2, 4, 5


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, IEEE binary64, no fused multiply-add)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("replacements", C.c_int32),
                ("pad", C.c_int32), ("relres", C.c_double), ("true_relres", C.c_double),
                ("bnorm", C.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.c_void_p
        dp = C.POINTER(C.c_double)
        lib.oracle_problem_new.restype = P
        lib.oracle_problem_new.argtypes = [C.c_int32, C.c_int32, C.c_void_p, dp, dp, dp]
        lib.oracle_problem_free.argtypes = [P]
        lib.oracle_n.restype = C.c_int32
        lib.oracle_n.argtypes = [P]
        lib.oracle_nnz.restype = C.c_int64
        lib.oracle_nnz.argtypes = [P]
        lib.oracle_get_csr.argtypes = [P, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        lib.oracle_spmv.argtypes = [P, dp, dp]
        lib.oracle_ainv.restype = C.c_int
        lib.oracle_ainv.argtypes = [P, C.c_int32, C.c_double, C.c_int32]
        lib.oracle_z_nnz.restype = C.c_int64
        lib.oracle_z_nnz.argtypes = [P]
        lib.oracle_get_z.argtypes = [P, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        lib.oracle_apply.restype = C.c_int
        lib.oracle_apply.argtypes = [P, dp, dp]
        lib.oracle_pcg.restype = C.c_int
        lib.oracle_pcg.argtypes = [P, dp, dp, C.c_int32, C.c_double, C.c_int32, C.c_int32,
                                   C.POINTER(_Stats), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


@dataclass
class PCGResult:
    x: np.ndarray            # wet-compressed solution
    iters: int
    status: int
    replacements: int
    relres: float            # recursive ||r|| / ||b|| at exit
    true_relres: float       # ||b - A x|| / ||b||
    alpha: np.ndarray
    beta: np.ndarray
    res: np.ndarray          # recursive relative residual after each iteration


class OracleProblem:
    """One grid's operator A over its wet points (natural order), plus the
    preconditioner built by the last call to :meth:`ainv`."""

    def __init__(self, nx, ny, wet, c_e, c_n, shift):
        self._lib = _load()
        self.nx, self.ny = int(nx), int(ny)
        self._wet = np.ascontiguousarray(wet, dtype=np.uint8)
        self._ce = np.ascontiguousarray(c_e, dtype=np.float64)
        self._cn = np.ascontiguousarray(c_n, dtype=np.float64)
        self._sh = np.ascontiguousarray(shift, dtype=np.float64)
        self._h = self._lib.oracle_problem_new(self.nx, self.ny, self._wet.ctypes.data,
                                               _dp(self._ce), _dp(self._cn), _dp(self._sh))
        if not self._h:
            raise ValueError("invalid grid")
        self.n = int(self._lib.oracle_n(self._h))
        self.wet_flat = np.flatnonzero(self._wet.ravel())

    @classmethod
    def from_grid(cls, g):
        return cls(g.nx, g.ny, g.wet, g.c_e, g.c_n, g.shift)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oracle_problem_free(h)
            self._h = None

    # layout helpers: [ny][nx] field <-> wet-compressed vector
    def to_wet(self, field2d) -> np.ndarray:
        return np.ascontiguousarray(np.asarray(field2d, dtype=np.float64).ravel()[self.wet_flat])

    def to_grid(self, v) -> np.ndarray:
        out = np.zeros(self.nx * self.ny)
        out[self.wet_flat] = v
        return out.reshape(self.ny, self.nx)

    def csr(self):
        """(rowptr, col, val, pi, pj) of A."""
        nnz = int(self._lib.oracle_nnz(self._h))
        rp = np.zeros(self.n + 1, np.int64)
        col = np.zeros(nnz, np.int32)
        val = np.zeros(nnz, np.float64)
        pi = np.zeros(self.n, np.int32)
        pj = np.zeros(self.n, np.int32)
        self._lib.oracle_get_csr(self._h, rp.ctypes.data, col.ctypes.data, val.ctypes.data,
                                 pi.ctypes.data, pj.ctypes.data)
        return rp, col, val, pi, pj

    def dense(self) -> np.ndarray:
        rp, col, val, _, _ = self.csr()
        A = np.zeros((self.n, self.n))
        for k in range(self.n):
            A[k, col[rp[k]:rp[k + 1]]] = val[rp[k]:rp[k + 1]]
        return A

    def spmv(self, x) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros(self.n)
        self._lib.oracle_spmv(self._h, _dp(x), _dp(y))
        return y

    def ainv(self, pattern: int, tau: float = 0.0, band_q: int = 0) -> int:
        return int(self._lib.oracle_ainv(self._h, int(pattern), float(tau), int(band_q)))

    def z(self):
        """(colptr, row, val, d): Z column by column over its pattern, and D."""
        nz = int(self._lib.oracle_z_nnz(self._h))
        cp = np.zeros(self.n + 1, np.int64)
        row = np.zeros(nz, np.int32)
        val = np.zeros(nz, np.float64)
        d = np.zeros(self.n, np.float64)
        self._lib.oracle_get_z(self._h, cp.ctypes.data, row.ctypes.data, val.ctypes.data, d.ctypes.data)
        return cp, row, val, d

    def z_dense(self):
        cp, row, val, d = self.z()
        Z = np.zeros((self.n, self.n))
        for j in range(self.n):
            Z[row[cp[j]:cp[j + 1]], j] = val[cp[j]:cp[j + 1]]
        return Z, d

    def apply(self, r) -> np.ndarray:
        r = np.ascontiguousarray(r, dtype=np.float64)
        s = np.zeros(self.n)
        st = self._lib.oracle_apply(self._h, _dp(r), _dp(s))
        if st != OK:
            raise RuntimeError("oracle_apply: no preconditioner built")
        return s

    def pcg(self, b, x0=None, rtol=1e-10, max_iter=None, max_replace=3, hist=False) -> PCGResult:
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
        max_iter = self.n if max_iter is None else int(max_iter)
        cap = max_iter + 1 if hist else 0
        ah = np.zeros(max(cap, 1))
        bh = np.zeros(max(cap, 1))
        rh = np.zeros(max(cap, 1))
        st = _Stats()
        self._lib.oracle_pcg(self._h, _dp(b), _dp(x), int(x0 is not None), float(rtol), max_iter,
                             int(max_replace), C.byref(st),
                             ah.ctypes.data if hist else None, bh.ctypes.data if hist else None,
                             rh.ctypes.data if hist else None, cap)
        it = int(st.iters)
        k = min(it, cap)
        return PCGResult(x=x, iters=it, status=int(st.status), replacements=int(st.replacements),
                         relres=float(st.relres), true_relres=float(st.true_relres),
                         alpha=ah[:k].copy(), beta=bh[:k].copy(), res=rh[:k].copy())


def lanczos_condition(alpha: np.ndarray, beta: np.ndarray) -> float:
    """Condition-number estimate of M^-1 A from the CG coefficients: the
    eigenvalues of the Lanczos tridiagonal T_k with T_ii = 1/alpha_i +
    beta_{i-1}/alpha_{i-1} and T_{i,i+1} = sqrt(beta_i)/alpha_i."""
    k = len(alpha)
    if k == 0:
        return 1.0
    diag = np.empty(k)
    off = np.empty(max(k - 1, 0))
    for i in range(k):
        diag[i] = 1.0 / alpha[i] + (beta[i - 1] / alpha[i - 1] if i > 0 else 0.0)
        if i + 1 < k:
            off[i] = np.sqrt(beta[i]) / alpha[i]
    T = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    ev = np.linalg.eigvalsh(T)
    return float(ev[-1] / ev[0])
