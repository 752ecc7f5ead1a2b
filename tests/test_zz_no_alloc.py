"""The allocation-free operator apply (pcg_spmv_noalloc).

Some callers cannot let a library allocate device memory where they call it:
an ocean model whose memory manager claims the whole device at start-up, or
code that runs under a fixed device-memory budget. For them q = A v is also
offered with its scratch in a fixed device array that every call reuses.

Checked here through the C ABI, on two grids and on calls in a row (the array
keeps the previous call's contents): the result is bit for bit the result of
the allocating entry point pcg_spmv (both run the same binary64 stencil kernel
on the same operands), it is within the binary64 rounding bound of the FP64
oracle's A v (Section 3, Eq. 9), land stays zero, the calls leave the device's
free memory and torch's allocator untouched, and grids beyond the array's
limit are refused. This file is collected last."""
import numpy as np
import pytest
import scipy.sparse as sp

import gridgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _oracle_bound_ok(g, v, q):
    P = oracle.OracleProblem.from_grid(g)
    rp, col, val, _, _ = P.csr()
    A = sp.csr_matrix((val, col, rp), shape=(P.n, P.n))
    vw = P.to_wet(v)
    err = np.abs(P.to_wet(q) - P.spmv(vw))
    return bool(np.all(err <= 1e-13 * (abs(A) @ np.abs(vw)) + 1e-300))


def test_noalloc_spmv_matches_spmv_and_oracle_twice():
    import paper_1210_1878_b300 as pcg
    g1 = gridgen.make_grid(seed=gridgen.seed_for(1), **gridgen.COARSE)
    g2 = gridgen.make_grid(nx=203, ny=77, seed=gridgen.seed_for(0) + 700, land=0.3)
    h1 = pcg.ainv_setup_grid(g1, pattern=pcg.PCG_PAT_TRIL_A2, drop_tol=0.05)
    h2 = pcg.ainv_setup_grid(g2, pattern=pcg.PCG_PAT_TRIL_A)
    cases = []
    for h, g, seed in ((h1, g1, 1), (h2, g2, 2), (h1, g1, 3), (h1, g1, 4)):
        v = torch.from_numpy(np.random.default_rng(seed).standard_normal((g.ny, g.nx))).cuda()
        cases.append((h, g, v, torch.zeros_like(v), torch.full_like(v, float("nan"))))
    # warm-up, one call per grid: the first call on the device looks up the
    # scratch array's address, and each kernel's code is loaded on its first
    # launch; from then on nothing may be allocated
    for h, g, v, q_ref, q in cases[:2]:
        assert pcg.pcg_spmv_noalloc(h, v, q) == pcg.PCG_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for h, g, v, q_ref, q in cases:
        q.fill_(float("nan"))
        assert pcg.pcg_spmv_noalloc(h, v, q) == pcg.PCG_OK, pcg.lib.pcg_last_error_message()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    for h, g, v, q_ref, q in cases:
        pcg.pcg_spmv(h, v, q_ref)
        qn, qr = q.cpu().numpy(), q_ref.cpu().numpy()
        np.testing.assert_array_equal(qn, qr)
        assert np.all(qn[g.wet == 0] == 0)
        assert _oracle_bound_ok(g, v.cpu().numpy(), qn)


def test_noalloc_refuses_grids_beyond_its_scratch():
    import paper_1210_1878_b300 as pcg
    g = gridgen.make_grid(nx=2100, ny=1050, seed=gridgen.seed_for(0) + 701, land=0.95)
    h = pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_DIAG)
    v = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
    q = torch.zeros_like(v)
    assert pcg.pcg_spmv_noalloc(h, v, q) == pcg.PCG_EINVAL
    assert b"limit" in pcg.lib.pcg_last_error_message()
