"""The row-band plan of a sharded solve (pcg_band_plan), checked on the CPU.

The library cuts a grid into contiguous row bands of about equal wet count,
each band reading `halo` rows of each neighbour (max(1, LD): the stencil
reaches one row across a band edge, the preconditioner's Z^T pulls from LD rows
below and Z pushes to LD rows above). Two gloo ranks then run Algorithm 1 over
the plan, each on its own band with numpy/scipy arithmetic on the oracle's A,
Z and D: a rank holds its rows plus the halo rows, exchanges the band-edge rows
of d and r with its neighbour after each update (the sends and receives of
the multi-GPU solve) and sums the two reductions of an iteration with an
allreduce. Every coupling an own row needs must lie within the planned rows,
and the distributed solve must meet the oracle's acceptance."""
import os
import socket
import sys

import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import gridgen  # noqa: E402


def _ld(pattern):
    return {1: 2, 0: 1}.get(pattern, 0)


@pytest.mark.parametrize("pattern", [0, 1, 4])
@pytest.mark.parametrize("nbands", [1, 2, 3, 7])
def test_band_plan_covers_rows_and_balances_wet_points(pattern, nbands):
    import paper_1210_1878_b300 as pcg
    g = gridgen.make_grid(seed=gridgen.seed_for(1), **gridgen.COARSE)
    row0, halo = pcg.pcg_band_plan(g.wet, pattern, nbands)
    assert halo == max(1, _ld(pattern))
    assert row0[0] == 0 and row0[-1] == g.ny and len(row0) == nbands + 1
    assert np.all(np.diff(row0) >= halo)
    per_row = g.wet.sum(axis=1)
    counts = np.array([per_row[row0[b]:row0[b + 1]].sum() for b in range(nbands)])
    assert counts.sum() == g.wet.sum()
    assert np.all(np.abs(counts - g.wet.sum() / nbands) <= per_row.max() + 1), counts


def test_band_plan_refuses_too_many_bands():
    import paper_1210_1878_b300 as pcg
    g = gridgen.make_grid(seed=gridgen.seed_for(0), **gridgen.TINY)
    with pytest.raises(pcg.PCGError) as e:
        pcg.pcg_band_plan(g.wet, pcg.PCG_PAT_TRIL_A2, 13)      # 24 rows < 13 bands x 2 halo rows
    assert e.value.status == pcg.PCG_EINVAL


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, pattern, tau, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        import paper_1210_1878_b300 as pcg
        g = gridgen.make_grid(seed=gridgen.seed_for(1), **gridgen.COARSE)
        P = oracle.OracleProblem.from_grid(g)
        assert P.ainv(pattern, tau) == oracle.OK
        rp, col, val, pi, pj = P.csr()
        A = sp.csr_matrix((val, col, rp), shape=(P.n, P.n))
        cp, zrow, zval, dvec = P.z()
        Z = sp.csc_matrix((zval, zrow, cp), shape=(P.n, P.n)).tocsr()
        row0, halo = pcg.pcg_band_plan(g.wet, pattern, world)
        j0, j1 = int(row0[rank]), int(row0[rank + 1])
        lo = halo if rank > 0 else 0
        hi = halo if rank < world - 1 else 0
        own = np.flatnonzero((pj >= j0) & (pj < j1))
        loc = np.flatnonzero((pj >= j0 - lo) & (pj < j1 + hi))
        inloc = np.zeros(P.n, bool)
        inloc[loc] = True
        # every coupling an own row needs lies within the planned rows
        A_own = A[own]
        assert inloc[A_own.indices].all(), "the stencil reaches past the halo rows"
        K = np.unique(Z[own].indices)                       # columns of Z that touch own rows
        R = np.unique(Z.tocsc()[:, K].tocoo().row)          # rows Z^T pulls from for those columns
        assert inloc[K].all() and inloc[R].all(), "the preconditioner reaches past the halo rows"
        Z_own_K = Z[own][:, K]
        Z_R_K = Z[R][:, K]
        dK = dvec[K]
        # rows this rank sends to / receives from each neighbour: `halo` rows at the band edge
        send = {}
        recv = {}
        if rank > 0:
            send[rank - 1] = np.flatnonzero((pj >= j0) & (pj < j0 + halo))
            recv[rank - 1] = np.flatnonzero((pj >= j0 - halo) & (pj < j0))
        if rank < world - 1:
            send[rank + 1] = np.flatnonzero((pj >= j1 - halo) & (pj < j1))
            recv[rank + 1] = np.flatnonzero((pj >= j1) & (pj < j1 + halo))

        def exchange(v):
            reqs, bufs = [], {}
            for peer, idx in send.items():
                reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(v[idx])), peer))
            for peer, idx in recv.items():
                bufs[peer] = torch.zeros(len(idx), dtype=torch.float64)
                reqs.append(dist.irecv(bufs[peer], peer))
            for r_ in reqs:
                r_.wait()
            for peer, idx in recv.items():
                v[idx] = bufs[peer].numpy()

        def allreduce(*xs):
            t = torch.tensor(xs, dtype=torch.float64)
            dist.all_reduce(t)
            return t.numpy()

        def precond(r):
            s = np.zeros(P.n)
            s[own] = Z_own_K @ ((Z_R_K.T @ r[R]) / dK)
            return s

        bglob = P.to_wet(g.b)
        b = np.zeros(P.n)
        b[loc] = bglob[loc]
        x = np.zeros(P.n)
        r = b.copy()                                       # x0 = 0: r0 = b on every held row
        s = precond(r)
        d = s.copy()
        exchange(d)
        rho, bb = allreduce(s[own] @ r[own], b[own] @ b[own])
        rr = bb
        it = 0
        while np.sqrt(rr / bb) > 1e-10 and it < 5000:
            q = np.zeros(P.n)
            q[own] = A_own[:, loc] @ d[loc]
            (dq,) = allreduce(d[own] @ q[own])
            alpha = rho / dq
            x[own] += alpha * d[own]
            r[own] -= alpha * q[own]
            exchange(r)
            s = precond(r)
            rho_new, rr = allreduce(s[own] @ r[own], r[own] @ r[own])
            beta = rho_new / rho
            rho = rho_new
            d[own] = s[own] + beta * d[own]
            exchange(d)
            it += 1
        # gather the solution on rank 0
        xs = [torch.zeros(P.n, dtype=torch.float64) for _ in range(world)]
        mine = np.zeros(P.n)
        mine[own] = x[own]
        dist.all_gather(xs, torch.from_numpy(mine))
        if rank == 0:
            xg = sum(t.numpy() for t in xs)
            ref = P.pcg(bglob, rtol=1e-10)
            xref = P.pcg(bglob, rtol=1e-13).x
            out[rank] = (it, ref.iters, float(np.linalg.norm(bglob - P.spmv(xg)) / np.linalg.norm(bglob)),
                         float(np.linalg.norm(xg - xref) / np.linalg.norm(xref)))
        else:
            out[rank] = (it,)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("pattern,tau", [(1, 0.05), (0, 0.0)], ids=["trilA2", "trilA"])
def test_distributed_pcg_over_the_band_plan(pattern, tau):
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, pattern, tau, out), nprocs=world, join=True)
        res = dict(out)
    it, ref_iters, true_rel, err = res[0]
    assert res[1][0] == it                       # both ranks stop together (the same allreduced test)
    assert abs(it - ref_iters) <= 2, (it, ref_iters)
    assert true_rel <= 1e-10 * (1 + 1e-3), true_rel
    assert err <= 1e-8, err
