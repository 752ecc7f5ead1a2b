"""Continuous-batching solver server: requests that arrive while others iterate
join the running batch, and each result equals the same solve run alone (same
kernels, same per-grid reduction order, same warm start), bit for bit, and
meets the oracle's acceptance: the true residual recomputed by the FP64 CPU
oracle from the returned x at most rtol, and x within 1e-8 of a tight
reference solution. Also admission by the HBM budget, per-grid ordering,
cancellation and statistics."""
import threading

import numpy as np
import pytest

import gridgen
import oracle
from oracle_checks import judge

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _grids():
    specs = [(dict(gridgen.COARSE), 1), (dict(nx=362, ny=292, land=0.3), 3), (dict(nx=203, ny=77, land=0.3), 7)]
    return [gridgen.make_grid(seed=gridgen.seed_for(ci), **cfg) for cfg, ci in specs]


def _rhs_sequence(g, n, seed):
    rng = np.random.default_rng(seed)
    out, b = [], g.b.copy()
    for _ in range(n):
        b = gridgen.next_rhs(b, g.wet, rng)
        out.append(b)
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_server_results_equal_alone(prec):
    import paper_1210_1878_b300 as pcg
    grids = _grids()
    opts = pcg.make_opts(rtol=1e-10, prec=prec)
    steps = 4
    seqs = [_rhs_sequence(g, steps, 100 + k) for k, g in enumerate(grids)]
    # alone: each grid's timesteps solved in order, warm-started from the previous solution
    alone = []
    for g, seq in zip(grids, seqs):
        h = pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A2, drop_tol=0.05)
        x = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
        res = []
        for k, b in enumerate(seq):
            o = pcg.make_opts(rtol=1e-10, prec=prec, use_x0=(k > 0))
            st = pcg.pcg_solve(h, torch.from_numpy(b).cuda(), x, o)
            res.append((x.cpu().numpy().copy(), st.iters))
        alone.append(res)
        h.close()
    # in the mix: all grids' timesteps submitted at once, interleaved
    hs = [pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A2, drop_tol=0.05) for g in grids]
    srv = pcg.Server(hbm_budget_bytes=8 << 30, max_slots=8, chunk_iters=8, opts=opts)
    gids = [srv.register(h) for h in hs]
    outs, reqs = {}, []
    for k in range(steps):
        for gi, g in enumerate(grids):
            xo = np.zeros((g.ny, g.nx))
            outs[(gi, k)] = xo
            reqs.append(((gi, k), srv.submit(gids[gi], np.ascontiguousarray(seqs[gi][k]), xo, warm_start=(k > 0))))
    probs = [oracle.OracleProblem.from_grid(g) for g in grids]
    for key, rid in reqs:
        rc, st = srv.wait(rid, timeout_ms=120000)
        assert rc == pcg.PCG_OK, (key, rc)
        gi, k = key
        xa, ia = alone[gi][k]
        assert st.iters == ia, (key, st.iters, ia)
        np.testing.assert_array_equal(outs[key], xa)
        P = probs[gi]
        judge(P, grids[gi], P.to_wet(seqs[gi][k]), outs[key], rtol=1e-10, stats=st)
    stats = srv.stats()
    assert stats["completed"] == steps * len(grids) and stats["failed"] == 0
    assert stats["p99_latency_ms"] >= stats["p50_latency_ms"] > 0
    srv.close()


def test_server_admission_budget_and_cancel():
    import paper_1210_1878_b300 as pcg
    coarse, ragged, orca1 = _grids()[0], _grids()[2], _grids()[1]
    grids = [coarse, ragged, orca1]
    hs = [pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A) for g in grids]
    rhs = [g.nx * g.ny * 8 for g in grids]
    # room for both small grids and the right-hand-side buffers of the requests below
    budget = hs[0].resident_bytes + hs[1].resident_bytes + 6 * rhs[0] + rhs[1]
    assert hs[2].resident_bytes > 6 * rhs[0] + rhs[1]
    srv = pcg.Server(hbm_budget_bytes=budget, max_slots=2, chunk_iters=4)
    g0 = srv.register(hs[0])
    g1 = srv.register(hs[1])
    with pytest.raises(pcg.PCGError) as e:
        srv.register(hs[2])
    assert e.value.status == pcg.PCG_EBUDGET
    # several timesteps of one grid queue behind each other (per-grid order);
    # the last one, still queued, can be cancelled
    xs = [np.zeros((grids[0].ny, grids[0].nx)) for _ in range(6)]
    ids = [srv.submit(g0, np.ascontiguousarray(grids[0].b), x, warm_start=False) for x in xs]
    other = srv.submit(g1, np.ascontiguousarray(grids[1].b), np.zeros((grids[1].ny, grids[1].nx)))
    # a seventh queued right-hand side of the first grid would exceed the budget
    # unless a buffer has already come back from a finished request
    try:
        extra = srv.submit(g0, np.ascontiguousarray(grids[0].b), np.zeros((grids[0].ny, grids[0].nx)))
        assert srv.wait(extra, timeout_ms=120000)[0] == pcg.PCG_OK
    except pcg.PCGError as e2:
        assert e2.status == pcg.PCG_EBUDGET
    cancelled = srv.cancel(ids[-1])
    for rid in ids[:-1] + [other]:
        rc, st = srv.wait(rid, timeout_ms=120000)
        assert rc == pcg.PCG_OK
    rc, _ = srv.wait(ids[-1], timeout_ms=120000)
    if cancelled == pcg.PCG_OK:
        assert rc == pcg.PCG_ECANCELLED
    else:
        assert rc == pcg.PCG_OK           # it had already been admitted
    for x in xs[:-1]:
        np.testing.assert_array_equal(x, xs[0])
    srv.close()


def test_server_concurrent_submitters():
    import paper_1210_1878_b300 as pcg
    grids = _grids()
    hs = [pcg.ainv_setup_grid(g, pattern=pcg.PCG_PAT_TRIL_A2, drop_tol=0.05) for g in grids]
    srv = pcg.Server(hbm_budget_bytes=8 << 30, max_slots=4, chunk_iters=8,
                     opts=pcg.make_opts(rtol=1e-10, prec=pcg.PCG_MIXED))
    gids = [srv.register(h) for h in hs]
    errors, done = [], []

    def worker(gi):
        g = grids[gi]
        for k, b in enumerate(_rhs_sequence(g, 3, 200 + gi)):
            x = np.zeros((g.ny, g.nx))
            rid = srv.submit(gids[gi], np.ascontiguousarray(b), x, warm_start=(k > 0))
            rc, st = srv.wait(rid, timeout_ms=120000)
            if rc != pcg.PCG_OK:
                errors.append((gi, k, rc))
            done.append((gi, b, x, st))

    th = [threading.Thread(target=worker, args=(gi,)) for gi in range(len(grids))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    assert srv.stats()["completed"] == 9 and len(done) == 9
    # every result judged by the oracle (not by the device-reported residual)
    probs = [oracle.OracleProblem.from_grid(g) for g in grids]
    for gi, b, x, st in done:
        P = probs[gi]
        judge(P, grids[gi], P.to_wet(b), x, rtol=1e-10, stats=st)
    srv.close()
