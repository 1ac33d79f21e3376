"""The continuous-batching request server (include/mbpcg_server.h) on the GPU: every result is
bit-identical whether its solve ran alone or among others (and equal to the plain handle API),
admission respects the HBM budget, concurrent solves really overlap, and errors come back per
request without disturbing the others."""
import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_07327_gb300 as mb
    mb.lib()
    return mb


def mix():
    """Requests of different kinds, n, nnz and s (one CG)."""
    return [
        dict(A=wl.poisson2d(24), s=4, precond=0, algo=0, seed=11),
        dict(A=wl.diffusion3d(10, 3), s=8, precond=1, algo=0, seed=12),
        dict(A=wl.poisson2d(40), s=1, precond=0, algo=0, seed=13),
        dict(A=wl.stencil27(8, 4), s=16, precond=0, algo=0, seed=14),
        dict(A=wl.poisson3d(12), s=4, precond=0, algo=0, seed=15),
        dict(A=wl.diffusion3d(14, 5), s=16, precond=1, algo=0, seed=16),
        dict(A=wl.poisson3d(16), s=1, precond=0, algo=1, seed=17),
        dict(A=wl.poisson2d(64), s=32, precond=0, algo=0, seed=18),
    ]


def submit_all(srv, reqs, tol=1e-8):
    return [srv.submit(r["A"], wl.rhs(r["A"].n, r["seed"]), s=r["s"], precond=r["precond"], algo=r["algo"], tol=tol,
                       maxit=20000, seed=r["seed"]) for r in reqs]


def test_results_identical_alone_and_in_the_mix(mb):
    reqs = mix()
    alone = []
    with mb.Server(slots=1) as srv:
        for r in reqs:
            (t,) = submit_all(srv, [r])
            alone.append(srv.wait(t))
    with mb.Server(slots=4) as srv:
        tickets = submit_all(srv, reqs)
        mixed = [srv.wait(t) for t in reversed(tickets)][::-1]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["peak_active"] >= 2
    for r, a, m in zip(reqs, alone, mixed):
        assert a["status"] == 0 and m["status"] == 0
        assert a["info"]["relres_true"] <= 1e-8
        assert a["info"]["iterations"] == m["info"]["iterations"]
        assert np.array_equal(a["x"], m["x"]), (r["A"].n, r["s"])
    # and the same bits as the plain handle API with the same seed
    r, a = reqs[1], alone[1]
    sv = mb.Solver(r["A"], s=r["s"], precond=r["precond"], seed=r["seed"])
    x, info = sv.solve(wl.rhs(r["A"].n, r["seed"]), tol=1e-8, maxit=20000)
    sv.close()
    assert np.array_equal(np.asarray(x), a["x"]) and info["iterations"] == a["info"]["iterations"]


def test_concurrent_solves_overlap_on_the_device(mb):
    """Eight copies of one mid-size solve: with 8 slots the batch finishes well before 8 x the time of
    one, because the solves run at the same time."""
    import time
    A = wl.diffusion3d(32, 7)
    b = wl.rhs(A.n, 1)
    with mb.Server(slots=8) as srv:
        t = srv.submit(A, b, s=4, precond=1, seed=1)
        srv.wait(t)  # warm-up
        t0 = time.perf_counter()
        srv.wait(srv.submit(A, b, s=4, precond=1, seed=1))
        one = time.perf_counter() - t0
        t0 = time.perf_counter()
        ts = [srv.submit(A, b, s=4, precond=1, seed=1) for _ in range(8)]
        res = [srv.wait(t) for t in ts]
        eight = time.perf_counter() - t0
        assert srv.stats()["peak_active"] >= 4
    assert all(r["status"] == 0 for r in res)
    assert all(np.array_equal(r["x"], res[0]["x"]) for r in res)
    assert eight < 0.6 * 8 * one, (one, eight)


def test_admission_respects_the_budget(mb):
    big = wl.poisson3d(30)
    need = mb.mbpcg_workspace_size_csr(big.n, big.nnz, 16) + 256
    budget = int(need * 1.5)  # room for one of these at a time (plus small ones)
    with mb.Server(slots=4, hbm_budget_bytes=budget) as srv:
        ts = [srv.submit(big, wl.rhs(big.n, i + 1), s=16, seed=i + 1) for i in range(4)]
        res = [srv.wait(t) for t in ts]
        st = srv.stats()
    assert all(r["status"] == 0 for r in res)
    assert st["peak_bytes"] <= budget and st["peak_active"] == 1 and st["budget_bytes"] == budget


def test_errors_are_per_request(mb):
    good = wl.poisson2d(20)
    bad = wl.poisson2d(20)
    bad.val[bad.row_ptr[5]:bad.row_ptr[6]] = 0.0  # row 5 loses its diagonal: not SPD
    with mb.Server(slots=2) as srv:
        t_good = srv.submit(good, wl.rhs(good.n, 1), s=4, seed=1)
        t_bad = srv.submit(bad, wl.rhs(bad.n, 1), s=4, seed=1)
        r_bad, r_good = srv.wait(t_bad), srv.wait(t_good)
        assert r_bad["status"] == mb._native.MBPCG_ERR_NOT_SPD and r_good["status"] == 0
        st, _, _, _ = mb.mbpcg_server_wait(srv._srv, t_good)  # already released
        assert st == mb._native.MBPCG_ERR_INVALID
        with pytest.raises(mb.MBPCGError):
            srv.submit(good, wl.rhs(good.n, 1), s=33)
    with mb.Server(slots=1, hbm_budget_bytes=1 << 16) as srv:
        with pytest.raises(mb.MBPCGError, match="budget"):
            srv.submit(good, wl.rhs(good.n, 1), s=4)
    with pytest.raises(mb.MBPCGError):
        mb.Server(slots=0)
