"""Batches of uneven systems in one graph launch (mbpcg_batch_*): every member's x and info are
bit-identical to a solo solve of the same handle, whatever the mix of matrix kinds, sizes, block
widths, algorithms and precisions, and with restarts (the mixed-precision member's refinement
steps at least).
Each member's true residual is recomputed here in FP64."""
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


def members(mb):
    """(matrix, Solver kwargs, tol) of an uneven mix."""
    return [
        (wl.poisson2d(64), dict(s=4), 1e-8),
        (wl.diffusion3d(24, 3), dict(s=8, precond=mb.MBPCG_PRECOND_JACOBI), 1e-8),
        (wl.poisson3d(20), dict(s=1, algo=mb.MBPCG_ALGO_CG), 1e-8),
        (wl.dense_spd(256, 0), dict(s=4), 1e-8),
        (wl.dense_spd(384, 1), dict(s=16, precision=mb.MBPCG_FP64_TC), 1e-8),
        (wl.stencil27(16, 2), dict(s=16, precision=mb.MBPCG_MIXED_FP32), 1e-10),
        (wl.poisson2d(37), dict(s=2), 1e-8),
    ]


def true_relres(A, x, b):
    if hasattr(A, "row_ptr"):
        r = b - A.to_scipy() @ x
    else:
        r = b - np.asarray(A.a) @ x
    return np.linalg.norm(r) / np.linalg.norm(b)


def test_batch_matches_solo_solves_bit_for_bit(mb):
    mem = members(mb)
    solvers = [mb.Solver(A, **kw) for A, kw, _ in mem]
    try:
        bs = [wl.rhs(A.n, 10 + i) for i, (A, _, _) in enumerate(mem)]
        tols = [t for _, _, t in mem]
        # one tolerance per batch call: the members with tol 1e-8 in one batch, the mixed one alone
        groups = {}
        for i, t in enumerate(tols):
            groups.setdefault(t, []).append(i)
        restarted = 0
        for t, idx in groups.items():
            solo = [solvers[i].solve(bs[i], tol=t) for i in idx]
            restarted += sum(info["restarts"] > 0 for _, info in solo)
            with mb.Batch([solvers[i] for i in idx]) as batch:
                got = batch.solve([bs[i] for i in idx], tol=t)
                again = batch.solve([bs[i] for i in idx], tol=t)
            for k, i in enumerate(idx):
                (xs, infs), (xb, infb), (xa, _) = solo[k], got[k], again[k]
                assert np.array_equal(xs, xb) and np.array_equal(xb, xa), i
                for key in ("iterations", "restarts", "status", "best_col"):
                    assert infs[key] == infb[key], (i, key, infs[key], infb[key])
                assert infb["status"] == 0 and true_relres(mem[i][0], xb, bs[i]) <= 1.1 * t, i
        assert restarted > 0, "the restart path (at least the mixed member's refinement) is exercised"
        # the members' own graphs are intact after the batch
        x1, i1 = solvers[0].solve(bs[0], tol=1e-8)
        x2, i2 = solvers[0].solve(bs[0], tol=1e-8)
        assert np.array_equal(x1, x2) and i1["iterations"] == i2["iterations"]
    finally:
        for sv in solvers:
            sv.close()


def test_batch_with_explicit_initial_blocks(mb):
    A1, A2 = wl.poisson2d(48), wl.diffusion3d(20, 1)
    s1, s2 = 4, 8
    sv1, sv2 = mb.Solver(A1, s=s1), mb.Solver(A2, s=s2, precond=1)
    try:
        b1, b2 = wl.rhs(A1.n, 1), wl.rhs(A2.n, 2)
        U1, U2 = wl.initial_block(A1.n, s1, 5), wl.initial_block(A2.n, s2, 6)
        solo = [sv1.solve(b1, U1), sv2.solve(b2, U2)]
        with mb.Batch([sv1, sv2]) as batch:
            got = batch.solve([b1, b2], [U1, U2])
        for (xs, infs), (xb, infb) in zip(solo, got):
            assert np.array_equal(xs, xb) and infs["iterations"] == infb["iterations"]
    finally:
        sv1.close()
        sv2.close()


def test_batch_rejects_bad_members(mb):
    sv = mb.Solver(wl.poisson2d(16), s=2)
    ev = mb.Solver(wl.poisson2d(16), s=2, launch_mode=mb.MBPCG_LAUNCH_EAGER)
    try:
        with pytest.raises(mb.MBPCGError):
            mb.Batch([sv, sv])
        with pytest.raises(mb.MBPCGError):
            mb.Batch([sv, ev])
        with pytest.raises(mb.MBPCGError):
            mb.Batch([])
    finally:
        sv.close()
        ev.close()
