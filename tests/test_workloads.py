"""The seeded input generators against closed forms (no GPU): sizes, symmetry, and the extreme
eigenvalues of the constant-coefficient Laplacians, plus the request mix of the serving workload."""
import collections

import numpy as np

import workloads as wl


def test_poisson2d_spectrum_closed_form():
    m = 9
    A = wl.poisson2d(m).to_scipy().toarray()
    h = np.pi / (m + 1)
    lam = np.linalg.eigvalsh(A)
    assert A.shape == (m * m, m * m) and np.array_equal(A, A.T)
    assert abs(lam[0] - (4 - 4 * np.cos(h))) < 1e-12 and abs(lam[-1] - (4 + 4 * np.cos(h))) < 1e-12


def test_poisson3d_sizes_and_spectrum_closed_form():
    for m in (1, 2, 5, 7):
        A = wl.poisson3d(m)
        assert A.n == m ** 3 and A.nnz == 7 * m ** 3 - 6 * m ** 2
    m = 6
    M = wl.poisson3d(m).to_scipy().toarray()
    h = np.pi / (m + 1)
    lam = np.linalg.eigvalsh(M)
    assert np.array_equal(M, M.T)
    assert abs(lam[0] - (6 - 6 * np.cos(h))) < 1e-12 and abs(lam[-1] - (6 + 6 * np.cos(h))) < 1e-12


def test_serving_requests_mix():
    reqs = wl.serving_requests(3000, 0)
    assert reqs == wl.serving_requests(3000, 0)  # seeded
    kinds = collections.Counter(r["kind"] for r in reqs)
    ss = collections.Counter(r["s"] for r in reqs)
    assert set(kinds) == {"poisson2d", "poisson3d", "diffusion3d"} and min(kinds.values()) > 900
    assert set(ss) == {1, 4, 8, 16} and min(ss.values()) > 650
    ns = np.array([r["n"] for r in reqs], dtype=float)
    assert ns.min() >= 900 and ns.max() <= 1.01e6
    # log-uniform: each decade holds about a third of the requests
    dec = np.histogram(np.log10(ns), bins=[2.9, 4.0, 5.0, 6.1])[0]
    assert dec.min() > 800
    assert all(r["precond"] == (1 if r["kind"] == "diffusion3d" else 0) for r in reqs)


def test_dense_spd_spectrum_and_symmetry():
    """The dense family A = Q diag(lambda) Q^T: exactly symmetric, eigenvalues the drawn lambdas
    (up to rounding), all inside [10^lo, 10^hi]; the kappa <= 1e4 variant stays inside its band."""
    for n, lo, hi in ((64, 0.0, 6.0), (100, 0.0, 4.0)):
        D = wl.dense_spd(n, 3, lo, hi)
        A = np.asarray(D.a)
        assert A.flags.f_contiguous and abs(A - A.T).max() == 0.0
        lam = 10.0 ** (lo + (hi - lo) * wl.uniform01(3, 2002, n))
        ev = np.linalg.eigvalsh(A)
        assert np.allclose(np.sort(ev), np.sort(lam), rtol=1e-9, atol=1e-9 * lam.max())
        assert ev.min() >= 10.0 ** lo * (1 - 1e-9) and ev.max() <= 10.0 ** hi * (1 + 1e-9)


def test_stencil27_diagonal_shift():
    """27-point family: every diagonal entry is the row's sum of |off-diagonals| plus 1e-2, so the
    smallest eigenvalue is at least 1e-2 (Gershgorin) and the matrix is SPD."""
    S = wl.stencil27(6, 1).to_scipy().tocsr()
    d = S.diagonal()
    off = np.asarray(abs(S).sum(axis=1)).ravel() - np.abs(d)
    assert np.allclose(d, off + 1e-2, rtol=0, atol=1e-12)
    assert np.linalg.eigvalsh(S.toarray()).min() >= 1e-2 - 1e-12


def test_diffusion3d_harmonic_faces_and_dirichlet_boundary():
    """7-point variable-coefficient diffusion: exactly symmetric, n = m^3 and nnz = 7 m^3 - 6 m^2;
    every off-diagonal is minus the harmonic mean 2 k_a k_b / (k_a + k_b) of the two cells'
    conductivities; each diagonal minus its row's |off-diagonals| is the cell's own k once per
    boundary face (6 minus its neighbours); and the matrix is SPD."""
    m = 5
    A = wl.diffusion3d(m, 2)
    kap = wl.conductivity(m, 2)
    assert kap.min() >= 1e-2 and kap.max() <= 1e2
    assert A.n == m ** 3 and A.nnz == 7 * m ** 3 - 6 * m ** 2
    S = A.to_scipy().tocoo()
    D = S.toarray()
    assert np.array_equal(D, D.T)
    off = S.row != S.col
    r, c, v = S.row[off], S.col[off], S.data[off]
    assert np.allclose(-v, 2 * kap[r] * kap[c] / (kap[r] + kap[c]), rtol=1e-15, atol=0)
    assert np.all(-v >= np.minimum(kap[r], kap[c])) and np.all(-v <= 2 * np.minimum(kap[r], kap[c]))
    nbrs = np.bincount(r, minlength=A.n)
    rowoff = np.bincount(r, weights=-v, minlength=A.n)
    assert np.allclose(np.diag(D) - rowoff, (6 - nbrs) * kap, rtol=1e-13, atol=0)
    assert np.linalg.eigvalsh(D).min() > 0


def test_stencil27_sizes_and_symmetry():
    for m in (1, 2, 4):
        A = wl.stencil27(m, 0)
        assert A.n == m ** 3 and A.nnz == (3 * m - 2) ** 3
        D = A.to_scipy().toarray()
        assert np.array_equal(D, D.T)
        o = D - np.diag(np.diag(D))
        assert np.all(o <= 0) and np.all(o >= -1)
