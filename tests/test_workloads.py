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
