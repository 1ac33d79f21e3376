"""Seeded synthetic inputs shared by the CUDA library's tests/benchmark and by the oracle.

This module holds input generation only -- no step of the solver. Every random draw comes from
one counter-based generator so that the same (seed, stream, index) gives the same number on any
machine and inside the CUDA library (which implements the same published generator for its own
"generate U on the device" option):

  SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
    mix(z):  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
             z = (z ^ (z >> 27)) * 0x94D049BB133111EB
             return z ^ (z >> 31)                          (all arithmetic mod 2^64)
  Counter-based use:  key  = mix(seed + (stream + 1) * 0x9E3779B97F4A7C15)
                      word = mix(key  + (index  + 1) * 0x9E3779B97F4A7C15)
  Uniform [0,1): (word >> 11) * 2^-53;  Uniform(-1,1): 2u - 1 (the paper's U and b, Sections 2, 4).

Stream assignment: b uses stream 0, column j of U uses stream 1 + j, coefficient fields use
streams >= 1000 (see each generator).

Workload families (synthetic stand-ins for the paper's SuiteSparse and random dense systems, whose
data is not available): 2D 5-point Poisson, 3D 7-point variable-coefficient diffusion, 3D 27-point
diagonally shifted stencil, dense Q diag(lambda) Q^T, and the paper's dense M^T M (Section 4).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix_words(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """64-bit words word(seed, stream, index) for index in [start, start+count)."""
    with np.errstate(over="ignore"):
        key = _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + np.uint64(stream + 1) * _GOLDEN)
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix(key + idx * _GOLDEN)


def uniform01(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    w = splitmix_words(seed, stream, count, start)
    return (w >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform01_at(seed: int, stream: int, index: np.ndarray) -> np.ndarray:
    """Uniform [0,1) at arbitrary counter values (same generator as uniform01)."""
    with np.errstate(over="ignore"):
        key = _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + np.uint64(stream + 1) * _GOLDEN)
        w = _mix(key + (np.asarray(index, dtype=np.uint64) + np.uint64(1)) * _GOLDEN)
    return (w >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    return 2.0 * uniform01(seed, stream, count, start) - 1.0


def rhs(n: int, seed: int) -> np.ndarray:
    """b with i.i.d. Uniform(-1,1) entries (Section 4), stream 0."""
    return uniform_pm1(seed, 0, n)


def perturbed_rhs(b: np.ndarray, k: int) -> np.ndarray:
    """b with every entry scaled by (1 + 1e-16 u), u ~ Uniform(-1,1) from seed k, stream 7000: a
    rounding-level change of b (about half the entries move by one ulp) used to measure how far
    an iteration count moves under rounding alone. k = 0 is b itself."""
    if k == 0:
        return np.array(b, dtype=np.float64)
    return b * (1 + 1e-16 * uniform_pm1(k, 7000, b.size))


def initial_block(n: int, k: int, seed: int) -> np.ndarray:
    """U (n x k, column-major / Fortran order) with i.i.d. Uniform(-1,1) entries (Algorithm 1);
    column j comes from stream 1 + j."""
    U = np.empty((n, k), dtype=np.float64, order="F")
    for j in range(k):
        U[:, j] = uniform_pm1(seed, 1 + j, n)
    return U


@dataclass
class CSR:
    """Square CSR matrix with int32 indices and float64 values, columns sorted in each row."""
    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col_idx, self.row_ptr), shape=(self.n, self.n))

    def diagonal(self) -> np.ndarray:
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        d = np.zeros(self.n)
        m = rows == self.col_idx
        np.add.at(d, rows[m], self.val[m])
        return d


@dataclass
class Dense:
    """Square dense matrix stored column-major (Fortran order), float64."""
    n: int
    a: np.ndarray

    @property
    def nnz(self) -> int:
        return self.n * self.n


def _csr_from_entries(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> CSR:
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2 ** 31:
        raise ValueError("nnz does not fit int32 indices")
    return CSR(n, row_ptr.astype(np.int32), cols.astype(np.int32), vals.astype(np.float64))


def poisson2d(m: int) -> CSR:
    """2D 5-point Poisson on an m x m interior grid with Dirichlet boundary: diagonal 4,
    neighbours -1, natural (row-major) ordering. n = m^2, nnz = 5 m^2 - 4 m."""
    n = m * m
    idx = np.arange(n, dtype=np.int64)
    y, x = idx // m, idx % m
    rows, cols, vals = [idx], [idx], [np.full(n, 4.0)]
    for dy, dx in ((-1, 0), (0, -1), (0, 1), (1, 0)):
        ok = (y + dy >= 0) & (y + dy < m) & (x + dx >= 0) & (x + dx < m)
        rows.append(idx[ok])
        cols.append(idx[ok] + dy * m + dx)
        vals.append(np.full(int(ok.sum()), -1.0))
    return _csr_from_entries(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def poisson3d(m: int) -> CSR:
    """3D 7-point Poisson Laplacian on an m^3 interior grid, Dirichlet: diagonal 6, neighbours -1.
    n = m^3, nnz = 7 m^3 - 6 m^2."""
    n = m ** 3
    idx = np.arange(n, dtype=np.int64)
    z, y, x = idx // (m * m), (idx // m) % m, idx % m
    rows, cols, vals = [idx], [idx], [np.full(n, 6.0)]
    for dz, dy, dx in ((-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 1), (0, 1, 0), (1, 0, 0)):
        ok = ((z + dz >= 0) & (z + dz < m) & (y + dy >= 0) & (y + dy < m) & (x + dx >= 0) & (x + dx < m))
        rows.append(idx[ok])
        cols.append(idx[ok] + dz * m * m + dy * m + dx)
        vals.append(np.full(int(ok.sum()), -1.0))
    return _csr_from_entries(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def serving_requests(count: int, seed: int, n_lo: float = 1e3, n_hi: float = 1e6, sizes: int = 24):
    """A stream of solve requests shaped like the serving workload: kind in {2D Poisson, 3D Poisson,
    3D diffusion (Jacobi)} uniformly, n log-uniform in [n_lo, n_hi] rounded to the nearest of
    `sizes` log-spaced grid sides per kind (so matrices can be cached), s uniform in {1, 4, 8, 16}.
    Returns dicts (kind, m, n, s, precond, rhs_seed); draws from streams 7000-7002 of `seed`."""
    u_kind = uniform01(seed, 7000, count)
    u_n = uniform01(seed, 7001, count)
    u_s = uniform01(seed, 7002, count)
    out = []
    for i in range(count):
        kind = ("poisson2d", "poisson3d", "diffusion3d")[min(int(u_kind[i] * 3), 2)]
        n = n_lo * (n_hi / n_lo) ** u_n[i]
        dim = 2 if kind == "poisson2d" else 3
        lo, hi = n_lo ** (1.0 / dim), n_hi ** (1.0 / dim)
        grid = np.unique(np.round(lo * (hi / lo) ** np.linspace(0.0, 1.0, sizes)).astype(int))
        m = int(grid[np.argmin(np.abs(np.log(grid) - np.log(n) / dim))])
        s = (1, 4, 8, 16)[min(int(u_s[i] * 4), 3)]
        out.append(dict(kind=kind, m=m, n=m ** dim, s=s, precond=1 if kind == "diffusion3d" else 0, rhs_seed=i + 1))
    return out


def conductivity(m: int, seed: int) -> np.ndarray:
    """Per-cell conductivity kappa = 10^U[-2,2] on an m^3 grid (stream 1000)."""
    return 10.0 ** (4.0 * uniform01(seed, 1000, m ** 3) - 2.0)


def diffusion3d(m: int, seed: int) -> CSR:
    """3D 7-point variable-coefficient diffusion on an m^3 grid, Dirichlet boundary.
    Face coefficient between cells a, b: harmonic mean 2 k_a k_b / (k_a + k_b); off-diagonal
    = -face coefficient; a boundary face adds the cell's own k to its diagonal.
    n = m^3, nnz = 7 m^3 - 6 m^2."""
    n = m ** 3
    kap = conductivity(m, seed)
    idx = np.arange(n, dtype=np.int64)
    z, y, x = idx // (m * m), (idx // m) % m, idx % m
    diag = np.zeros(n)
    rows, cols, vals = [], [], []
    for dz, dy, dx in ((-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 1), (0, 1, 0), (1, 0, 0)):
        ok = ((z + dz >= 0) & (z + dz < m) & (y + dy >= 0) & (y + dy < m) & (x + dx >= 0) & (x + dx < m))
        nb = idx[ok] + dz * m * m + dy * m + dx
        ka, kb = kap[idx[ok]], kap[nb]
        face = 2.0 * ka * kb / (ka + kb)
        rows.append(idx[ok])
        cols.append(nb)
        vals.append(-face)
        np.add.at(diag, idx[ok], face)
        diag[~ok] += kap[~ok]
    rows.append(idx)
    cols.append(idx)
    vals.append(diag)
    return _csr_from_entries(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def stencil27(m: int, seed: int, shift: float = 1e-2) -> CSR:
    """3D 27-point stencil on an m^3 grid: symmetric off-diagonals -U[0,1) drawn per undirected
    edge (stream 1001, indexed by min(i,j) * n + max(i,j)), diagonal = sum |off| + shift.
    n = m^3, nnz = (3m - 2)^3."""
    n = m ** 3
    idx = np.arange(n, dtype=np.int64)
    z, y, x = idx // (m * m), (idx // m) % m, idx % m
    diag = np.full(n, float(shift))
    rows, cols, vals = [], [], []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dz == dy == dx == 0:
                    continue
                ok = ((z + dz >= 0) & (z + dz < m) & (y + dy >= 0) & (y + dy < m) & (x + dx >= 0) & (x + dx < m))
                a = idx[ok]
                b = a + dz * m * m + dy * m + dx
                key = np.minimum(a, b) * n + np.maximum(a, b)
                off = -uniform01_at(seed, 1001, key)
                rows.append(a)
                cols.append(b)
                vals.append(off)
                np.add.at(diag, a, -off)
    rows.append(idx)
    cols.append(idx)
    vals.append(diag)
    return _csr_from_entries(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def dense_spd(n: int, seed: int, log10_lo: float = 0.0, log10_hi: float = 6.0) -> Dense:
    """Dense SPD A = Q diag(lambda) Q^T, Q from the QR factorisation of a seeded Gaussian matrix
    (Box-Muller on streams 2000/2001), lambda_i = 10^U[lo,hi] (stream 2002); symmetrised."""
    u1 = uniform01(seed, 2000, n * n)
    u2 = uniform01(seed, 2001, n * n)
    g = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    Q, _ = np.linalg.qr(g.reshape(n, n))
    lam = 10.0 ** (log10_lo + (log10_hi - log10_lo) * uniform01(seed, 2002, n))
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    return Dense(n, np.asfortranarray(A))


def dense_mtm(n: int, seed: int) -> Dense:
    """The paper's dense generator (Section 4): A = M^T M, M with i.i.d. Uniform(-1,1) entries
    (stream 2003)."""
    M = uniform_pm1(seed, 2003, n * n).reshape(n, n)
    A = M.T @ M
    A = 0.5 * (A + A.T)
    return Dense(n, np.asfortranarray(A))


def random_spd_csr(n: int, seed: int, density: float = 0.05, empty_rows_ok: bool = False) -> CSR:
    """Small random sparse SPD matrix (diagonally dominant) for kernel edge cases; draws from
    streams 3000-3002."""
    cnt = max(1, int(density * n * n))
    r = (uniform01(seed, 3000, cnt) * n).astype(np.int64)
    c = (uniform01(seed, 3001, cnt) * n).astype(np.int64)
    v = -uniform01(seed, 3002, cnt)
    keep = r != c
    r, c, v = r[keep], c[keep], v[keep]
    rows = np.concatenate([r, c])
    cols = np.concatenate([c, r])
    vals = np.concatenate([v, v])
    key = rows * n + cols
    uk, inv = np.unique(key, return_inverse=True)
    acc = np.zeros(len(uk))
    np.add.at(acc, inv, vals)
    rows, cols, vals = uk // n, uk % n, acc
    diag = np.ones(n)
    np.add.at(diag, rows, np.abs(vals))
    rows = np.concatenate([rows, np.arange(n)])
    cols = np.concatenate([cols, np.arange(n)])
    vals = np.concatenate([vals, diag])
    return _csr_from_entries(n, rows, cols, vals)


# Named workloads: the five configurations of the benchmark, by what they are.
POISSON2D_64 = dict(kind="poisson2d", m=64, s=4, precond=0, tol=1e-8)
DENSE_4096 = dict(kind="dense_spd", n=4096, s=(1, 2, 4, 8, 16, 32), precond=0, tol=1e-8)
DIFFUSION3D_128 = dict(kind="diffusion3d", m=128, s=(1, 4, 8, 16, 32), precond=1, tol=1e-8)
STENCIL27_96 = dict(kind="stencil27", m=96, s=16, precond=0, tol=1e-10)
