"""Seeded synthetic inputs for randomized Krylov-Schur (rKS) runs.

This module holds input data only: sparse test operators, coefficient fields and
random start vectors. It contains none of the eigensolver's arithmetic, and it
is the one module that both the CUDA path's tests/benchmark and the CPU oracle
read, so that both see identical inputs.

Operators:

* ``toeplitz_tridiag``: a tridiagonal Toeplitz matrix (sub, diag, sup), whose
  spectrum is diag + 2*sqrt(sub*sup)*cos(j*pi/(n+1)), j = 1..n.
* ``convdiff_2d`` / ``convdiff_3d``: the operator
  L u = div(nu grad u) - b . grad u on the unit square / cube, Dirichlet zero,
  first-order upwind convection (b >= 0, backward differences), face
  diffusivity = harmonic mean of the two node values (node value on a boundary
  face), unknowns numbered lexicographically with x fastest.  With constant nu
  the 2D operator is a Kronecker sum of two 1D tridiagonal Toeplitz operators,
  so its spectrum is known in closed form (``convdiff_2d_eigenvalues``).
* ``paper_tridiag``: the synthetic non-symmetric tridiagonal matrices of the
  paper's first experiment (Sec. 5.1, Table 1, Eq. 5.1): a diagonal from one of
  four spectra over n equispaced points in [2, 10] and N(0,1)/100 off-diagonals.

Random numbers: every draw comes from the SplitMix64 generator (Steele, Lea &
Flood, OOPSLA 2014): state += 0x9E3779B97F4A7C15, output = mix(state).  It is
counter based, so draw r of a stream with seed s is mix(s + (r+1)*gamma).
Uniforms take the top 53 bits; normals use the Box-Muller cosine branch on
draws (2i, 2i+1).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64_draws(seed: int, start: int, count: int) -> np.ndarray:
    """Draws start .. start+count-1 of the SplitMix64 stream seeded with ``seed``."""
    r = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + r * GAMMA
    return splitmix64_mix(state)


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each draw."""
    h = splitmix64_draws(seed, start, count)
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, count: int) -> np.ndarray:
    """N(0,1) samples: Box-Muller (cosine branch) on draws 2i and 2i+1."""
    u = uniform01(seed, 2 * count)
    u1 = u[0::2]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


def start_vector(n: int, seed: int = 1) -> np.ndarray:
    """The rKS start vector: n entries N(0,1) from ``seed``."""
    return normal(seed, n)


@dataclass
class CSR:
    """A square sparse matrix in CSR form (int32 indices)."""
    n: int
    rowptr: np.ndarray   # int32 (n+1)
    colind: np.ndarray   # int32 (nnz)
    vals: np.ndarray     # float64 or float32 (nnz)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self, dtype=np.float64):
        import scipy.sparse as sp
        return sp.csr_matrix((self.vals.astype(dtype), self.colind, self.rowptr),
                             shape=(self.n, self.n))

    def astype(self, dtype) -> "CSR":
        return CSR(self.n, self.rowptr, self.colind, self.vals.astype(dtype))


def _from_triplets(n, rows, cols, vals, dtype) -> CSR:
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSR(n, rowptr.astype(np.int32), cols.astype(np.int32),
               vals.astype(dtype))


def toeplitz_tridiag(n: int, sub: float = -1.3, diag: float = 2.0,
                     sup: float = -0.7, dtype=np.float64) -> CSR:
    """Tridiagonal Toeplitz matrix with A[i,i-1]=sub, A[i,i]=diag, A[i,i+1]=sup."""
    i = np.arange(n)
    rows = np.concatenate([i[1:], i, i[:-1]])
    cols = np.concatenate([i[:-1], i, i[1:]])
    vals = np.concatenate([np.full(n - 1, sub), np.full(n, diag), np.full(n - 1, sup)])
    return _from_triplets(n, rows, cols, vals, dtype)


def toeplitz_eigenvalues(n: int, sub: float, diag: float, sup: float) -> np.ndarray:
    """Closed-form spectrum of ``toeplitz_tridiag`` (requires sub*sup > 0)."""
    j = np.arange(1, n + 1)
    return diag + 2.0 * np.sqrt(sub * sup) * np.cos(j * np.pi / (n + 1))


def _harm(a, b):
    return 2.0 * a * b / (a + b)


def convdiff_2d(nx: int, ny: int, nu=1.0, bx: float = 0.0, by: float = 0.0,
                dtype=np.float64) -> CSR:
    """5-point upwind convection-diffusion operator on an nx-by-ny interior grid.

    ``nu`` is a scalar or an (ny, nx) array of node diffusivities.  The grid
    spacing is hx = 1/(nx+1), hy = 1/(ny+1).  Row p = ix + nx*iy.
    """
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    nu = np.broadcast_to(np.asarray(nu, dtype=np.float64), (ny, nx))
    n = nx * ny
    # face diffusivities (node value on boundary faces)
    nw = nu.copy(); nw[:, 1:] = _harm(nu[:, 1:], nu[:, :-1])
    ne = nu.copy(); ne[:, :-1] = _harm(nu[:, :-1], nu[:, 1:])
    ns = nu.copy(); ns[1:, :] = _harm(nu[1:, :], nu[:-1, :])
    nn = nu.copy(); nn[:-1, :] = _harm(nu[:-1, :], nu[1:, :])
    cw = nw / hx**2 + bx / hx
    ce = ne / hx**2
    cs = ns / hy**2 + by / hy
    cn = nn / hy**2
    cp = -(nw + ne) / hx**2 - (ns + nn) / hy**2 - bx / hx - by / hy
    iy, ix = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    p = ix + nx * iy
    parts_r, parts_c, parts_v = [p.ravel()], [p.ravel()], [cp.ravel()]
    for mask, off, coef in ((ix > 0, -1, cw), (ix < nx - 1, 1, ce),
                            (iy > 0, -nx, cs), (iy < ny - 1, nx, cn)):
        parts_r.append(p[mask]); parts_c.append(p[mask] + off); parts_v.append(coef[mask])
    return _from_triplets(n, np.concatenate(parts_r), np.concatenate(parts_c),
                          np.concatenate(parts_v), dtype)


def convdiff_1d_eigenvalues(N: int, nu: float, b: float) -> np.ndarray:
    """Spectrum of the 1D factor of ``convdiff_2d`` with constant nu (N nodes)."""
    h = 1.0 / (N + 1)
    lo, up, dg = nu / h**2 + b / h, nu / h**2, -(2 * nu / h**2 + b / h)
    return toeplitz_eigenvalues(N, lo, dg, up)


def convdiff_2d_eigenvalues(nx: int, ny: int, nu: float, bx: float, by: float) -> np.ndarray:
    """Closed-form spectrum (Kronecker sum) of ``convdiff_2d`` with constant nu."""
    mx = convdiff_1d_eigenvalues(nx, nu, bx)
    my = convdiff_1d_eigenvalues(ny, nu, by)
    return (mx[None, :] + my[:, None]).ravel()


def convdiff_3d(nx: int, ny: int, nz: int, nu=1.0, b=(0.0, 0.0, 0.0),
                dtype=np.float64) -> CSR:
    """7-point upwind convection-diffusion operator; row p = ix + nx*(iy + ny*iz).

    ``nu`` is a scalar or an (nz, ny, nx) array of node diffusivities.
    """
    h = (1.0 / (nx + 1), 1.0 / (ny + 1), 1.0 / (nz + 1))
    nu = np.broadcast_to(np.asarray(nu, dtype=np.float64), (nz, ny, nx))
    n = nx * ny * nz
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    p = ix + nx * (iy + ny * iz)
    strides = (1, nx, nx * ny)
    idx = (ix, iy, iz)
    sizes = (nx, ny, nz)
    diag = np.zeros_like(nu)
    parts_r, parts_c, parts_v = [], [], []
    for a in range(3):
        ax = 2 - a  # array axis of direction a (arrays are indexed [z, y, x])
        lo = nu.copy(); hi = nu.copy()
        sl_hi = [slice(None)] * 3; sl_lo = [slice(None)] * 3
        sl_hi[ax] = slice(1, None); sl_lo[ax] = slice(None, -1)
        lo[tuple(sl_hi)] = _harm(nu[tuple(sl_hi)], nu[tuple(sl_lo)])
        hi[tuple(sl_lo)] = _harm(nu[tuple(sl_lo)], nu[tuple(sl_hi)])
        c_lo = lo / h[a]**2 + b[a] / h[a]
        c_hi = hi / h[a]**2
        diag -= (lo + hi) / h[a]**2 + b[a] / h[a]
        m_lo = idx[a] > 0
        m_hi = idx[a] < sizes[a] - 1
        parts_r += [p[m_lo], p[m_hi]]
        parts_c += [p[m_lo] - strides[a], p[m_hi] + strides[a]]
        parts_v += [c_lo[m_lo], c_hi[m_hi]]
    parts_r.append(p.ravel()); parts_c.append(p.ravel()); parts_v.append(diag.ravel())
    return _from_triplets(n, np.concatenate(parts_r), np.concatenate(parts_c),
                          np.concatenate(parts_v), dtype)


def lognormal_field(shape, sigma: float = 1.0, seed: int = 2) -> np.ndarray:
    """exp(sigma*g) with g i.i.d. N(0,1) per node, in C order of ``shape``."""
    count = int(np.prod(shape))
    return np.exp(sigma * normal(seed, count)).reshape(shape)


def gaussian_random_field(nx: int, ny: int, ell: float = 0.1, seed: int = 0) -> np.ndarray:
    """Unit-variance Gaussian random field with squared-exponential covariance.

    Spectral synthesis on a periodic grid twice the size of the unit square
    (the [0,1]^2 corner is returned), correlation length ``ell``.
    """
    Mx, My = 2 * (nx + 1), 2 * (ny + 1)
    kx = np.fft.fftfreq(Mx, d=1.0 / (nx + 1))
    ky = np.fft.fftfreq(My, d=1.0 / (ny + 1))
    K2 = (2 * np.pi) ** 2 * (kx[None, :] ** 2 + ky[:, None] ** 2)
    spec = np.exp(-K2 * ell ** 2 / 4.0)
    g = normal(seed, 2 * Mx * My).reshape(2, My, Mx)
    f = np.fft.ifft2(np.sqrt(spec) * (g[0] + 1j * g[1])).real
    f = f[1:ny + 1, 1:nx + 1]
    return (f - f.mean()) / f.std()


def paper_tridiag(n: int, kind: str = "exponential", seed: int = 0,
                  dtype=np.float64) -> CSR:
    """Synthetic tridiagonal test matrix of the paper's first experiment.

    Diagonal (Table 1) over t = n equispaced points in [2, 10]:
    exponential exp(t/10), logarithmic log(t+1), harmonic 1 + 1/t^2,
    geometric 0.99^t.  Off-diagonals g/100 with g ~ N(0,1) (Eq. 5.1).
    """
    t = np.linspace(2.0, 10.0, n)
    diag = {"exponential": np.exp(t / 10.0), "logarithmic": np.log(t + 1.0),
            "harmonic": 1.0 + 1.0 / t**2, "geometric": 0.99 ** t}[kind]
    g = normal(seed, 2 * (n - 1)) / 100.0
    i = np.arange(n)
    rows = np.concatenate([i[1:], i, i[:-1]])
    cols = np.concatenate([i[:-1], i, i[1:]])
    vals = np.concatenate([g[: n - 1], diag, g[n - 1:]])
    return _from_triplets(n, rows, cols, vals, dtype)


def norm1(A: CSR) -> float:
    """Max column sum of |A| (the 1-norm used to scale residuals)."""
    s = np.zeros(A.n)
    np.add.at(s, A.colind, np.abs(A.vals.astype(np.float64)))
    return float(s.max())


# ---------------------------------------------------------------------------
# Named workloads (sizes follow the benchmark definitions)
# ---------------------------------------------------------------------------

@dataclass
class Problem:
    name: str
    A: CSR
    k: int
    p: int
    d: int
    zeta: int
    which: str
    tol: float
    omega_seed: int = 0
    u1_seed: int = 1
    lock: bool = True
    conv: str = "eig"

    @property
    def m(self) -> int:
        return self.k + self.p

    def solver_opts(self) -> dict:
        """Solver settings that meet ``tol`` on the stated residual scale.

        With conv="norm1" the target is ||A x - l x|| / (||A||_1 ||x||) <= tol.
        The estimate |b^T y| / ||A||_1 differs from it by the embedding
        distortion sqrt((1+eps)/(1-eps)) (Sec. 4.1) and a locked pair by a
        further sqrt(q) (Eq. 4.21), so the iteration runs at tol/4, locks at
        tol/8, and the FP64 residuals are verified at tol.
        """
        if self.conv == "norm1":
            return dict(tol=self.tol / 4, eta_lock=self.tol / 8, conv="norm1", verify=self.tol)
        return dict(tol=self.tol, conv="eig")


def toeplitz_problem(n: int = 2000) -> Problem:
    """Non-symmetric Toeplitz (2, -1.3, -0.7), LM, k=10, p=30, d=80, zeta=4, tol 1e-10."""
    return Problem(f"toeplitz{n}", toeplitz_tridiag(n), 10, 30, 80, 4, "LM", 1e-10)


def convdiff2d_problem(N: int = 1000, k: int = 20, p: int = 60, d: int = 320,
                       tol: float = 1e-8) -> Problem:
    """2D convection-diffusion N x N, nu=1, b=(20,10), FP64, LR, zeta=8, locking.

    The tolerance applies to ||A x - l x|| / (||A||_1 ||x||).
    """
    return Problem(f"convdiff2d_{N}", convdiff_2d(N, N, 1.0, 20.0, 10.0), k, p, d, 8, "LR", tol,
                   conv="norm1")


def convdiff3d_problem(N: int = 160, k: int = 50, p: int = 100, d: int = 600,
                       tol: float = 1e-8, field_seed: int = 2) -> Problem:
    """3D convection-diffusion N^3, log-normal nu (sigma=1), b=(10,5,2), FP32 values, LR."""
    nu = lognormal_field((N, N, N), 1.0, field_seed)
    A = convdiff_3d(N, N, N, nu, (10.0, 5.0, 2.0), dtype=np.float32)
    return Problem(f"convdiff3d_{N}", A, k, p, d, 8, "LR", tol, conv="norm1")


def uneven_convdiff2d_problem(i: int, seed0: int = 1000, k: int = 8, p: int = 24, d: int = 64,
                              tol: float = 1e-8) -> Problem:
    """Problem i of the batch of uneven 2D convection-diffusion operators.

    Seed seed0 + i draws (from SplitMix64 uniforms, in this order) the grid
    sides a, b ~ U{70..450}, the convection (bx, by) ~ U[0, 30]^2, then the
    log-normal diffusivity exp(g), g ~ N(0,1) per node; FP32 values, LR.
    """
    s = seed0 + i
    u = uniform01(s, 4)
    a, b = 70 + int(u[0] * 381), 70 + int(u[1] * 381)
    bx, by = 30.0 * u[2], 30.0 * u[3]
    nu = lognormal_field((b, a), 1.0, s + 7919)
    A = convdiff_2d(a, b, nu, bx, by, dtype=np.float32)
    return Problem(f"uneven2d_{i}_{a}x{b}", A, k, p, d, 8, "LR", tol, conv="norm1")


def grf_convdiff2d_problem(i: int, seed0: int = 20000, N: int = 512, k: int = 16, p: int = 48,
                           d: int = 192, tol: float = 1e-8) -> Problem:
    """Member i of the parametric 2D family on an N x N grid: seed seed0 + i
    draws (bx, by) ~ U[0, 50]^2 and the diffusivity exp(GRF), correlation
    length 0.1 (held-out members use seed0 = 20000, training ones 10000)."""
    s = seed0 + i
    u = uniform01(s, 2)
    nu = np.exp(gaussian_random_field(N, N, 0.1, s + 7919))
    A = convdiff_2d(N, N, nu, 50.0 * u[0], 50.0 * u[1])
    return Problem(f"grf2d_{N}_{s}", A, k, p, d, 8, "LR", tol, conv="norm1")


def grf_member_fields(i: int, seed0: int = 20000, N: int = 512) -> np.ndarray:
    """Coefficient planes of member i of the parametric 2D family (the
    operator of ``grf_convdiff2d_problem(i, seed0, N)``): log nu, bx / 50 and
    by / 50 on the N x N grid, float32, shape (3, N, N), row y, column x (the
    solver's numbering, x fastest, after flattening)."""
    s = seed0 + i
    u = uniform01(s, 2)
    g = gaussian_random_field(N, N, 0.1, s + 7919)
    out = np.empty((3, N, N), dtype=np.float32)
    out[0] = g
    out[1] = u[0]
    out[2] = u[1]
    return out


def powerlaw_matrix(n: int, seed: int = 0, max_len: int = 10000, alpha: float = 1.2,
                    lead=(10.0, 9.0, 8.0, 7.0, 6.0, 5.5, 5.0, 4.5)) -> CSR:
    """Sparse non-symmetric matrix whose row lengths follow a power law (rows
    of 1 to ``max_len`` entries, P(L >= l) ~ l^-alpha), like the irregular
    matrices of large sparse collections.  Row i: L_i = min(max_len,
    floor(u^(-1/alpha))) entries at distinct random columns (SplitMix64
    uniforms of ``seed``), values N(0,1) * 0.5 / sqrt(L_i), plus a diagonal:
    ``lead`` for the first rows (well separated eigenvalues of largest
    modulus), then values in [0, 2)."""
    u = uniform01(seed, n)
    L = np.minimum(max_len, np.floor(np.maximum(u, 1e-300) ** (-1.0 / alpha))).astype(np.int64)
    L = np.maximum(L, 1)
    tot = int(L.sum())
    uc = uniform01(seed + 1, tot)
    g = normal(seed + 2, tot)
    rows = np.repeat(np.arange(n, dtype=np.int64), L)
    cols = np.minimum((uc * n).astype(np.int64), n - 1)
    vals = g * (0.5 / np.sqrt(L[rows]))
    keep = cols != rows                      # the diagonal is set below
    rows, cols, vals = rows[keep], cols[keep], vals[keep]
    key = rows * n + cols                    # drop repeated (row, column) pairs
    _, first = np.unique(key, return_index=True)
    rows, cols, vals = rows[first], cols[first], vals[first]
    diag = 2.0 * uniform01(seed + 3, n)
    diag[:len(lead)] = lead
    rows = np.concatenate([rows, np.arange(n)])
    cols = np.concatenate([cols, np.arange(n)])
    vals = np.concatenate([vals, diag])
    return _from_triplets(n, rows, cols, vals, np.float64)


def wide_rows_matrix(n: int, seed: int = 0, lo: int = 32, hi: int = 48,
                     lead=(10.0, 9.0, 8.0, 7.0, 6.0, 5.5, 5.0, 4.5)) -> CSR:
    """Sparse non-symmetric matrix with rows of lo..hi entries at random
    columns (values N(0,1) * 0.5 / sqrt(L_i)) plus the diagonal of
    ``powerlaw_matrix``."""
    u = uniform01(seed, n)
    L = (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)
    tot = int(L.sum())
    uc = uniform01(seed + 1, tot)
    g = normal(seed + 2, tot)
    rows = np.repeat(np.arange(n, dtype=np.int64), L)
    cols = np.minimum((uc * n).astype(np.int64), n - 1)
    vals = g * (0.5 / np.sqrt(L[rows]))
    keep = cols != rows
    rows, cols, vals = rows[keep], cols[keep], vals[keep]
    key = rows * n + cols
    _, first = np.unique(key, return_index=True)
    rows, cols, vals = rows[first], cols[first], vals[first]
    diag = 2.0 * uniform01(seed + 3, n)
    diag[:len(lead)] = lead
    rows = np.concatenate([rows, np.arange(n)])
    cols = np.concatenate([cols, np.arange(n)])
    vals = np.concatenate([vals, diag])
    return _from_triplets(n, rows, cols, vals, np.float64)
