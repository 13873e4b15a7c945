"""Pins of the synthetic operators against closed forms and structure."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2508_05400_gb300 import inputs as I


def _dense(A):
    return A.to_scipy().toarray()


def test_toeplitz_structure_and_spectrum():
    A = I.toeplitz_tridiag(7)
    D = _dense(A)
    assert D[3, 2] == -1.3 and D[3, 3] == 2.0 and D[3, 4] == -0.7
    assert A.nnz == 3 * 7 - 2
    s = np.sqrt(0.91)
    ev = np.sort(np.linalg.eigvalsh(_dense(I.toeplitz_tridiag(50, -s, 2.0, -s))))
    assert np.allclose(ev, np.sort(I.toeplitz_eigenvalues(50, -s, 2.0, -s)), atol=1e-13)
    ev = np.sort(np.linalg.eigvals(_dense(I.toeplitz_tridiag(20))).real)
    assert np.allclose(ev, np.sort(I.toeplitz_eigenvalues(20, -1.3, 2.0, -0.7)), rtol=1e-9)


def test_convdiff_2d_kronecker_closed_form():
    nx, ny = 9, 7
    A = I.convdiff_2d(nx, ny, 1.0, 20.0, 10.0)
    ev = np.linalg.eigvals(_dense(A))
    assert np.max(np.abs(ev.imag)) < 1e-8
    got = np.sort(ev.real)
    want = np.sort(I.convdiff_2d_eigenvalues(nx, ny, 1.0, 20.0, 10.0))
    assert np.allclose(got, want, rtol=1e-10)
    assert A.nnz == 5 * nx * ny - 2 * nx - 2 * ny


def test_convdiff_2d_stencil_rows():
    N = 6
    h = 1.0 / (N + 1)
    D = _dense(I.convdiff_2d(N, N, 2.0, 3.0, 5.0))
    p = 2 + N * 3                       # interior node
    assert np.isclose(D[p, p - 1], 2 / h**2 + 3 / h)   # west: diffusion + upwind
    assert np.isclose(D[p, p + 1], 2 / h**2)
    assert np.isclose(D[p, p - N], 2 / h**2 + 5 / h)   # south
    assert np.isclose(D[p, p + N], 2 / h**2)
    assert np.isclose(D[p, p], -(8 / h**2 + 8 / h))
    assert np.isclose(D.sum(axis=1)[p], 0.0, atol=1e-9)  # interior rows conserve
    # corner row: Dirichlet faces still enter the diagonal
    assert np.isclose(D[0, 0], -(8 / h**2 + 8 / h))
    assert np.count_nonzero(D[0]) == 3


def test_convdiff_variable_nu_is_symmetric_without_convection():
    nu = I.lognormal_field((5, 6), 1.0, 2)
    A = I.convdiff_2d(6, 5, nu, 0.0, 0.0).to_scipy()
    assert abs(A - A.T).max() < 1e-9 * abs(A).max()
    nu3 = I.lognormal_field((4, 3, 5), 1.0, 2)
    A3 = I.convdiff_3d(5, 3, 4, nu3, (0.0, 0.0, 0.0)).to_scipy()
    assert abs(A3 - A3.T).max() < 1e-9 * abs(A3).max()
    # negative definite (diffusion only)
    assert np.linalg.eigvalsh(A3.toarray()).max() < 0


def test_convdiff_3d_constant_nu_closed_form():
    nx, ny, nz = 5, 4, 3
    b = (10.0, 5.0, 2.0)
    A = I.convdiff_3d(nx, ny, nz, 1.0, b)
    ev = np.sort(np.linalg.eigvals(_dense(A)).real)
    m = [I.convdiff_1d_eigenvalues(N, 1.0, bb) for N, bb in zip((nx, ny, nz), b)]
    want = np.sort((m[0][None, None, :] + m[1][None, :, None] + m[2][:, None, None]).ravel())
    assert np.allclose(ev, want, rtol=1e-10)
    N = 6
    assert I.convdiff_3d(N, N, N, 1.0, b).nnz == 7 * N**3 - 6 * N**2


def test_norm1_and_dtype():
    A = I.convdiff_2d(8, 8, 1.0, 20.0, 10.0)
    assert np.isclose(I.norm1(A), abs(A.to_scipy()).sum(axis=0).max())
    A32 = I.convdiff_2d(8, 8, 1.0, 20.0, 10.0, dtype=np.float32)
    assert A32.vals.dtype == np.float32 and A32.rowptr.dtype == np.int32


def test_paper_tridiag_table1():
    A = _dense(I.paper_tridiag(50, "exponential", 0))
    t = np.linspace(2, 10, 50)
    assert np.allclose(np.diag(A), np.exp(t / 10))
    off = np.concatenate([np.diag(A, -1), np.diag(A, 1)])
    assert 0.002 < off.std() < 0.02
    for kind, f in (("logarithmic", np.log(t + 1)), ("harmonic", 1 + 1 / t**2), ("geometric", 0.99 ** t)):
        assert np.allclose(np.diag(_dense(I.paper_tridiag(50, kind, 0))), f)


def test_grf_statistics():
    g = I.gaussian_random_field(64, 64, 0.1, 3)
    assert g.shape == (64, 64)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1) < 1e-12
    # neighbouring nodes are strongly correlated at ell = 0.1, h = 1/65
    c = np.corrcoef(g[:, :-1].ravel(), g[:, 1:].ravel())[0, 1]
    assert c > 0.8


def test_uneven_batch_problems():
    # 256 problems: sides in [70, 450], log-uneven sizes, FP32 values, seeded
    sizes = []
    for i in (0, 1, 2, 255):
        P = I.uneven_convdiff2d_problem(i)
        a, b = (int(x) for x in P.name.split("_")[-1].split("x"))
        assert 70 <= a <= 450 and 70 <= b <= 450 and P.A.n == a * b
        assert P.A.vals.dtype == np.float32 and P.A.nnz == 5 * a * b - 2 * (a + b)
        assert (P.k, P.p, P.d, P.zeta, P.which) == (8, 24, 64, 8, "LR")
        sizes.append(P.A.n)
    again = I.uneven_convdiff2d_problem(2)
    assert np.array_equal(again.A.vals, I.uneven_convdiff2d_problem(2).A.vals)
    assert len(set(sizes)) == 4


def test_grf_family_member():
    P = I.grf_convdiff2d_problem(0, N=64)
    assert P.A.n == 64 * 64 and P.A.nnz == 5 * 64 * 64 - 4 * 64
    A = P.A.to_scipy()
    # the diffusive part is a weighted graph Laplacian: A + A^T has non-positive
    # row sums only through the convection and boundary terms (off-diagonals >= 0)
    off = A - sp.diags(A.diagonal())
    assert off.min() >= 0
    assert np.all(A.diagonal() < 0)
    assert I.grf_convdiff2d_problem(0, N=64).A.vals.tobytes() == P.A.vals.tobytes()
    assert I.grf_convdiff2d_problem(1, N=64).A.vals.tobytes() != P.A.vals.tobytes()
