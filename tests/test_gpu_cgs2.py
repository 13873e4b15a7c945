"""The Krylov-Schur baseline with Euclidean CGS2 (the paper's KS-CGS2, Sec. 5).

Its oracle is the same FP64 oracle with Omega = I (d = n): the sketch is the
vector itself, the least squares is the Euclidean projection, so Algorithm 2
is Arnoldi and the restart is Krylov-Schur.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import rks as R
from paper_2508_05400_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _K():
    from paper_2508_05400_gb300 import rks
    return rks


def test_first_expansion_is_euclidean_arnoldi():
    A = I.convdiff_2d(40, 37, 1.0, 20.0, 10.0)
    u1 = I.start_vector(A.n, 1)
    k, p = 6, 18
    with _K().Solver.from_csr(A, k, p, 64, which="LR", tol=1e-8, u1=u1, max_restarts=-1, ortho="cgs2") as s:
        s.solve()
        U, _, H = s.krylov()
    st = R.start(sp.csr_matrix(A.to_scipy()), sp.identity(A.n, format="csr"), u1)
    R.extend(st, k + p)
    assert np.linalg.norm(H - st.Ba) <= 1e-12 * np.linalg.norm(st.Ba)
    assert np.linalg.norm(U - st.Ua) <= 1e-11 * np.linalg.norm(st.Ua)
    assert np.linalg.norm(U.T @ U - np.eye(U.shape[1])) < 1e-13
    m = k + p
    AU = A.to_scipy() @ U[:, :m]
    assert np.linalg.norm(AU - U @ H) < 1e-13 * np.linalg.norm(AU)


@pytest.mark.parametrize("keep", [0, 6])
def test_closed_form_spectrum(keep):
    N = 30
    A = I.convdiff_2d(N, N, 1.0, 20.0, 10.0)
    ex = np.sort(I.convdiff_2d_eigenvalues(N, N, 1.0, 20.0, 10.0))[::-1][:6]
    u1 = I.start_vector(A.n, 1)
    with _K().Solver.from_csr(A, 6, 18, 64, which="LR", tol=1e-13, u1=u1, ortho="cgs2", keep=keep) as s:
        info = s.solve(allow_noconv=False)
        lam, X, res = s.eigpairs()
    o = R.rks(A.to_scipy(), 6, 18, A.n, u1, Omega=sp.identity(A.n, format="csr"), which="LR", tol=1e-13,
              keep=keep)
    assert o.converged and info["converged"] == 1
    assert np.max(np.abs(lam[:6] - ex) / np.abs(ex)) < 1e-10
    assert np.max(np.abs(lam[:6] - o.eigvals[:6]) / np.abs(ex)) < 1e-10
    assert res.max() < 1e-13


def test_same_pairs_as_the_sketched_method():
    # rKS and KS-CGS2 find the same wanted eigenvalues at the benchmark's tolerance
    P = I.convdiff2d_problem(N=200)
    out = {}
    for ortho in ("sketch", "cgs2"):
        with _K().Solver.from_csr(P.A, P.k, P.p, P.d, which=P.which, zeta=P.zeta, u1=I.start_vector(P.A.n, 1),
                                  ortho=ortho, keep=P.k, **P.solver_opts()) as s:
            info = s.solve(allow_noconv=False)
            lam, X, res = s.eigpairs()
        assert res.max() <= P.tol
        out[ortho] = np.sort_complex(lam[:P.k])
    # a residual of tol * ||A||_1 fixes these (condition number ~ 1 to 10)
    # eigenvalues to about that absolute accuracy, not to the closed form's digits
    ex = np.sort(I.convdiff_2d_eigenvalues(200, 200, 1.0, 20.0, 10.0))[::-1][:P.k]
    bound = 50 * P.tol * I.norm1(P.A)
    for lam in out.values():
        assert np.max(np.abs(np.sort(lam.real)[::-1] - ex)) < bound


def test_cgs2_requires_the_df_path():
    A = I.convdiff_2d(20, 20, 1.0, 20.0, 10.0)
    for prec in ("fp64", "mixed"):
        with pytest.raises(_K().RKSError):
            _K().Solver.from_csr(A, 4, 12, 40, which="LR", tol=1e-8, ortho="cgs2", prec=prec)
