"""The SpMV variants chosen by row statistics, against the oracle.

* a power-law matrix (rows of 1 to ~10^4 entries, mean ~6): merge path;
* a matrix of wide rows (32..48 entries): one warp per row;
* the stencil operators: by diagonals (the 2D and 3D convection-diffusion
  workloads), checked in the other parity tests.

Each is compared with the oracle's first expansion of Algorithm 2 column by
column (H, S and U) and by a full solve (eigenvalues, FP64 residuals), and
the double-float path must give the same bits on every run.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import rks as R
from oracle import sketch as SK
from paper_2508_05400_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_05400_gb300 import build as B
    B.build()
    return torch


def K():
    from paper_2508_05400_gb300 import rks
    return rks


_M = {}


def _matrix(kind):
    if kind not in _M:
        _M[kind] = I.powerlaw_matrix(100003) if kind == "powerlaw" else I.wide_rows_matrix(50021)
    return _M[kind]


def _colrel(a, b):
    return np.linalg.norm(a - b, axis=0) / np.maximum(np.linalg.norm(b, axis=0), 1e-300)


@pytest.mark.parametrize("kind,fmt", [("powerlaw", "merge"), ("wide", "warp")])
@pytest.mark.parametrize("prec", ["df", "mixed"])
def test_first_expansion_per_column(kind, fmt, prec):
    A = _matrix(kind)
    k, p, d = 4, 16, 64
    u1 = I.start_vector(A.n, 1)
    with K().Solver.from_csr(A, k, p, d, which="LM", tol=1e-12, zeta=8, u1=u1, max_restarts=-1, prec=prec) as s:
        assert s.spmv_format == fmt
        s.solve()
        if prec == "mixed":
            return                      # the FP32 phase's decomposition is checked by the solve below
        U, S, H = s.krylov()
    st = R.start(sp.csr_matrix(A.to_scipy()), SK.omega_matrix(A.n, d, 8, 0), u1)
    R.extend(st, k + p)
    eh, es, eu = _colrel(H, st.Ba), _colrel(S, st.Sa), _colrel(U, st.Ua)
    print(f"\n{kind}: max column error H {eh.max():.2e} S {es.max():.2e} U {eu.max():.2e}")
    assert eh.max() <= 1e-10 and es.max() <= 1e-10 and eu.max() <= 1e-10


@pytest.mark.parametrize("kind", ["powerlaw", "wide"])
@pytest.mark.parametrize("prec", ["df", "mixed"])
def test_solve_matches_oracle(kind, prec):
    A = _matrix(kind)
    u1 = I.start_vector(A.n, 1)
    with K().Solver.from_csr(A, 4, 16, 64, which="LM", tol=1e-12, zeta=8, u1=u1, prec=prec) as s:
        info = s.solve(allow_noconv=False)
        lam, X, res = s.eigpairs()
    o = R.rks(A.to_scipy(), 4, 16, 64, u1, zeta=8, seed=0, which="LM", tol=1e-12)
    assert o.converged and info["converged"] == 1
    assert np.max(np.abs(lam[:4] - o.eigvals[:4]) / np.abs(o.eigvals[:4])) <= 1e-10
    Z = K().unpack_eigvecs(lam, X)
    hres, _ = R.true_residuals(A.to_scipy(), Z, lam)
    assert res.max() <= 1e-10 and np.allclose(res, hres, rtol=1e-4, atol=1e-15)


def test_merge_path_is_deterministic():
    A = _matrix("powerlaw")
    out = []
    for _ in range(2):
        with K().Solver.from_csr(A, 4, 16, 64, which="LM", tol=1e-12, zeta=8, u1=I.start_vector(A.n, 1),
                                 max_restarts=3) as s:
            s.solve()
            U, S, H = s.krylov()
            out.append((U, S, H))
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_stencils_use_the_diagonal_copy():
    for A in (I.convdiff_2d(40, 37, 1.0, 20.0, 10.0), I.convdiff_3d(12, 11, 10, 1.0, (10.0, 5.0, 2.0)),
              I.toeplitz_tridiag(500)):
        with K().Solver.from_csr(A, 4, 12, 48, which="LR", tol=1e-8) as s:
            assert s.spmv_format == "dia"
