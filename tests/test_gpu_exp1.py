"""The paper's first experiment family on the GPU (Sec. 5.1, Table 1, Eq. 5.1).

Tridiagonal matrices with Table 1's diagonals (exponential, logarithmic,
harmonic, geometric over n equispaced points of [2, 10]) and N(0,1)/100
off-diagonals, LM and SM, k = 10, m = 40, d = 2m, zeta = 8, |b^T y|/|l| <=
1e-10: the GPU paths against the oracle's solve and against the dense
eigenvalues of the same matrix (n = 1000, brute force).
"""
import numpy as np
import pytest

from oracle import rks as R
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


@pytest.mark.parametrize("which", ["LM", "SM"])
@pytest.mark.parametrize("kind", ["exponential", "logarithmic", "harmonic", "geometric"])
@pytest.mark.parametrize("prec", ["df", "fp64"])
def test_table1_family_against_oracle_and_dense(kind, which, prec):
    from paper_2508_05400_gb300 import rks
    A = I.paper_tridiag(1000, kind)
    u1 = I.start_vector(A.n, 1)
    with rks.Solver.from_csr(A, 10, 30, 80, which=which, tol=1e-10, zeta=8, u1=u1, keep=10, maxit=2000,
                             prec=prec) as s:
        info = s.solve(allow_noconv=False)
        lam, X, res = s.eigpairs()
    o = R.rks(A.to_scipy(), 10, 30, 80, u1, zeta=8, seed=0, which=which, tol=1e-10, keep=10, maxit=2000)
    assert o.converged and info["converged"] == 1
    ev = np.linalg.eigvals(A.to_scipy().toarray())
    ev = ev[np.argsort(R.key(ev, which), kind="stable")][:10]
    lam = lam[:10]
    # the oracle's and the GPU's eigenvalues, and the dense ones (clustered
    # ends of the logarithmic diagonal fix them to ~1e-9)
    assert np.max(np.abs(lam - o.eigvals[:10]) / np.abs(o.eigvals[:10])) <= 1e-8
    assert max(np.min(np.abs(ev - l)) / abs(l) for l in lam) <= 1e-8
    assert res.max() <= 1e-9
