"""GPU parity of the FP64 finish: residuals and Rayleigh-quotient refinement.

rks_get_eigpairs returns the residuals ||A x - l x|| / (||A||_1 ||x||) and
rks_get_rayleigh the Rayleigh quotients x^H A x / x^H x of the returned Ritz
vectors (Sec. 4.1), both summed in FP64 on the device.  They are compared
element by element with the oracle's ``true_residuals`` of the same vectors
(pinned by closed forms in test_oracle_residuals.py), and the quotients also
with those of the oracle's own solve.
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


def K():
    from paper_2508_05400_gb300 import rks
    return rks


def _case(name):
    if name == "convdiff":
        return I.convdiff_2d(30, 30, 1.0, 20.0, 10.0), 6, 18, 64, "LR"
    if name == "planted":          # three complex pairs among the wanted (LM)
        from test_oracle_rks import _planted_spectrum_matrix
        Ad, _, _ = _planted_spectrum_matrix(150, 11)
        As = sp.csr_matrix(Ad)
        return I.CSR(150, As.indptr.astype(np.int32), As.indices.astype(np.int32), As.data), 5, 16, 64, "LM"
    from test_oracle_rks import _exterior_pair_matrix   # 0.9 +- 5i wanted second (LR)
    As = sp.csr_matrix(_exterior_pair_matrix())
    n = As.shape[0]
    return I.CSR(n, As.indptr.astype(np.int32), As.indices.astype(np.int32), As.data), 3, 12, 48, "LR"


@pytest.mark.parametrize("prec", ["df", "fp64", "mixed"])
@pytest.mark.parametrize("case", ["convdiff", "planted", "exterior_pair"])
def test_rayleigh_quotients_and_residuals_match_oracle(case, prec):
    A, k, p, d, which = _case(case)
    u1 = I.start_vector(A.n, 1)
    with K().Solver.from_csr(A, k, p, d, which=which, tol=1e-12, zeta=8, u1=u1, prec=prec) as s:
        info = s.solve(allow_noconv=False)
        lam, X, res = s.eigpairs()
        rq = s.rayleigh()
    assert rq.shape == lam.shape
    Z = K().unpack_eigvecs(lam, X)
    res_o, rq_o = R.true_residuals(A.to_scipy(), Z, lam)
    # the same FP64 sums of the same vectors, in another order: element by element
    err = np.abs(rq - rq_o) / np.abs(rq_o)
    assert err.max() <= 1e-13, (rq, rq_o)
    assert np.allclose(res, res_o, rtol=1e-6, atol=1e-16), (res, res_o)
    # a conjugate pair gets conjugate quotients
    for t in range(lam.size - 1):
        if lam[t].imag > 0:
            assert rq[t + 1] == np.conj(rq[t])
    # the quotient of a converged Ritz vector refines the Ritz value: both agree
    # with the oracle's solve to the accuracy the residual fixes
    ores = R.rks(A.to_scipy(), k, p, d, u1, zeta=8, seed=0, which=which, tol=1e-12)
    assert ores.converged and info["converged"] == 1
    kk = min(lam.size, ores.eigvals.size, k)
    assert np.max(np.abs(rq[:kk] - ores.lam_rq[:kk]) / np.abs(ores.lam_rq[:kk])) <= 1e-10
    assert np.max(np.abs(rq[:kk] - lam[:kk]) / np.abs(lam[:kk])) <= 1e-10


def test_rayleigh_before_solve_is_a_state_error():
    A, k, p, d, which = _case("convdiff")
    with K().Solver.from_csr(A, k, p, d, which=which, tol=1e-10) as s:
        with pytest.raises(K().RKSError) as e:
            s.rayleigh()
    assert e.value.code == -7
