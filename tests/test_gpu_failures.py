"""Failure paths of rks_solve on the GPU, made on the host or by a wait that
nothing completes (nothing faults or hangs the device).

* RKS_ENOCONV: the restart limit is reached; the results are partial and valid.
* RKS_ETIMEOUT: the test hook opts.debug_stall makes every grid barrier of the
  cooperative least-squares kernel wait for one CTA more than the grid holds,
  so each wait runs out its short limit; the kernel records the timeout and
  finishes, the host reports it, and the device (and a new context) keeps
  working.
* RKS_EINVAL: matrix values outside the FP32 exponent range under the
  double-float and mixed paths.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("prec", ["df", "fp64", "mixed"])
def test_restart_limit_reports_enoconv_with_valid_results(prec):
    A = I.convdiff_2d(40, 40, 1.0, 20.0, 10.0)
    with K().Solver.from_csr(A, 6, 18, 64, which="LR", tol=1e-14, u1=I.start_vector(A.n, 1), maxit=1,
                             prec=prec) as s:
        with pytest.raises(K().RKSError) as e:
            s.solve(allow_noconv=False)
        assert e.value.code == K().RKS_ENOCONV
        lam, X, res = s.eigpairs()
        T, U, b = s.schur()
    assert np.all(np.isfinite(lam)) and np.all(np.isfinite(res)) and np.all(np.isfinite(X))
    # still an rKS decomposition A U = U T + u b^T: A U - U T is rank one along b
    AU = A.to_scipy() @ U
    r = AU - U @ T
    Pb = np.eye(b.size) - np.outer(b, b) / (b @ b)
    assert np.linalg.norm(r @ Pb) <= 1e-10 * np.linalg.norm(AU)


def test_grid_barrier_timeout_reports_etimeout_and_device_stays_usable():
    A = I.convdiff_2d(60, 60, 1.0, 20.0, 10.0)
    u1 = I.start_vector(A.n, 1)
    with K().Solver.from_csr(A, 6, 18, 64, which="LR", tol=1e-12, u1=u1, debug_stall=1) as s:
        with pytest.raises(K().RKSError) as e:
            s.solve()
        assert e.value.code == -9          # RKS_ETIMEOUT
    # the same problem on a fresh context converges as usual
    with K().Solver.from_csr(A, 6, 18, 64, which="LR", tol=1e-12, u1=u1) as s:
        info = s.solve(allow_noconv=False)
        _, _, res = s.eigpairs(want_vectors=False)
    assert info["converged"] == 1 and res.max() <= 1e-10


def test_debug_stall_values_are_validated():
    A = I.convdiff_2d(10, 10, 1.0, 1.0, 1.0)
    with pytest.raises(K().RKSError) as e:
        K().Solver.from_csr(A, 2, 6, 16, which="LR", debug_stall=2)
    assert e.value.code == K().RKS_EINVAL


@pytest.mark.parametrize("bad", [1e39, -5e38, 1e-39])
@pytest.mark.parametrize("prec", ["df", "mixed"])
def test_values_outside_fp32_range_are_rejected(prec, bad):
    A = I.convdiff_2d(12, 12, 1.0, 1.0, 1.0)
    v = A.vals.copy()
    v[7] = bad
    with pytest.raises(K().RKSError) as e:
        K().Solver(A.n, A.rowptr, A.colind, v, 3, 8, 24, which="LR", prec=prec)
    assert e.value.code == K().RKS_EINVAL
    # the FP64 path takes them
    with K().Solver(A.n, A.rowptr, A.colind, v, 3, 8, 24, which="LR", prec="fp64"):
        pass
