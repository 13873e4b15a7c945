"""The mixed path's hand-over from the FP32 phase to double-float.

The double-float restarts continue from the FP32 Krylov-Schur decomposition
A U = U T + u b^T once its relation error (the FP32 rounding of the stored
vectors) has been corrected below what the target asks.  Checked: the hand-over
happens and keeps the FP32 phase's progress (the first double-float restart's
estimate stays at the FP32 level instead of that of a fresh start), the
results meet the target in FP64 on the host and agree with the double-float
path and the FP64 oracle, and a target the corrected relation cannot meet
falls back to a double-float solve from the sum of the FP32 Schur vectors, as
does the truncation of Algorithm 1 (keep = 0).
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
    return torch


def K():
    from paper_2508_05400_gb300 import rks
    return rks


def _solve(P, prec, **kw):
    u1 = I.start_vector(P.A.n, 1)
    opts = dict(P.solver_opts())
    opts.update(kw)
    with K().Solver.from_csr(P.A, P.k, P.p, P.d, which=P.which, zeta=P.zeta, u1=u1, prec=prec, **opts) as s:
        info = s.solve(allow_noconv=False)
        st = s.stats()
        hist, _ = s.history()
        lam, X, res = s.eigpairs()
        nrm = s.norm1
    return info, st, hist, lam, X, res, nrm


def test_mixed_continues_from_the_fp32_decomposition():
    # the 160^3 workload's structure at 48^3 (n = 110 592), thick restart
    P = I.convdiff3d_problem(N=48, k=16, p=48, d=192)
    info, st, hist, lam, X, res, nrm = _solve(P, "mixed", keep=16)
    assert st["mixed_phase2"] == 1                      # continued from the hand-over
    o = P.solver_opts()
    assert 0.0 < st["handover_rel"] <= o["verify"] - o["tol"]
    r = st["fp32_restarts"]
    assert 0 < r < info["restarts"] == len(hist)
    # the FP32 phase ended above the target; the first double-float restart
    # starts from its accuracy (a fresh start is back near 1e-2)
    assert hist[r - 1] > o["tol"]
    assert hist[r] <= 10.0 * hist[r - 1]
    # FP64 residuals recomputed on the host
    A = P.A.to_scipy()
    Z = K().unpack_eigvecs(lam, X)
    hres, _ = R.true_residuals(A, Z, lam)
    assert hres.max() <= P.tol and res.max() <= P.tol
    # the same eigenvalues as the double-float path (which the FP64 oracle
    # pins elsewhere), to what residuals of 1e-8 ||A||_1 fix of these
    # well-separated rightmost ones
    info2, st2, _, lam2, _, res2, _ = _solve(P, "df", keep=16)
    assert st2["mixed_phase2"] == 0 and res2.max() <= P.tol
    a, b = np.sort(lam.real)[::-1][:4], np.sort(lam2.real)[::-1][:4]
    assert np.allclose(a, b, rtol=1e-5)


def test_mixed_with_the_truncation_of_algorithm_1_starts_phase_2_afresh():
    # keep = 0: the FP32 phase locks and the double-float phase starts from
    # the sum of the FP32 Schur vectors; the result matches the FP64 oracle
    P = I.convdiff3d_problem(N=20, k=8, p=24, d=96)
    info, st, hist, lam, X, res, nrm = _solve(P, "mixed")
    assert st["mixed_phase2"] == 2 and st["handover_rel"] == 0.0
    assert res.max() <= P.tol
    o = P.solver_opts()
    ores = R.rks(P.A.to_scipy(), P.k, P.p, P.d, I.start_vector(P.A.n, 1), zeta=P.zeta, seed=0, which=P.which,
                 tol=o["tol"], eta_lock=o["eta_lock"], conv="norm1")
    assert ores.converged
    assert np.allclose(np.sort(lam.real)[::-1][:4], np.sort(ores.eigvals.real)[::-1][:4], rtol=1e-4)


def test_mixed_falls_back_when_the_target_is_below_the_corrected_relation():
    # |b^T y| / |lambda| <= 1e-13: far below the FP32 relation error even
    # after the correction, so phase 2 restarts from the sum of the FP32
    # Schur vectors, and the result still meets the target
    A = I.convdiff_2d(30, 30, 1.0, 20.0, 10.0)
    u1 = I.start_vector(A.n, 1)
    with K().Solver.from_csr(A, 6, 18, 64, which="LR", tol=1e-13, zeta=8, u1=u1, prec="mixed", keep=6) as s:
        info = s.solve(allow_noconv=False)
        st = s.stats()
        lam, X, res = s.eigpairs()
        est = s.estimates()
    assert st["mixed_phase2"] == 2
    assert st["handover_rel"] > 1e-13
    assert info["converged"] == 1 and est.max() <= 1e-13
    ex = np.sort(I.convdiff_2d_eigenvalues(30, 30, 1.0, 20.0, 10.0))[::-1]
    assert np.max(np.abs(lam[:6] - ex[:6]) / np.abs(ex[:6])) <= 1e-10
