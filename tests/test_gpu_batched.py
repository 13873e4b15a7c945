"""Batched solve of independent problems (rks_create_batched / rks_solve_batched).

Members of the batch of uneven 2D operators are solved concurrently; each
problem's results must be the bits of its solve alone (the kernels are
deterministic) and meet the residual tolerance.
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


def _K():
    from paper_2508_05400_gb300 import rks
    return rks


def _kw(P):
    return dict(which=P.which, zeta=P.zeta, keep=P.k, maxit=3000, **P.solver_opts())


@pytest.mark.parametrize("prec", ["df", "mixed"])
def test_batched_equals_single_solves(prec):
    probs = [I.uneven_convdiff2d_problem(i) for i in range(10)]
    P0 = probs[0]
    with _K().Batch([P.A for P in probs], P0.k, P0.p, P0.d, nthreads=5, prec=prec, **_kw(P0)) as b:
        infos = b.solve(nthreads=5, allow_noconv=False)
        got = [b.member(i).eigpairs() for i in range(len(probs))]
        hist = [b.member(i).history()[0] for i in range(len(probs))]
    for i, P in enumerate(probs):
        with _K().Solver.from_csr(P.A, P.k, P.p, P.d, prec=prec, **_kw(P)) as s:
            info = s.solve(allow_noconv=False)
            lam, X, res = s.eigpairs()
            h, _ = s.history()
        assert infos[i]["status"] == "RKS_OK"
        assert (infos[i]["restarts"], infos[i]["nmatvec"]) == (info["restarts"], info["nmatvec"])
        assert np.array_equal(got[i][0], lam) and np.array_equal(got[i][1], X) and np.array_equal(got[i][2], res)
        assert np.array_equal(hist[i], h)
        assert res.max() <= P.tol


def test_batched_rejects_a_bad_member():
    good = I.uneven_convdiff2d_problem(0).A
    tiny = I.convdiff_2d(4, 4, 1.0, 1.0, 1.0, dtype=np.float32)   # n = 16 < k + p + 1
    with pytest.raises(_K().RKSError):
        _K().Batch([good, tiny], 8, 24, 64, which="LR", tol=1e-8)
