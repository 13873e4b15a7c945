"""The restart product on the tensor cores (tcgen05).

FP32 basis (split-BF16): compared with the FP64 product of the same FP32
inputs, the six leading split products are exact and accumulate in FP32, so
every entry is within a small multiple of 2^-24 of sum_l |u_l| |q_l|.
Double-float basis (exact 7-bit digit products): within a small multiple of
2^-46 of the row's largest entry times sum_l |q_l|.
"""
import numpy as np
import pytest

from paper_2508_05400_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _K():
    from paper_2508_05400_gb300 import rks
    return rks


@pytest.mark.parametrize("n,nin,nout", [(1000, 20, 8), (100003, 150, 50), (4099, 37, 64), (300, 256, 1),
                                        (128, 32, 16), (257, 33, 17)])
def test_product_matches_fp64(torch_cuda, n, nin, nout):
    rng = np.random.default_rng(n + nin)
    ldu = (n + 31) // 32 * 32
    U = np.zeros((nin, ldu), dtype=np.float32)          # column-major n x nin, leading dimension ldu
    U[:, :n] = rng.standard_normal((nin, n)).astype(np.float32) * np.exp(rng.standard_normal((nin, 1)))
    Q = rng.standard_normal((nin, nout))
    dU = torch_cuda.from_numpy(U).cuda()
    dO = torch_cuda.full((nout, ldu), 7.0, dtype=torch_cuda.float32, device="cuda")
    _K().basis_product_f32(dU, ldu, n, nin, Q, dO)
    got = dO.cpu().numpy()
    Ud = U[:, :n].T.astype(np.float64)
    ref = Ud @ Q
    scale = np.abs(Ud) @ np.abs(Q)
    err = np.abs(got[:, :n].T - ref) / scale
    assert err.max() < 2e-6, err.max()
    assert np.median(err) < 3e-7
    assert np.all(got[:, n:] == 7.0)                      # rows past n are not written


def test_product_in_place(torch_cuda):
    # the restart forms U_k = U Q' over the first columns of U itself
    n, nin, nout = 70001, 96, 40
    rng = np.random.default_rng(3)
    ldu = (n + 31) // 32 * 32
    U = np.zeros((nin, ldu), dtype=np.float32)
    U[:, :n] = rng.standard_normal((nin, n)).astype(np.float32)
    Q = rng.standard_normal((nin, nout))
    dU = torch_cuda.from_numpy(U.copy()).cuda()
    _K().basis_product_f32(dU, ldu, n, nin, Q, dU)
    got = dU.cpu().numpy()
    ref = U[:, :n].T.astype(np.float64) @ Q
    scale = np.abs(U[:, :n].T.astype(np.float64)) @ np.abs(Q)
    assert np.max(np.abs(got[:nout, :n].T - ref) / scale) < 2e-6
    assert np.array_equal(got[nout:, :n], U[nout:, :n])   # columns past nout untouched


def test_bad_sizes_rejected(torch_cuda):
    K = _K()
    dU = torch_cuda.zeros((8, 64), dtype=torch_cuda.float32, device="cuda")
    for nin, nout in [(257, 4), (8, 65)]:
        with pytest.raises(K.RKSError):
            K.basis_product_f32(dU, 64, 64, nin, np.ones((nin, nout)), dU)
    with pytest.raises(K.RKSError):
        K.basis_product_f32(dU, 64, 64, 0, np.ones((1, 4)), dU)


@pytest.mark.parametrize("n,nin,nout", [(1000, 20, 8), (100003, 150, 50), (4099, 37, 64), (300, 160, 1),
                                        (257, 33, 17), (128, 16, 16)])
def test_df_product_matches_fp64(torch_cuda, n, nin, nout):
    rng = np.random.default_rng(7 * n + nin)
    ldu = (n + 31) // 32 * 32
    U = np.zeros((nin, ldu))
    # rows of very different magnitude (each row has its own scale) and mixed column scales
    U[:, :n] = rng.standard_normal((nin, n)) * np.exp(3 * rng.standard_normal(n)) * np.exp(rng.standard_normal((nin, 1)))
    Q = rng.standard_normal((nin, nout)) * np.exp(2 * rng.standard_normal(nout))
    dU = torch_cuda.from_numpy(U).cuda()
    dO = torch_cuda.full((nout, ldu), 7.0, dtype=torch_cuda.float64, device="cuda")
    _K().basis_product_df(dU, ldu, n, nin, Q, dO)
    got = dO.cpu().numpy()
    Ud = U[:, :n].T
    ref = Ud @ Q
    bound = np.abs(Ud).max(axis=1)[:, None] * np.abs(Q).sum(axis=0)[None, :]
    err = np.abs(got[:, :n].T - ref) / bound
    assert err.max() < 2.0 ** -44, err.max()
    rel = np.abs(got[:, :n].T - ref) / (np.abs(Ud) @ np.abs(Q))
    assert np.median(rel) < 1e-13
    assert np.all(got[:, n:] == 7.0)


def test_solver_same_pairs_with_and_without_tensor_core_restart():
    # the double-float solve with the exact-digit restart and with the SIMT one
    P = I.convdiff2d_problem(N=150)
    out = {}
    for tc in (True, False):
        with _K().Solver.from_csr(P.A, P.k, P.p, P.d, which=P.which, zeta=P.zeta, u1=I.start_vector(P.A.n, 1),
                                  keep=P.k, tc_restart=tc, **P.solver_opts()) as s:
            s.solve(allow_noconv=False)
            lam, X, res = s.eigpairs()
        assert res.max() <= P.tol
        out[tc] = np.sort(lam.real[:P.k])
    assert np.max(np.abs(out[True] - out[False])) < 50 * P.tol * I.norm1(P.A)
