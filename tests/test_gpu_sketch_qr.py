"""GPU parity of the randomized QR of a block (rks_sketch_qr) against the oracle.

The four processes of Sec. 2 (randomized Gram-Schmidt, sketch and whiten,
randomized Cholesky QR, randomized Householder QR) on the double-float device
path, compared with the FP64
oracle on the same Omega (the SplitMix64 sparse-sign hash, bit-exact on both
sides) and checked for the properties that define them: K = Q R with R upper
triangular and a positive diagonal, Omega Q orthonormal (RGS, whitening) or
Q^T Q = I (RCholQR).  Double-float products carry ~2^-48 relative error, so
the tolerances are those of the FP64 oracle times a small factor, scaled by
the condition number of K where the algorithm's own error is.
"""
import numpy as np
import pytest

from oracle import sketch_qr as SQ
from oracle.sketch import omega_matrix

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


def _graded_block(n, s, cond, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, s)))
    V, _ = np.linalg.qr(rng.standard_normal((s, s)))
    return (U * np.logspace(0, -np.log10(cond), s)) @ V.T


def _run(gpu, Kh, d, method, zeta=8, seed=0):
    Kd = gpu.from_numpy(np.ascontiguousarray(Kh.T)).cuda()
    Qd, R, S = K().sketch_qr(Kd, d, zeta=zeta, seed=seed, method=method)
    return Qd.cpu().numpy().T, R, S


ORACLE = {"rgs": lambda K_, Om: SQ.rgs(K_, Om)[:2], "whiten": lambda K_, Om: SQ.sketch_whiten(K_, Om)[:2],
          "rcholqr": SQ.rcholqr}


@pytest.mark.parametrize("method", ["rgs", "whiten", "rcholqr"])
@pytest.mark.parametrize("n,s,d,cond", [(50_021, 24, 96, 1e4), (20_000, 100, 256, 1e2)])
def test_sketch_qr_matches_oracle(gpu, method, n, s, d, cond):
    # n = 50 021: 49 tiles and a ragged tail; s = 100: products in two column blocks
    Kh = _graded_block(n, s, cond, 7)
    Q, R, S = _run(gpu, Kh, d, method)
    Om = omega_matrix(n, d, 8, 0)
    Qo, Ro = ORACLE[method](Kh, Om)
    u = 2.0 ** -46                                  # double-float unit with a margin
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
    assert np.linalg.norm(Kh - Q @ R) <= 10 * s * u * np.linalg.norm(Kh)
    assert np.linalg.norm(R - Ro) <= 10 * s * u * cond * np.linalg.norm(Ro)
    assert np.linalg.norm(Q - Qo) <= 10 * s * u * cond * np.sqrt(s)
    if method == "rcholqr":
        assert np.linalg.norm(Q.T @ Q - np.eye(s)) <= 10 * s * u
    else:
        assert np.linalg.norm(S.T @ S - np.eye(s)) <= 10 * s * u * cond
        assert np.linalg.norm(Om @ Q - S) <= 10 * s * u * cond


def test_rgs_and_whitening_agree_on_device(gpu):
    # the sketch-orthonormal QR is unique: both processes give the same Q and R
    n, s, d = 100_003, 40, 160
    Kh = _graded_block(n, s, 1e6, 9)
    Qg, Rg, _ = _run(gpu, Kh, d, "rgs")
    Qw, Rw, _ = _run(gpu, Kh, d, "whiten")
    assert np.linalg.norm(Rg - Rw) <= 1e-11 * np.linalg.norm(Rw)
    assert np.linalg.norm(Qg - Qw) <= 1e-7


def test_sketch_qr_full_size_properties(gpu):
    # a Krylov-sized block of the 1000^2 workload (n = 1e6, s = 80, d = 320),
    # checked through properties on the device (the oracle would need minutes)
    torch = gpu
    n, s, d = 1_000_000, 80, 320
    rng = np.random.default_rng(11)
    Kd = torch.from_numpy(rng.standard_normal((s, n))).cuda()
    for method in ("rgs", "whiten", "rcholqr", "rhqr"):
        Qd, R, S = K().sketch_qr(Kd, d, method=method)
        Rd = torch.from_numpy(np.ascontiguousarray(R.T)).cuda()        # rows of R^T
        res = torch.linalg.norm(Kd - Rd @ Qd) / torch.linalg.norm(Kd)   # K^T = R^T Q^T
        assert res.item() <= 1e-13
        if method == "rcholqr":
            G = (Qd @ Qd.T).cpu().numpy()
            assert np.linalg.norm(G - np.eye(s)) <= 1e-12
        elif method == "rhqr":                       # Theta Q = [Q[:s]; S]
            Qt = Qd[:, :s].cpu().numpy().T
            assert np.linalg.norm(Qt.T @ Qt + S.T @ S - np.eye(s)) <= 1e-12
        else:
            assert np.linalg.norm(S.T @ S - np.eye(s)) <= 1e-12


def test_rank_deficient_block_reports_breakdown(gpu):
    n, s, d = 4096, 6, 48
    Kh = _graded_block(n, s, 10.0, 3)
    Kh[:, 4] = 0.0                                   # a zero column: R[4, 4] = 0
    for method in ("rgs", "whiten", "rcholqr", "rhqr"):
        with pytest.raises(K().RKSError) as e:
            _run(gpu, Kh, d, method)
        assert e.value.code in (K().RKS_EBREAKDOWN, K().RKS_EDENSE)


@pytest.mark.parametrize("n,s,d,cond", [(50_021, 24, 96, 1e4), (20_000, 100, 256, 1e2)])
def test_rhqr_matches_oracle(gpu, n, s, d, cond):
    # Theta = [[I_s, 0], [0, Omega']], Omega' the embedding of dimension n - s
    Kh = _graded_block(n, s, cond, 17)
    Q, R, S = _run(gpu, Kh, d, "rhqr")
    Ob = omega_matrix(n - s, d, 8, 0)
    Qo, Ro, TQo = SQ.rhqr(Kh, Ob)
    u = 2.0 ** -46
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
    assert np.linalg.norm(Kh - Q @ R) <= 10 * s * u * np.linalg.norm(Kh)
    assert np.linalg.norm(R - Ro) <= 10 * s * u * cond * np.linalg.norm(Ro)
    assert np.linalg.norm(Q - Qo) <= 10 * s * u * cond * np.sqrt(s)
    # Theta Q = [Q[:s]; Omega' Q[s:]] orthonormal, to rounding (no kappa factor)
    TQ = np.vstack([Q[:s], S])
    assert np.linalg.norm(TQ.T @ TQ - np.eye(s)) <= 10 * s * u
    assert np.linalg.norm(Ob @ Q[s:] - S) <= 10 * s * u


def test_rhqr_stays_orthonormal_for_ill_conditioned_blocks(gpu):
    # kappa(K) = 1e12: the reflectors keep Theta Q orthonormal to rounding
    # where K R^{-1} (sketch and whiten) loses about u kappa
    n, s, d = 30_011, 20, 80
    Kh = _graded_block(n, s, 1e12, 19)
    Q, R, S = _run(gpu, Kh, d, "rhqr")
    TQ = np.vstack([Q[:s], S])
    u = 2.0 ** -46
    assert np.linalg.norm(TQ.T @ TQ - np.eye(s)) <= 10 * s * u
    assert np.linalg.norm(Kh - Q @ R) <= 10 * s * u * np.linalg.norm(Kh)
