"""Parity at full size: the kernel paths the benchmarked sizes take.

At n = 1e6 every one of the up to 304 sketch CTAs owns about 3 300 rows, so
its rows run through several 1024-row tiles with double-buffered staging and
per-tile bin lists; the small parity tests (n <= 2 773) never reach that.
Here the first expansion of Algorithm 2 (m + 1 basis vectors) is compared
with the oracle column by column, and whole solves are pinned by closed
forms whose accuracy the eigenvalue condition number bounds:

* the Kronecker-sum spectrum of the constant-coefficient 2D operator at
  N = 200 and N = 1000, to kappa(l) ||A||_1 times the computed residual
  (first-order perturbation bound; kappa from the closed-form left and right
  eigenvectors);
* the non-symmetric Toeplitz workload (n = 2000, k = 10, p = 30, d = 80,
  zeta = 4) run to a residual of 1e-8, against the oracle's residual and
  decomposition invariants (its eigenvalues have condition numbers ~1e261
  and are not pinned);
* the symmetric Toeplitz matrix with the same spectrum, n = 2000, to 1e-10.
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
    return torch


def K():
    from paper_2508_05400_gb300 import rks
    return rks


def _colrel(a, b):
    """Per-column relative error ||a_j - b_j|| / ||b_j||."""
    return np.linalg.norm(a - b, axis=0) / np.maximum(np.linalg.norm(b, axis=0), 1e-300)


def _first_expansion(A, k, p, d, zeta, prec):
    u1 = I.start_vector(A.n, 1)
    with K().Solver.from_csr(A, k, p, d, which="LR", tol=1e-8, zeta=zeta, u1=u1, max_restarts=-1,
                             prec=prec) as s:
        s.solve()
        U, S, H = s.krylov()
    st = R.start(sp.csr_matrix(A.to_scipy()), SK.omega_matrix(A.n, d, zeta, 0), u1)
    R.extend(st, k + p)
    return U, S, H, st


_EXP = {}


@pytest.mark.parametrize("prec", ["df", "fp64"])
def test_first_expansion_per_column_at_1e6(prec):
    # the 1000 x 1000 convection-diffusion workload: n = 1e6, m = 80, d = 320
    P = I.convdiff2d_problem()
    U, S, H, st = _first_expansion(P.A, P.k, P.p, P.d, P.zeta, prec)
    m = P.k + P.p
    assert U.shape == (P.A.n, m + 1) and H.shape == (m + 1, m)
    eh, es, eu = _colrel(H, st.Ba), _colrel(S, st.Sa), _colrel(U, st.Ua)
    print(f"\n{prec} n=1e6: max column error H {eh.max():.2e} S {es.max():.2e} U {eu.max():.2e}")
    # double-float carries a 48-bit significand, FP64 53 bits; the error of
    # column j grows with j through the recurrence
    tol = 1e-9 if prec == "df" else 1e-10
    assert eh.max() <= tol and es.max() <= tol and eu.max() <= tol
    # sketch orthonormality of the device basis (Def. 2.1) and the hash: Omega U = S
    assert np.abs(S.T @ S - np.eye(m + 1)).max() < 1e-12
    Om = SK.omega_matrix(P.A.n, P.d, P.zeta, 0)
    assert np.max(_colrel(Om @ U, S)) < 1e-12


def test_first_expansion_per_column_3d_fp32_values():
    # the 3D log-normal operator with FP32 values (the 160^3 workload's
    # structure) at 72^3 = 373 248 rows: two tiles per CTA, the second ragged
    P = I.convdiff3d_problem(N=72, k=10, p=30, d=160)
    U, S, H, st = _first_expansion(P.A, P.k, P.p, P.d, P.zeta, "df")
    eh, es, eu = _colrel(H, st.Ba), _colrel(S, st.Sa), _colrel(U, st.Ua)
    print(f"\n3D 72^3: max column error H {eh.max():.2e} S {es.max():.2e} U {eu.max():.2e}")
    assert eh.max() <= 1e-9 and es.max() <= 1e-9 and eu.max() <= 1e-9


# ---------------------------------------------------------------------------
# Closed-form Kronecker-sum spectrum at N = 200 and N = 1000
# ---------------------------------------------------------------------------

def _kappa_1d(N, nu, b, j):
    """Condition number ||x|| ||y|| / |y^T x| of eigenvalue j of the 1D upwind
    operator tridiag(nu/h^2 + b/h, -2nu/h^2 - b/h, nu/h^2): right eigenvector
    r^i sin(i j pi/(N+1)), left r^-i sin(...), r = sqrt(1 + b h / nu)."""
    h = 1.0 / (N + 1)
    i = np.arange(1, N + 1)
    lr = 0.5 * i * np.log1p(b * h / nu)
    s = np.sin(i * j * np.pi / (N + 1))
    x = np.exp(lr - lr.max()) * s
    y = np.exp(-lr) * s
    return np.linalg.norm(x) * np.linalg.norm(y) / abs(y @ x)


def _kronecker_pairs(N, bx, by, count):
    mx = I.convdiff_1d_eigenvalues(N, 1.0, bx)
    my = I.convdiff_1d_eigenvalues(N, 1.0, by)
    lam = (mx[:, None] + my[None, :]).ravel()
    idx = np.argsort(-lam)[: 4 * count]
    jx, jy = np.unravel_index(idx, (N, N))
    order_x = np.argsort(-mx)      # eigenvalue index -> 1-based mode number
    mode_x = {int(o): t + 1 for t, o in enumerate(order_x)}
    order_y = np.argsort(-my)
    mode_y = {int(o): t + 1 for t, o in enumerate(order_y)}
    kap = np.array([_kappa_1d(N, 1.0, bx, mode_x[int(a)]) * _kappa_1d(N, 1.0, by, mode_y[int(b)])
                    for a, b in zip(jx, jy)])
    return lam[idx], kap


@pytest.mark.parametrize("prec", ["fp64", "df"])
@pytest.mark.parametrize("N", [200, 1000])
def test_kronecker_closed_form_large(N, prec):
    A = I.convdiff_2d(N, N, 1.0, 20.0, 10.0)
    k, p, d = 6, 34, 160
    u = 2.0 ** -53 if prec == "fp64" else 2.0 ** -48
    tol = 16 * u                         # on the ||A||_1 scale, near the rounding floor
    with K().Solver.from_csr(A, k, p, d, which="LR", zeta=8, u1=I.start_vector(A.n, 1), prec=prec,
                             keep=k, tol=tol, eta_lock=tol / 2, conv="norm1", maxit=3000) as s:
        info = s.solve(allow_noconv=True)
        lam, X, res = s.eigpairs()
        nrm = s.norm1
    ex, kap = _kronecker_pairs(N, 20.0, 10.0, k)
    lam = lam[:k]
    err, bound = [], []
    for t, l in enumerate(lam):
        i = int(np.argmin(np.abs(ex - l)))
        err.append(abs(l - ex[i]))
        # first order: |dl| <= kappa ||E|| with a backward error ||E|| = ||r|| / ||x||
        bound.append(2.0 * kap[i] * max(res[t], u) * nrm)
    err, bound = np.array(err), np.array(bound)
    rel = err / np.abs(lam)
    print(f"\nN={N} {prec}: restarts {info['restarts']} est {info['max_est']:.1e} resid {res.max():.1e} "
          f"rel err {rel.max():.2e} kappa {kap[:k].max():.1e} bound/|l| {np.max(bound / np.abs(lam)):.2e}")
    # the k rightmost, each once
    assert len({int(np.argmin(np.abs(ex - l))) for l in lam}) == k
    assert np.all(np.sort(lam.real)[::-1] <= ex[0] + bound.max())
    assert np.all(err <= bound), (err, bound)
    assert res.max() <= 1e3 * u
    if N == 200 and prec == "fp64":
        assert rel.max() <= 1e-9


# ---------------------------------------------------------------------------
# Toeplitz workloads at n = 2000
# ---------------------------------------------------------------------------

def test_toeplitz_2000_to_convergence_against_oracle():
    # The non-symmetric Toeplitz workload (n = 2000, k = 10, p = 30, d = 80,
    # zeta = 4), run to ||A x - l x|| / (||A||_1 ||x||) <= 1e-8 with the thick
    # restart (keep = k): the estimate |b^T y| / ||A||_1 at 1e-8 / 4, locking
    # at 1e-8 / 8, FP64 verification at 1e-8 (about 2 200 restarts in the
    # oracle).  At the stated 1e-10 on |b^T y| / |l| the estimate stalls near
    # 1e-5..1e-3 for thousands of restarts, in the oracle as on the GPU (with
    # keep <= k; the oracle converges with keep = 20): the Ritz values wander
    # in a pseudospectrum of condition ~1e261.
    P = I.toeplitz_problem()
    u1 = I.start_vector(P.A.n, 1)
    kw = dict(tol=2.5e-9, eta_lock=1.25e-9, conv="norm1")
    with K().Solver.from_csr(P.A, P.k, P.p, P.d, which=P.which, zeta=P.zeta, u1=u1, keep=P.k, maxit=6000,
                             verify=1e-8, **kw) as s:
        info = s.solve(allow_noconv=False)
        lam, X, res = s.eigpairs()
        T, U, b = s.schur()
    assert info["converged"] == 1
    assert res.max() <= 1e-8
    Z = K().unpack_eigvecs(lam, X)
    hres, _ = R.true_residuals(P.A.to_scipy(), Z, lam)
    assert np.allclose(res, hres, rtol=1e-5, atol=1e-15)
    # A U = U T + u b^T on the active columns (a locked column carries the
    # perturbation its locking made: its b entry, up to eta_lock ||A||_1,
    # set to zero, Sec. 4.4)
    A = P.A.to_scipy()
    q = info["nlocked"]
    AU = A @ U
    r = (AU - U @ T)[:, q:]
    ba = b[q:]
    if ba.size and ba @ ba > 0:
        Pb = np.eye(ba.size) - np.outer(ba, ba) / (ba @ ba)
        assert np.linalg.norm(r @ Pb) <= 1e-10 * np.linalg.norm(AU)
    ores = R.rks(A, P.k, P.p, P.d, u1, zeta=P.zeta, seed=0, which="LM", keep=P.k, maxit=6000, **kw)
    assert ores.converged and ores.resid.max() <= 1e-8
    print(f"\ntoeplitz 2000: restarts GPU {info['restarts']} oracle {ores.restarts}; |l| GPU "
          f"{np.abs(lam).min():.4f}..{np.abs(lam).max():.4f} oracle {np.abs(ores.eigvals).min():.4f}.."
          f"{np.abs(ores.eigvals).max():.4f} (closed form max 3.9079)")
    # the computed eigenvalues lie in the tol-pseudospectrum, which fills the
    # symbol ellipse 2 - 1.3 e^{it} - 0.7 e^{-it} (|l| <= 4), not on the
    # closed-form segment (condition numbers ~1e261): a bound, not a pin
    for v in (lam, ores.eigvals):
        assert np.all(np.abs(v) <= 4.0 + 1e-6) and np.all(np.abs(v) >= 3.85)


def test_symmetric_toeplitz_2000_closed_form():
    # tridiag(-sqrt(0.91), 2, -sqrt(0.91)) is similar to the non-symmetric
    # workload (same closed-form spectrum 2 + 2 sqrt(0.91) cos(j pi/(n+1))) but
    # normal: its eigenvalues are pinned to 1e-10
    n = 2000
    s91 = np.sqrt(0.91)
    A = I.toeplitz_tridiag(n, -s91, 2.0, -s91)
    ex = I.toeplitz_eigenvalues(n, -s91, 2.0, -s91)
    ex = ex[np.argsort(-np.abs(ex))][:10]
    for prec in ("df", "fp64"):
        with K().Solver.from_csr(A, 10, 30, 80, which="LM", tol=1e-12, zeta=4, u1=I.start_vector(n, 1),
                                 keep=10, prec=prec, maxit=3000) as s:
            info = s.solve(allow_noconv=False)
            lam, X, res = s.eigpairs()
        assert np.max(np.abs(lam[:10] - ex) / np.abs(ex)) <= 1e-10, (prec, lam[:10], ex)
        # |b^T y| / |l| <= 1e-12 bounds the normwise residual only up to the
        # embedding's distortion sqrt((1 + eps) / (1 - eps)) and |l| / ||A||_1
        assert res.max() <= 5e-12
