"""CPU-side tests of librks: it builds, loads, exports the ABI, validates
arguments, and its host-side dense step (Algorithm 1 contraction) agrees with
the oracle's LAPACK-based ordered Schur form.  No GPU is touched."""
import os
import re

import numpy as np
import pytest

from oracle import rks as R
from paper_2508_05400_gb300 import build as B
from paper_2508_05400_gb300 import rks as K

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return K.lib()


def _declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "rks.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(rks_[a-z0-9_]+)\s*\(", hdr)))


def test_exports_every_declared_symbol(lib):
    names = _declared_symbols()
    assert "rks_create" in names and "rks_solve" in names and len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_strerror_and_defaults(lib):
    for code in K.STATUS:
        assert K.strerror(code)
    o = K.Opts()
    lib.rks_opts_default(o)
    assert (o.zeta, o.maxit, o.lock, o.mem_device, o.max_restarts) == (8, 1000, 1, 0, 0)


@pytest.mark.parametrize("kw", [dict(k=0), dict(p=1), dict(d=5), dict(tol=0.0), dict(which=7),
                                dict(n_override=3), dict(zeta=40),
                                dict(opt=dict(aggressive=2)), dict(opt=dict(keep=-1)), dict(opt=dict(keep=5)),
                                dict(opt=dict(ortho=5)), dict(opt=dict(ortho=1, prec=1)),
                                dict(opt=dict(conv=3)), dict(opt=dict(prec=7))])
def test_create_rejects_bad_arguments_before_any_device_call(lib, kw):
    from paper_2508_05400_gb300 import inputs as I
    A = I.toeplitz_tridiag(50)
    args = dict(k=4, p=8, d=40, tol=1e-8, which=0, zeta=4)
    n_override = kw.pop("n_override", None)
    opt = kw.pop("opt", {})
    args.update(kw)
    o = K.Opts()
    lib.rks_opts_default(o)
    o.zeta = args["zeta"]
    for f, v in opt.items():
        setattr(o, f, v)
    h = K._P()
    rc = lib.rks_create(h, n_override or A.n, A.rowptr.ctypes.data, A.colind.ctypes.data,
                        A.vals.ctypes.data, 0, args["k"], args["p"], args["d"], args["which"],
                        args["tol"], 0, o)
    assert rc == K.RKS_EINVAL
    assert not h.value


@pytest.mark.parametrize("which", ["LM", "SM", "LR", "SR"])
def test_host_ordered_schur_matches_oracle(lib, which):
    rng = np.random.default_rng(7)
    for m in (4, 17, 40, 120):
        Bm = rng.standard_normal((m, m))
        T, Q = K.host_ordered_schur(Bm, which, 12)
        To, Qo = R.ordered_schur(Bm, which, 12)
        assert np.linalg.norm(Q @ T @ Q.T - Bm) < 1e-13 * m * np.linalg.norm(Bm)
        assert np.linalg.norm(Q.T @ Q - np.eye(m)) < 1e-13 * m
        assert np.all(np.tril(T, -2) == 0)
        lam = np.array([R.block_eigenvalue(T, s, z) for s, z in R.schur_blocks(T)])
        lamo = np.array([R.block_eigenvalue(To, s, z) for s, z in R.schur_blocks(To)])
        nb = min(12, lam.size, lamo.size)
        assert np.allclose(lam[:nb], lamo[:nb], atol=1e-10 * np.abs(lamo).max())
        # same leading invariant subspace as the oracle's (up to rotation)
        kcols = sum(z for _, z in R.schur_blocks(T)[:nb])
        if kcols == sum(z for _, z in R.schur_blocks(To)[:nb]):
            sv = np.linalg.svd(Q[:, :kcols].T @ Qo[:, :kcols], compute_uv=False)
            assert sv.min() > 1 - 1e-8


def test_host_quasi_eig_matches_scipy(lib):
    import scipy.linalg as sla
    rng = np.random.default_rng(3)
    T, _ = K.host_ordered_schur(rng.standard_normal((25, 25)), "LR", 25)
    lam, Y = K.host_quasi_eig(T)
    assert np.linalg.norm(T @ Y - Y * lam) < 1e-12 * np.linalg.norm(T)
    assert np.allclose(np.linalg.norm(Y, axis=0), 1.0)
    assert np.allclose(np.sort_complex(lam), np.sort_complex(sla.eigvals(T)), atol=1e-12)
    # pairs come Im > 0 first
    for j in range(24):
        if lam[j].imag > 0:
            assert np.isclose(lam[j + 1], lam[j].conj())


@pytest.mark.parametrize("ka,drift", [(8, 1e-7), (20, 1e-3), (1, 0.3)])
def test_host_sketch_reorthonormalize_keeps_the_decomposition(lib, ka, drift):
    # A built so that A U = U T + u b^T holds exactly for a basis [U u] that
    # is only nearly orthonormal under a sketch Omega (as after the mixed
    # path's correction): [V v] = [U u] R^-1 must satisfy A V = V Tn + v bn^T
    # and have orthonormal sketches Q = Omega [V v]
    rng = np.random.default_rng(40 + ka)
    n, d = 300, 4 * ka + 20
    Om = rng.standard_normal((d, n)) / np.sqrt(d)
    W = np.linalg.qr(rng.standard_normal((n, ka + 1)))[0]
    # sketch-orthonormal start, then a drift of relative size `drift`
    Qs, Rs = np.linalg.qr(Om @ W)
    W = W @ np.linalg.inv(Rs)
    W = W + drift * rng.standard_normal(W.shape) * np.linalg.norm(W, axis=0) / np.sqrt(n)
    U, u = W[:, :ka], W[:, ka]
    T = np.triu(rng.standard_normal((ka, ka))) + np.diag(rng.uniform(1, 2, ka))
    b = rng.standard_normal(ka)
    Up = np.linalg.pinv(U)
    A = (U @ T + np.outer(u, b)) @ Up + rng.standard_normal((n, n)) @ (np.eye(n) - U @ Up)
    assert np.linalg.norm(A @ U - U @ T - np.outer(u, b)) <= 1e-9 * np.linalg.norm(A @ U)
    S = Om @ W
    Q, Rinv, Tn, bn = K.host_sketch_reorthonormalize(S, T, b)
    Vv = W @ Rinv
    V, v = Vv[:, :ka], Vv[:, ka]
    assert np.allclose(Rinv, np.triu(Rinv))
    assert np.linalg.norm(Q.T @ Q - np.eye(ka + 1)) <= 1e-12 * (ka + 1)
    assert np.linalg.norm(Om @ Vv - Q) <= 1e-10 * np.linalg.norm(Q)
    rel = A @ V - V @ Tn - np.outer(v, bn)
    assert np.linalg.norm(rel) <= 1e-9 * np.linalg.norm(A @ V)
    # the eigenvalues of T are those of Tn (a similarity of the projected part)
    assert np.allclose(np.sort_complex(np.linalg.eigvals(Tn + np.outer(
        np.linalg.lstsq(V, v, rcond=None)[0], bn))), np.sort_complex(np.linalg.eigvals(
        T + np.outer(np.linalg.lstsq(U, u, rcond=None)[0], b))), atol=1e-7 * np.linalg.norm(T))


def test_host_reorder_select_matches_lapack_dtrsen(lib):
    # The aggressive-deflation reorder (Sec. 4.3): flagged blocks first, both
    # groups in their original order, as LAPACK dtrsen orders them.  Same
    # block eigenvalue sequence, T = Z T' Z^T with Z orthogonal, and the same
    # leading invariant subspace as dtrsen's.
    import scipy.linalg as sla
    from scipy.linalg.lapack import dtrsen
    rng = np.random.default_rng(11)
    for m in (6, 23, 60):
        T0, _ = sla.schur(rng.standard_normal((m, m)), output="real")
        blocks = R.schur_blocks(T0)
        for trial in range(4):
            flags = rng.random(len(blocks)) < 0.4
            if trial == 0:
                flags[:] = False; flags[-1] = True          # last block to the top
            sel = np.zeros(m, dtype=np.int32)
            for (s, z), f in zip(blocks, flags):
                sel[s:s + z] = int(f)
            T, Z = K.host_reorder_select(T0, sel)
            To, Zo, *_, info = dtrsen(sel, T0, np.eye(m), job="N")
            assert info == 0
            assert np.linalg.norm(Z @ T @ Z.T - T0) < 1e-13 * m * np.linalg.norm(T0)
            assert np.linalg.norm(Z.T @ Z - np.eye(m)) < 1e-13 * m
            assert np.all(np.tril(T, -2) == 0)
            lam = [R.block_eigenvalue(T, s, z) for s, z in R.schur_blocks(T)]
            lamo = [R.block_eigenvalue(To, s, z) for s, z in R.schur_blocks(To)]
            assert np.allclose(lam, lamo, atol=1e-10 * np.abs(lamo).max())
            want = [R.block_eigenvalue(T0, s, z) for (s, z), f in zip(blocks, flags) if f]
            want += [R.block_eigenvalue(T0, s, z) for (s, z), f in zip(blocks, flags) if not f]
            assert np.allclose(lam, want, atol=1e-10 * np.abs(want).max())
            kc = int(sel.sum())
            if kc:
                sv = np.linalg.svd(Z[:, :kc].T @ Zo[:, :kc], compute_uv=False)
                assert sv.min() > 1 - 1e-8


@pytest.mark.parametrize("kw", [dict(s=0), dict(s=193), dict(d=15), dict(zeta=0), dict(zeta=17), dict(method=4),
                                dict(ldk=99), dict(s=50, d=40), dict(nullK=True), dict(nullR=True),
                                dict(method=3, n=9, ldk=9, ldq=9)])
def test_sketch_qr_rejects_bad_arguments_before_any_device_call(lib, kw):
    # argument checks of rks_sketch_qr return before any CUDA call (no GPU here)
    a = dict(n=100, s=8, ldk=100, d=32, zeta=8, method=0, ldq=100)
    nullK, nullR = kw.pop("nullK", False), kw.pop("nullR", False)
    a.update(kw)
    fake = 0x1000      # never dereferenced: the call must fail first
    R = np.zeros((max(a["s"], 1), max(a["s"], 1)))
    rc = lib.rks_sketch_qr(a["n"], a["s"], None if nullK else fake, a["ldk"], a["d"], a["zeta"], 0, a["method"],
                           fake, a["ldq"], None if nullR else R.ctypes.data, None, None)
    assert rc == K.RKS_EINVAL


def test_profile_mask_selects_kernel_classes():
    # rks_opts.profile > 1: bit c + 1 times class c (RKS_K_* order = KCLASSES order)
    assert K.profile_mask() == 1
    assert K.profile_mask("update_sketch") == 1 | 2 << 2
    assert K.profile_mask("spmv_sketch", "restart") == 1 | 2 << 0 | 2 << 4
    hdr = open(os.path.join(ROOT, "include", "rks.h")).read()
    for i, name in enumerate(["RKS_K_SPMV", "RKS_K_LS", "RKS_K_UPDATE", "RKS_K_FINISH", "RKS_K_RESTART",
                              "RKS_K_OTHER"]):
        assert re.search(r"\b%s = %d\b" % (name, i), hdr)


def test_bench_kernel_hash_finds_the_update_kernel():
    # the traffic figure is keyed to the update kernel's source; the markers
    # that delimit it must exist
    import sys
    sys.path.insert(0, ROOT)
    import bench
    h = bench._kernel_hash()
    assert h is not None and re.fullmatch(r"[0-9a-f]{16}", h)


def test_create_batched_rejects_bad_arguments_before_any_device_call(lib):
    # count, missing arrays and per-problem options (streams, start vectors)
    # are checked before the first CUDA call
    import ctypes as C
    from paper_2508_05400_gb300 import inputs as I
    A = I.toeplitz_tridiag(50)
    ns = np.array([A.n], dtype=np.int64)
    ptrs = [np.array([a.ctypes.data], dtype=np.uint64) for a in (A.rowptr, A.colind, A.vals)]
    h = K._P()

    def call(count=1, opts=None, null=None):
        arrs = [None if null == j else ptrs[j].ctypes.data for j in range(3)]
        return lib.rks_create_batched(C.byref(h), count, ns.ctypes.data, arrs[0], arrs[1], arrs[2], 0, 4, 8, 40, 0,
                                      1e-8, 0, C.byref(opts) if opts is not None else None, 1)
    assert call(count=0) == K.RKS_EINVAL
    for j in range(3):
        assert call(null=j) == K.RKS_EINVAL
    o = K.Opts()
    lib.rks_opts_default(o)
    o.u1 = 0x1000
    assert call(opts=o) == K.RKS_EINVAL
    o.u1 = None
    o.stream = 0x1000
    assert call(opts=o) == K.RKS_EINVAL
    assert not h.value


def test_binding_constants_match_the_header():
    # the ctypes binding's names for statuses and options carry the header's values
    hdr = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "rks.h")).read(), flags=re.S)
    val = lambda name: int(re.search(r"\b%s\s*=\s*(-?\d+)" % name, hdr).group(1))
    for code, name in K.STATUS.items():
        assert val(name) == code, name
    for name, v in K.WHICH.items():
        assert val("RKS_" + name) == v
    assert {n: val("RKS_CONV_" + n.upper()) for n in K.CONV} == K.CONV
    assert {n: val("RKS_PREC_" + n.upper()) for n in K.PREC} == K.PREC
    assert {n: val("RKS_ORTHO_" + n.upper()) for n in K.ORTHO} == K.ORTHO
    assert {n: val("RKS_QR_" + n.upper()) for n in K.QR_METHODS} == K.QR_METHODS
    # the options struct: same field order and count as the header's rks_opts
    for cname, py in (("rks_opts", K.Opts), ("rks_info", K.Info), ("rks_stats", K.Stats)):
        body = re.search(r"typedef struct \{([^{}]*)\} %s;" % cname, hdr).group(1)
        fields = re.findall(r"(\w+)(?:\[\w+\])?;", body)
        assert fields == [f for f, _ in py._fields_], cname


def test_noalloc_binding_rejects_bad_buffers_before_any_call(monkeypatch):
    # the allocation-free sketch writes d values into z without knowing its
    # size: the binding checks z's size, the dtypes, contiguity and devices
    # before anything reaches the library (no GPU needed to see it)
    torch = pytest.importorskip("torch")
    from paper_2508_05400_gb300 import rks

    def never(*a):
        raise AssertionError("the library was called")
    monkeypatch.setattr(rks, "lib", never)
    x = torch.zeros(1000, dtype=torch.float64)
    for z, msg in ((torch.zeros(79, dtype=torch.float64), "fewer than d"),
                   (torch.zeros(80, dtype=torch.float32), "float64"),
                   (torch.zeros(160, dtype=torch.float64)[::2], "contiguous"),
                   (torch.zeros(80, dtype=torch.float64), "CUDA")):
        with pytest.raises(ValueError, match=msg):
            rks.sketch_apply_noalloc(x, z, 80, 4, 0)
    with pytest.raises(ValueError, match="float64"):
        rks.sketch_apply_noalloc(x.float(), torch.zeros(80, dtype=torch.float64), 80, 4, 0)


def test_create_batched_dev_rejects_bad_arguments_before_any_device_call(lib):
    # sizes, keep, cluster size, CSR structure, values and the unsupported
    # options are all checked before the first CUDA call
    import ctypes as C
    from paper_2508_05400_gb300 import inputs as I
    A = I.toeplitz_tridiag(200)
    bad_col = A.colind.copy()
    bad_col[5] = A.n
    bad_val = np.ascontiguousarray(A.vals, dtype=np.float64).copy()
    bad_val[3] = np.nan
    h = K._P()

    def call(k=8, p=24, d=64, count=1, ctas=0, opts=None, colind=None, vals=None, n=None, which=2, tol=1e-8):
        ci = A.colind if colind is None else colind
        vv = np.ascontiguousarray(A.vals, dtype=np.float64) if vals is None else vals
        ns = np.array([A.n if n is None else n], dtype=np.int64)
        ptrs = [np.array([a.ctypes.data], dtype=np.uint64) for a in (A.rowptr, ci, vv)]
        return lib.rks_create_batched_dev(C.byref(h), count, ns.ctypes.data, ptrs[0].ctypes.data, ptrs[1].ctypes.data,
                                          ptrs[2].ctypes.data, 0, k, p, d, which, tol, 0,
                                          C.byref(opts) if opts is not None else None, ctas)
    assert call(count=0) == K.RKS_EINVAL
    assert call(k=0) == K.RKS_EINVAL
    assert call(p=1) == K.RKS_EINVAL
    assert call(k=40, p=30) == K.RKS_EINVAL            # m > 64
    assert call(k=32, p=8, d=64) == K.RKS_EINVAL        # k + 1 > 32
    assert call(d=32) == K.RKS_EINVAL                   # d < m + 1
    assert call(ctas=3) == K.RKS_EINVAL
    assert call(which=4) == K.RKS_EINVAL
    assert call(tol=0.0) == K.RKS_EINVAL
    assert call(n=20) == K.RKS_EINVAL                   # n < m + 1
    assert call(colind=bad_col) == K.RKS_EINVAL
    assert call(vals=bad_val) == K.RKS_EINVAL
    o = K.Opts()
    lib.rks_opts_default(o)
    o.keep = 40                                         # keep >= m
    assert call(opts=o) == K.RKS_EINVAL
    o.keep = 0
    o.mem_device = 1
    assert call(opts=o) == K.RKS_EINVAL
    o.mem_device = 0
    o.u1 = 0x1000
    assert call(opts=o) == K.RKS_EINVAL
    assert not h.value
