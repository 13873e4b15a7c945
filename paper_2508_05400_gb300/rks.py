"""Python binding of librks (ctypes): argument marshalling only.

Every computation happens in the C ABI declared in ``include/rks.h`` (CUDA
kernels for sm_103a plus the host-side small dense step).  PyTorch is used
only to hold device buffers and to provide streams.  If ``librks.so`` has not
been built, loading fails with an error: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librks.so")

WHICH = {"LM": 0, "SM": 1, "LR": 2, "SR": 3}
STATUS = {0: "RKS_OK", -1: "RKS_EINVAL", -2: "RKS_ENOMEM", -3: "RKS_ECUDA", -4: "RKS_ENOCONV",
          -5: "RKS_EBREAKDOWN", -6: "RKS_ENAN", -7: "RKS_ESTATE", -8: "RKS_EDENSE",
          -9: "RKS_ETIMEOUT"}
RKS_OK, RKS_EINVAL, RKS_ENOCONV, RKS_EBREAKDOWN, RKS_EDENSE = 0, -1, -4, -5, -8


class RKSError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} ({strerror(code)})")


class Opts(C.Structure):
    _fields_ = [("zeta", C.c_int), ("maxit", C.c_int), ("lock", C.c_int), ("mem_device", C.c_int),
                ("stream", C.c_void_p), ("u1", C.c_void_p), ("eta_lock", C.c_double),
                ("max_restarts", C.c_int), ("profile", C.c_int), ("conv", C.c_int),
                ("prec", C.c_int), ("mixed_tol", C.c_double), ("verify", C.c_double), ("keep", C.c_int), ("ortho", C.c_int),
                ("tc_restart", C.c_int), ("aggressive", C.c_int),
                ("debug_stall", C.c_int)]


CONV = {"eig": 0, "norm1": 1}
PREC = {"df": 0, "fp64": 1, "mixed": 2}
ORTHO = {"sketch": 0, "cgs2": 1}


KCLASSES = ("spmv_sketch", "ls", "update_sketch", "finish", "restart", "other")


def profile_mask(*classes: str) -> int:
    """rks_opts.profile value that times only the given kernel classes."""
    m = 1
    for c in classes:
        m |= 2 << KCLASSES.index(c)
    return m


class Stats(C.Structure):
    _fields_ = [("launches", C.c_int64 * 6), ("ms", C.c_double * 6), ("bytes", C.c_double * 6),
                ("flops", C.c_double * 6), ("host_ms", C.c_double), ("whitenings", C.c_int64),
                ("reorders", C.c_int64), ("fp32_restarts", C.c_int), ("mixed_phase2", C.c_int),
                ("handover_rel", C.c_double), ("launches_f32", C.c_int64 * 6), ("ms_f32", C.c_double * 6),
                ("bytes_f32", C.c_double * 6)]

    def as_dict(self) -> dict:
        out = {name: {"launches": self.launches[i], "ms": self.ms[i], "bytes": self.bytes[i],
                      "flops": self.flops[i], "launches_f32": self.launches_f32[i], "ms_f32": self.ms_f32[i],
                      "bytes_f32": self.bytes_f32[i]} for i, name in enumerate(KCLASSES)}
        out["host_ms"] = self.host_ms
        out["whitenings"] = self.whitenings
        out["reorders"] = self.reorders
        out["fp32_restarts"] = self.fp32_restarts
        out["mixed_phase2"] = self.mixed_phase2     # 0 none, 1 from the hand-over, 2 from the sum of Schur vectors
        out["handover_rel"] = self.handover_rel
        out["launches_total"] = int(sum(self.launches))
        return out


class Info(C.Structure):
    _fields_ = [("nconv", C.c_int), ("nlocked", C.c_int), ("restarts", C.c_int),
                ("nmatvec", C.c_int64), ("converged", C.c_int), ("max_est", C.c_double),
                ("max_resid", C.c_double), ("t_solve_ms", C.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
_P = C.c_void_p
_D = C.POINTER(C.c_double)


def lib() -> C.CDLL:
    """Load librks.so (built by ``paper_2508_05400_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"librks.so is not built ({LIB_PATH}); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        L.rks_opts_default.argtypes = [C.POINTER(Opts)]
        L.rks_opts_default.restype = None
        L.rks_strerror.argtypes = [C.c_int]
        L.rks_strerror.restype = C.c_char_p
        L.rks_create.argtypes = [C.POINTER(_P), C.c_int64, _P, _P, _P, C.c_int, C.c_int, C.c_int,
                                 C.c_int, C.c_int, C.c_double, C.c_uint64, C.POINTER(Opts)]
        L.rks_create.restype = C.c_int
        L.rks_solve.argtypes = [_P, C.POINTER(Info)]
        L.rks_solve.restype = C.c_int
        L.rks_get_schur.argtypes = [_P, _P, _P, _P]
        L.rks_get_schur.restype = C.c_int
        L.rks_get_eigpairs.argtypes = [_P, _P, _P, _P, _P]
        L.rks_get_eigpairs.restype = C.c_int
        L.rks_get_estimates.argtypes = [_P, _P]
        L.rks_get_rayleigh.argtypes = [_P, _P, _P]
        L.rks_get_rayleigh.restype = C.c_int
        L.rks_get_estimates.restype = C.c_int
        L.rks_get_krylov.argtypes = [_P, C.POINTER(C.c_int), _P, _P, _P]
        L.rks_get_krylov.restype = C.c_int
        L.rks_get_stats.argtypes = [_P, C.POINTER(Stats)]
        L.rks_get_stats.restype = C.c_int
        L.rks_get_history.argtypes = [_P, _P, _P, C.c_int]
        L.rks_get_history.restype = C.c_int
        L.rks_spmv_format.argtypes = [_P]
        L.rks_spmv_format.restype = C.c_int
        L.rks_nkept.argtypes = [_P]
        L.rks_nkept.restype = C.c_int
        L.rks_nwanted.argtypes = [_P]
        L.rks_nwanted.restype = C.c_int
        L.rks_norm1.argtypes = [_P]
        L.rks_norm1.restype = C.c_double
        L.rks_basis_product_f32.argtypes = [C.c_int64, _P, C.c_int64, C.c_int, _P, C.c_int, _P, _P]
        L.rks_basis_product_f32.restype = C.c_int
        L.rks_create_batched.argtypes = [C.POINTER(_P), C.c_int, _P, _P, _P, _P, C.c_int, C.c_int, C.c_int,
                                         C.c_int, C.c_int, C.c_double, C.c_uint64, C.POINTER(Opts), C.c_int]
        L.rks_create_batched.restype = C.c_int
        L.rks_solve_batched.argtypes = [_P, C.c_int, _P]
        L.rks_solve_batched.restype = C.c_int
        L.rks_batch_count.argtypes = [_P]
        L.rks_batch_count.restype = C.c_int
        L.rks_batch_get.argtypes = [_P, C.c_int]
        L.rks_batch_get.restype = _P
        L.rks_batch_status.argtypes = [_P, C.c_int]
        L.rks_batch_status.restype = C.c_int
        L.rks_destroy_batched.argtypes = [_P]
        L.rks_destroy_batched.restype = None
        L.rks_create_batched_dev.argtypes = [C.POINTER(_P), C.c_int, _P, _P, _P, _P, C.c_int, C.c_int, C.c_int,
                                             C.c_int, C.c_int, C.c_double, C.c_uint64, _P, C.c_int]
        L.rks_create_batched_dev.restype = C.c_int
        L.rks_solve_batched_dev.argtypes = [_P, _P]
        L.rks_solve_batched_dev.restype = C.c_int
        L.rks_dbatch_config.argtypes = [_P, _P, _P, C.c_int, _P]
        L.rks_dbatch_config.restype = C.c_int
        L.rks_dbatch_status.argtypes = [_P, C.c_int]
        L.rks_dbatch_status.restype = C.c_int
        L.rks_dbatch_phase_cycles.argtypes = [_P, _P, C.c_int]
        L.rks_dbatch_phase_cycles.restype = C.c_int
        L.rks_dbatch_eigpairs.argtypes = [_P, C.c_int, _P, _P, _P, _P, _P, _P, _P]
        L.rks_dbatch_eigpairs.restype = C.c_int
        L.rks_destroy_batched_dev.argtypes = [_P]
        L.rks_destroy_batched_dev.restype = None
        L.rks_dev_ordered_schur.argtypes = [C.c_int, _P, C.c_int, C.c_int, _P, _P, _P, _P, _P, _P]
        L.rks_dev_ordered_schur.restype = C.c_int
        L.rks_basis_product_df.argtypes = [C.c_int64, _P, C.c_int64, C.c_int, _P, C.c_int, _P, _P]
        L.rks_basis_product_df.restype = C.c_int
        L.rks_sketch_qr.argtypes = [C.c_int64, C.c_int, _P, C.c_int64, C.c_int, C.c_int, C.c_uint64, C.c_int, _P,
                                    C.c_int64, _P, _P, _P]
        L.rks_sketch_qr.restype = C.c_int
        L.rks_destroy.argtypes = [_P]
        L.rks_ws_nparams.argtypes = []
        L.rks_ws_nparams.restype = C.c_int64
        L.rks_ws_create.argtypes = [C.POINTER(_P), C.c_int, C.c_int, C.c_uint64, _P]
        L.rks_ws_create.restype = C.c_int
        L.rks_ws_get_params.argtypes = [_P, _P]
        L.rks_ws_get_params.restype = C.c_int
        L.rks_ws_set_params.argtypes = [_P, _P]
        L.rks_ws_set_params.restype = C.c_int
        L.rks_ws_forward.argtypes = [_P, _P, _P]
        L.rks_ws_forward.restype = C.c_int
        L.rks_ws_accumulate.argtypes = [_P, _P, _P, C.c_int, C.POINTER(C.c_double)]
        L.rks_ws_accumulate.restype = C.c_int
        L.rks_ws_get_grad.argtypes = [_P, _P]
        L.rks_ws_get_grad.restype = C.c_int
        L.rks_ws_zero_grad.argtypes = [_P]
        L.rks_ws_zero_grad.restype = C.c_int
        L.rks_ws_adam_step.argtypes = [_P, C.c_float]
        L.rks_ws_adam_step.restype = C.c_int
        L.rks_ws_start_vector.argtypes = [_P, _P, C.c_double, C.c_uint64, _P]
        L.rks_ws_start_vector.restype = C.c_int
        L.rks_ws_destroy.argtypes = [_P]
        L.rks_ws_destroy.restype = None
        L.rks_destroy.restype = None
        L.rks_sketch_pairs.argtypes = [C.c_int64, C.c_int, C.c_int, C.c_uint64, _P, _P, _P]
        L.rks_sketch_pairs.restype = C.c_int
        L.rks_sketch_apply.argtypes = [C.c_int64, C.c_int, C.c_int, C.c_uint64, _P, _P, _P]
        L.rks_sketch_apply.restype = C.c_int
        L.rks_sketch_apply_noalloc.argtypes = [C.c_int64, C.c_int, C.c_int, C.c_uint64, _P, _P, _P]
        L.rks_sketch_apply_noalloc.restype = C.c_int
        L.rks_host_ordered_schur.argtypes = [C.c_int, _P, C.c_int, C.c_int, _P, _P]
        L.rks_host_ordered_schur.restype = C.c_int
        L.rks_host_reorder_select.argtypes = [C.c_int, _P, _P, _P]
        L.rks_host_reorder_select.restype = C.c_int
        L.rks_host_quasi_eig.argtypes = [C.c_int, _P, _P, _P, _P, _P]
        L.rks_host_quasi_eig.restype = C.c_int
        L.rks_host_sketch_reorthonormalize.argtypes = [C.c_int, C.c_int, _P, _P, _P, _P, _P, _P]
        L.rks_host_sketch_reorthonormalize.restype = C.c_int
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().rks_strerror(code).decode()


def _check(code: int, where: str, ok=(RKS_OK,)):
    if code not in ok:
        raise RKSError(code, where)
    return code


def _ptr(a) -> int | None:
    """Address of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _host(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def _fortran(shape) -> np.ndarray:
    return np.zeros(shape, dtype=np.float64, order="F")


class Solver:
    """One rKS problem: ``rks_create`` on construction, ``rks_destroy`` on close.

    Host mode (default): rowptr/colind/vals/u1 are numpy arrays.  Device mode
    (``device=True``): they are CUDA tensors (torch) and results that are
    n-dimensional are written into CUDA tensors the caller passes.
    """

    def __init__(self, n, rowptr, colind, vals, k, p, d, which="LM", tol=1e-10, seed=0, *,
                 zeta=8, maxit=1000, lock=True, u1=None, eta_lock=0.0, max_restarts=0,
                 device=False, stream=None, profile=False, conv="eig", verify=0.0, prec="df",
                 mixed_tol=0.0, keep=0, ortho="sketch", tc_restart=True,
                 aggressive=False, debug_stall=0):
        L = lib()
        self.n, self.k, self.p, self.d = int(n), int(k), int(p), int(d)
        self.device = bool(device)
        if device:
            self._keep = (rowptr, colind, vals, u1)
            vdt = 0 if str(vals.dtype).endswith("float64") else 1
        else:
            rowptr = _host(rowptr, np.int32)
            colind = _host(colind, np.int32)
            vals = np.ascontiguousarray(vals)
            if vals.dtype not in (np.float64, np.float32):
                vals = vals.astype(np.float64)
            vdt = 0 if vals.dtype == np.float64 else 1
            if u1 is not None:
                u1 = _host(u1, np.float64)
            self._keep = (rowptr, colind, vals, u1)
        o = Opts()
        L.rks_opts_default(C.byref(o))
        o.zeta, o.maxit, o.lock, o.mem_device = int(zeta), int(maxit), int(bool(lock)), int(device)
        o.stream = stream
        o.u1 = _ptr(u1)
        o.eta_lock = float(eta_lock)
        o.max_restarts = int(max_restarts)
        o.profile = int(profile)      # True/1: every kernel class; see rks_opts.profile for a class mask
        o.conv = CONV[conv]
        o.verify = float(verify)
        o.prec = PREC[prec]
        o.mixed_tol = float(mixed_tol)
        o.keep = int(keep)
        o.ortho = ORTHO[ortho]
        o.tc_restart = int(bool(tc_restart))
        o.aggressive = int(bool(aggressive))
        o.debug_stall = int(debug_stall)
        h = _P()
        _check(L.rks_create(C.byref(h), self.n, _ptr(rowptr), _ptr(colind), _ptr(vals), vdt,
                            self.k, self.p, self.d, WHICH[which] if isinstance(which, str) else int(which),
                            float(tol), int(seed) & 0xFFFFFFFFFFFFFFFF, C.byref(o)), "rks_create")
        self._h = h

    @classmethod
    def from_csr(cls, A, k, p, d, **kw):
        """From an ``inputs.CSR`` (host arrays)."""
        return cls(A.n, A.rowptr, A.colind, A.vals, k, p, d, **kw)

    def solve(self, allow_noconv=True) -> dict:
        info = Info()
        rc = lib().rks_solve(self._h, C.byref(info))
        _check(rc, "rks_solve", ok=(RKS_OK, RKS_ENOCONV) if allow_noconv else (RKS_OK,))
        out = info.as_dict()
        out["status"] = STATUS.get(rc, rc)
        return out

    def history(self, cap: int = 100000):
        """(max convergence quantity, locked count) after each restart."""
        h = np.zeros(cap)
        q = np.zeros(cap, dtype=np.int32)
        nh = lib().rks_get_history(self._h, h.ctypes.data, q.ctypes.data, cap)
        _check(min(nh, 0), "rks_get_history")
        return h[:nh], q[:nh]

    def stats(self) -> dict:
        st = Stats()
        _check(lib().rks_get_stats(self._h, C.byref(st)), "rks_get_stats")
        return st.as_dict()

    SPMV_FORMATS = ("csr", "ell", "dia", "warp", "merge")

    @property
    def spmv_format(self) -> str:
        """Storage the SpMV reads (rks_spmv_format)."""
        return self.SPMV_FORMATS[_check(lib().rks_spmv_format(self._h), "rks_spmv_format", ok=(0, 1, 2, 3, 4))]

    @property
    def nkept(self) -> int:
        return lib().rks_nkept(self._h)

    @property
    def nwanted(self) -> int:
        return lib().rks_nwanted(self._h)

    @property
    def norm1(self) -> float:
        return lib().rks_norm1(self._h)

    def schur(self, U_out=None):
        """(T, U, b) of the decomposition A U = U T + u b^T (U on host unless U_out given)."""
        kk = self.nkept
        T = _fortran((kk, kk))
        b = np.zeros(kk)
        U = U_out if U_out is not None else _fortran((self.n, kk))
        _check(lib().rks_get_schur(self._h, T.ctypes.data, _ptr(U), b.ctypes.data), "rks_get_schur")
        return T, U, b

    def eigpairs(self, X_out=None, want_vectors=True):
        """(lam complex[nw], X real-packed n x nw or None, resid[nw]), best first."""
        kk = self.nwanted
        lre, lim, res = np.zeros(kk), np.zeros(kk), np.zeros(kk)
        X = None
        if want_vectors:
            X = X_out if X_out is not None else _fortran((self.n, kk))
        _check(lib().rks_get_eigpairs(self._h, lre.ctypes.data, lim.ctypes.data, _ptr(X),
                                      res.ctypes.data), "rks_get_eigpairs")
        return lre + 1j * lim, X, res

    def rayleigh(self) -> np.ndarray:
        """Rayleigh quotients x^H A x / x^H x of the returned Ritz vectors (complex[nw])."""
        nw = self.nwanted
        re, im = np.zeros(nw), np.zeros(nw)
        _check(lib().rks_get_rayleigh(self._h, re.ctypes.data, im.ctypes.data), "rks_get_rayleigh")
        return re + 1j * im

    def estimates(self) -> np.ndarray:
        e = np.zeros(self.nwanted)
        _check(lib().rks_get_estimates(self._h, e.ctypes.data), "rks_get_estimates")
        return e

    def krylov(self):
        """(U, S, H) of the current sketch-orthonormal Krylov decomposition."""
        m = self.k + self.p
        U = _fortran((self.n, m + 1))
        S = _fortran((self.d, m + 1))
        H = _fortran((m + 1, m))
        nc = C.c_int()
        Hbuf = np.zeros((m + 1) * m)
        _check(lib().rks_get_krylov(self._h, C.byref(nc), U.ctypes.data, S.ctypes.data,
                                    Hbuf.ctypes.data), "rks_get_krylov")
        j = nc.value
        H = Hbuf[: j * (j - 1)].reshape((j, j - 1), order="F")
        return U[:, :j], S[:, :j], H

    def close(self):
        if getattr(self, "_h", None):
            if not getattr(self, "_borrowed", False):
                lib().rks_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def unpack_eigvecs(lam: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Complex eigenvectors from the LAPACK dgeev real packing."""
    kk = lam.size
    Z = np.zeros((X.shape[0], kk), dtype=complex)
    j = 0
    while j < kk:
        if lam[j].imag > 0 and j + 1 < kk:
            Z[:, j] = X[:, j] + 1j * X[:, j + 1]
            Z[:, j + 1] = X[:, j] - 1j * X[:, j + 1]
            j += 2
        else:
            Z[:, j] = X[:, j]
            j += 1
    return Z


def sketch_pairs(n: int, d: int, zeta: int, seed: int):
    """All (row, sign) pairs of Omega from the device hash, as numpy arrays (n, zeta)."""
    import torch
    rows = torch.empty(n * zeta, dtype=torch.int32, device="cuda")
    signs = torch.empty(n * zeta, dtype=torch.int8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    _check(lib().rks_sketch_pairs(n, d, zeta, seed, rows.data_ptr(), signs.data_ptr(), stream),
           "rks_sketch_pairs")
    torch.cuda.synchronize()
    return rows.cpu().numpy().reshape(n, zeta), signs.cpu().numpy().reshape(n, zeta)


def sketch_apply(x, d: int, zeta: int, seed: int):
    """z = Omega x on the device for a CUDA float64 tensor x."""
    import torch
    z = torch.empty(d, dtype=torch.float64, device=x.device)
    stream = torch.cuda.current_stream().cuda_stream
    _check(lib().rks_sketch_apply(x.numel(), d, zeta, seed, x.data_ptr(), z.data_ptr(), stream),
           "rks_sketch_apply")
    return z


def sketch_apply_noalloc(x, z, d: int, zeta: int, seed: int) -> int:
    """z = Omega x through the allocation-free entry point (x, z: CUDA float64 tensors).

    For callers that cannot allocate device memory; returns the status code.
    x and z must be contiguous float64 tensors on the same CUDA device and z
    must hold at least d values: the entry point writes d values into z
    without knowing its size, so these are checked here (ValueError) before
    anything runs.
    """
    import torch
    for name, t in (("x", x), ("z", z)):
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if t.dtype != torch.float64:
            raise ValueError(f"{name} must be float64, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if z.numel() < d:
        raise ValueError(f"z holds {z.numel()} values, fewer than d = {d}")
    if x.device != z.device:
        raise ValueError(f"x and z are on different devices ({x.device}, {z.device})")
    if not x.is_cuda:
        raise ValueError("x and z must be CUDA tensors")
    with torch.cuda.device(x.device):
        stream = torch.cuda.current_stream(x.device).cuda_stream
        return lib().rks_sketch_apply_noalloc(x.numel(), d, zeta, seed, x.data_ptr(), z.data_ptr(), stream)


def basis_product_f32(U, ldu: int, n: int, nin: int, Q: np.ndarray, out) -> None:
    """out = U Q on the tensor cores (split-BF16) for an FP32 basis.

    U, out: CUDA float32 tensors holding column-major n x nin / n x nout data
    with leading dimension ldu (out may be U); Q: nin x nout FP64 host array.
    """
    import torch
    Qf = np.asfortranarray(Q, dtype=np.float64)
    stream = torch.cuda.current_stream().cuda_stream
    _check(lib().rks_basis_product_f32(n, U.data_ptr(), ldu, nin, Qf.ctypes.data, Qf.shape[1], out.data_ptr(),
                                       stream), "rks_basis_product_f32")


QR_METHODS = {"rgs": 0, "whiten": 1, "rcholqr": 2, "rhqr": 3}


def sketch_qr(K, d: int, zeta: int = 8, seed: int = 0, method: str = "rgs", Q=None):
    """Randomized QR of a block (rks_sketch_qr).  K: CUDA float64 tensor of
    shape (s, n), row j = column j of the n x s block; Q (same shape, may be
    K) receives the orthogonal factor.  Returns (Q, R, S): R the s x s upper
    triangular factor, S = Omega Q (d x s), both host arrays."""
    import torch
    s, n = K.shape
    if Q is None:
        Q = torch.empty_like(K)
    R, S = _fortran((s, s)), _fortran((d, s))
    stream = torch.cuda.current_stream().cuda_stream
    _check(lib().rks_sketch_qr(n, s, K.data_ptr(), K.stride(0), d, zeta, int(seed) & 0xFFFFFFFFFFFFFFFF,
                               QR_METHODS[method], Q.data_ptr(), Q.stride(0), R.ctypes.data, S.ctypes.data,
                               stream), "rks_sketch_qr")
    return Q, R, S


def basis_product_df(U, ldu: int, n: int, nin: int, Q: np.ndarray, out) -> None:
    """out = U Q with the double-float restart's exact digit products on the
    tensor cores.  U, out: CUDA float64 tensors holding column-major n x nin /
    n x nout data with leading dimension ldu; Q: nin x nout FP64 host array.
    """
    import torch
    Qf = np.asfortranarray(Q, dtype=np.float64)
    stream = torch.cuda.current_stream().cuda_stream
    _check(lib().rks_basis_product_df(n, U.data_ptr(), ldu, nin, Qf.ctypes.data, Qf.shape[1], out.data_ptr(),
                                      stream), "rks_basis_product_df")


def host_ordered_schur(B: np.ndarray, which: str, nsort: int):
    m = B.shape[0]
    Bf = np.asfortranarray(B, dtype=np.float64)
    T, Q = _fortran((m, m)), _fortran((m, m))
    _check(lib().rks_host_ordered_schur(m, Bf.ctypes.data, WHICH[which], nsort, T.ctypes.data,
                                        Q.ctypes.data), "rks_host_ordered_schur")
    return T, Q


def host_reorder_select(T: np.ndarray, select):
    """Flagged diagonal blocks of quasi-triangular T first (rks_host_reorder_select):
    returns (T', Z) with T = Z T' Z^T."""
    n = T.shape[0]
    Tf = np.asfortranarray(T, dtype=np.float64).copy(order="F")
    Z = np.asfortranarray(np.eye(n))
    sel = np.ascontiguousarray(select, dtype=np.int32)
    _check(lib().rks_host_reorder_select(n, Tf.ctypes.data, sel.ctypes.data, Z.ctypes.data),
           "rks_host_reorder_select")
    return Tf, Z


def host_sketch_reorthonormalize(S: np.ndarray, T: np.ndarray, b: np.ndarray):
    """(Q, Rinv, Tn, bn) of rks_host_sketch_reorthonormalize for S = [Omega U, Omega u]."""
    d, kb = S.shape
    ka = kb - 1
    Sf = np.asfortranarray(S, dtype=np.float64).copy(order="F")
    Tf = np.asfortranarray(T, dtype=np.float64)
    bf = np.ascontiguousarray(b, dtype=np.float64)
    Rinv, Tn, bn = _fortran((kb, kb)), _fortran((ka, ka)), np.zeros(ka)
    _check(lib().rks_host_sketch_reorthonormalize(d, ka, Sf.ctypes.data, Tf.ctypes.data, bf.ctypes.data,
                                                  Rinv.ctypes.data, Tn.ctypes.data, bn.ctypes.data),
           "rks_host_sketch_reorthonormalize")
    return Sf, Rinv, Tn, bn


def host_quasi_eig(T: np.ndarray):
    n = T.shape[0]
    Tf = np.asfortranarray(T, dtype=np.float64)
    lre, lim = np.zeros(n), np.zeros(n)
    Yr, Yi = _fortran((n, n)), _fortran((n, n))
    _check(lib().rks_host_quasi_eig(n, Tf.ctypes.data, lre.ctypes.data, lim.ctypes.data,
                                    Yr.ctypes.data, Yi.ctypes.data), "rks_host_quasi_eig")
    return lre + 1j * lim, Yr + 1j * Yi


class Batch:
    """Independent problems solved concurrently (rks_create_batched).

    ``problems``: list of ``inputs.CSR`` (host arrays, one value type); the
    other arguments are shared and mean what they mean for ``Solver``.
    ``member(i)`` gives a Solver view of problem i (eigpairs, history, ...),
    valid while the batch lives.
    """

    def __init__(self, problems, k, p, d, which="LM", tol=1e-10, seed=0, *, nthreads=16, zeta=8, maxit=1000,
                 lock=True, eta_lock=0.0, conv="eig", verify=0.0, prec="df", keep=0, ortho="sketch",
                 aggressive=False):
        L = lib()
        self.count = len(problems)
        self._keep = [(_host(A.rowptr, np.int32), _host(A.colind, np.int32), np.ascontiguousarray(A.vals))
                      for A in problems]
        vdt = 0 if self._keep[0][2].dtype == np.float64 else 1
        if any((0 if a[2].dtype == np.float64 else 1) != vdt for a in self._keep):
            raise ValueError("all problems must share one value type")
        ns = np.array([A.n for A in problems], dtype=np.int64)
        ptrs = [np.array([a[j].ctypes.data for a in self._keep], dtype=np.uint64) for j in range(3)]
        self._arrays = (ns, *ptrs)
        o = Opts()
        L.rks_opts_default(C.byref(o))
        o.zeta, o.maxit, o.lock = int(zeta), int(maxit), int(bool(lock))
        o.eta_lock, o.conv, o.verify = float(eta_lock), CONV[conv], float(verify)
        o.prec, o.keep, o.ortho = PREC[prec], int(keep), ORTHO[ortho]
        o.aggressive = int(bool(aggressive))
        self.n = ns
        self.k, self.p, self.d = int(k), int(p), int(d)
        h = _P()
        _check(L.rks_create_batched(C.byref(h), self.count, ns.ctypes.data, ptrs[0].ctypes.data,
                                    ptrs[1].ctypes.data, ptrs[2].ctypes.data, vdt, self.k, self.p, self.d,
                                    WHICH[which] if isinstance(which, str) else int(which), float(tol),
                                    int(seed) & 0xFFFFFFFFFFFFFFFF, C.byref(o), int(nthreads)),
               "rks_create_batched")
        self._h = h

    def solve(self, nthreads=16, allow_noconv=True):
        infos = (Info * self.count)()
        rc = lib().rks_solve_batched(self._h, int(nthreads), C.cast(infos, _P))
        _check(rc, "rks_solve_batched", ok=(RKS_OK, RKS_ENOCONV) if allow_noconv else (RKS_OK,))
        out = []
        for i in range(self.count):
            d = infos[i].as_dict()
            d["status"] = STATUS.get(lib().rks_batch_status(self._h, i), None)
            out.append(d)
        return out

    def member(self, i) -> "Solver":
        s = Solver.__new__(Solver)
        s.n, s.k, s.p, s.d = int(self.n[i]), self.k, self.p, self.d
        s.device = False
        s._borrowed = True
        s._batch = self
        s._h = lib().rks_batch_get(self._h, int(i))
        if not s._h:
            raise IndexError(i)
        return s

    def close(self):
        if getattr(self, "_h", None):
            lib().rks_destroy_batched(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class DevBatch:
    """Independent problems solved by one persistent launch
    (rks_create_batched_dev): clusters of CTAs take problems from a device
    work queue and run the whole of Algorithm 1 for each on the device.

    ``problems``: list of ``inputs.CSR`` (host arrays, one value type).
    ``ctas``: CTAs per problem (1, 2, 4, 8) or 0 to pick the fastest by
    timing one restart of the batch.  Restarts keep max(k, min(keep, m // 2))
    Schur vectors and lock nothing; ``tol``, ``conv``, ``verify``, ``maxit``,
    ``zeta`` and ``seed`` mean what they mean for ``Solver``.
    """

    def __init__(self, problems, k, p, d, which="LM", tol=1e-10, seed=0, *, zeta=8, maxit=1000, conv="eig",
                 verify=0.0, keep=0, ctas=0, **ignored):
        L = lib()
        self.count = len(problems)
        self._keep = [(_host(A.rowptr, np.int32), _host(A.colind, np.int32), np.ascontiguousarray(A.vals))
                      for A in problems]
        vdt = 0 if self._keep[0][2].dtype == np.float64 else 1
        if any((0 if a[2].dtype == np.float64 else 1) != vdt for a in self._keep):
            raise ValueError("all problems must share one value type")
        ns = np.array([A.n for A in problems], dtype=np.int64)
        ptrs = [np.array([a[j].ctypes.data for a in self._keep], dtype=np.uint64) for j in range(3)]
        o = Opts()
        L.rks_opts_default(C.byref(o))
        o.zeta, o.maxit, o.conv, o.verify, o.keep = int(zeta), int(maxit), CONV[conv], float(verify), int(keep)
        self.n = ns
        self.k, self.p, self.d = int(k), int(p), int(d)
        h = _P()
        _check(L.rks_create_batched_dev(C.byref(h), self.count, ns.ctypes.data, ptrs[0].ctypes.data,
                                        ptrs[1].ctypes.data, ptrs[2].ctypes.data, vdt, self.k, self.p, self.d,
                                        WHICH[which] if isinstance(which, str) else int(which), float(tol),
                                        int(seed) & 0xFFFFFFFFFFFFFFFF, C.byref(o), int(ctas)),
               "rks_create_batched_dev")
        self._h = h
        self._keep = None

    def config(self) -> dict:
        """The launch configuration (front kernel: nL clusters of GL CTAs; back
        kernel: nS clusters of GS CTAs), the tuning times (ms, candidate order)
        and the last solve's event time."""
        cfg = (C.c_int * 4)()
        tune = (C.c_float * 16)()
        last = C.c_float()
        nt = lib().rks_dbatch_config(self._h, C.cast(cfg, _P), C.cast(tune, _P), 16, C.byref(last))
        _check(min(nt, 0), "rks_dbatch_config")
        return {"GL": cfg[0], "nL": cfg[1], "GS": cfg[2], "nS": cfg[3],
                "tune_ms": [float(tune[i]) for i in range(min(nt, 16))], "last_ms": float(last.value)}

    PHASES = ("start", "spmv_sketch", "hessenberg", "exchange", "ls", "update_sketch", "francis", "beta",
              "reorder", "kept_whiten", "restart", "ritz", "final", "queue")

    def phase_cycles(self) -> dict:
        """Cycle counts of the last solve by phase (summed over CTAs)."""
        buf = (C.c_int64 * len(self.PHASES))()
        nc = lib().rks_dbatch_phase_cycles(self._h, C.cast(buf, _P), len(self.PHASES))
        _check(min(nc, 0), "rks_dbatch_phase_cycles")
        return {name: int(buf[q]) for q, name in enumerate(self.PHASES[:nc])}

    def solve(self, allow_noconv=True):
        infos = (Info * self.count)()
        rc = lib().rks_solve_batched_dev(self._h, C.cast(infos, _P))
        _check(rc, "rks_solve_batched_dev", ok=(RKS_OK, RKS_ENOCONV) if allow_noconv else (RKS_OK,))
        out = []
        for i in range(self.count):
            d = infos[i].as_dict()
            d["status"] = STATUS.get(lib().rks_dbatch_status(self._h, i), None)
            out.append(d)
        return out

    def eigpairs(self, i, want_vectors=True):
        """(lam, X, resid, rq, est) of problem i: nw Ritz values (complex),
        X (n x nw complex, or None), FP64 residuals, Rayleigh quotients and
        estimates."""
        kk = self.k + 1
        a = [np.zeros(kk) for _ in range(6)]
        n = int(self.n[i])
        Xp = _fortran((n, kk)) if want_vectors else None
        nw = lib().rks_dbatch_eigpairs(self._h, int(i), *(x.ctypes.data for x in a),
                                       Xp.ctypes.data if Xp is not None else None)
        _check(min(nw, 0), "rks_dbatch_eigpairs")
        lre, lim, res, rqr, rqi, est = (x[:nw] for x in a)
        lam = lre + 1j * lim
        X = None
        if Xp is not None:
            X = np.zeros((n, nw), dtype=np.complex128)
            t = 0
            while t < nw:
                if lim[t] > 0 and t + 1 < nw:
                    X[:, t] = Xp[:, t] + 1j * Xp[:, t + 1]
                    X[:, t + 1] = Xp[:, t] - 1j * Xp[:, t + 1]
                    t += 2
                else:
                    X[:, t] = Xp[:, t]
                    t += 1
        return lam, X, res, rqr + 1j * rqi, est

    def close(self):
        if getattr(self, "_h", None):
            lib().rks_destroy_batched_dev(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def dev_ordered_schur(B: np.ndarray, which: str, nsort: int):
    """The device dense step (rks_dev_ordered_schur): T, Q with B = Q T Q^T,
    the best nsort blocks leading, and the eigenvalues / unit eigenvectors of T."""
    m = B.shape[0]
    Bf = np.asfortranarray(B, dtype=np.float64)
    T, Q, Yr, Yi = (_fortran((m, m)) for _ in range(4))
    lre, lim = np.zeros(m), np.zeros(m)
    _check(lib().rks_dev_ordered_schur(m, Bf.ctypes.data, WHICH[which], int(nsort), T.ctypes.data, Q.ctypes.data,
                                       lre.ctypes.data, lim.ctypes.data, Yr.ctypes.data, Yi.ctypes.data),
           "rks_dev_ordered_schur")
    return T, Q, lre + 1j * lim, Yr + 1j * Yi


class WarmStart:
    """The start-vector network (rks_ws_*): a 4-level U-Net from the
    coefficient planes (3 x H x W) of an operator to a start vector (H W).

    Inputs and outputs are CUDA float32 tensors; parameters are exchanged as
    host float32 arrays in the flat layout of ``include/rks.h``.
    """

    def __init__(self, H: int, W: int, seed: int = 0, stream=None):
        h = _P()
        _check(lib().rks_ws_create(C.byref(h), int(H), int(W), int(seed) & 0xFFFFFFFFFFFFFFFF, stream),
               "rks_ws_create")
        self._h, self.H, self.W = h, int(H), int(W)
        self.nparams = int(lib().rks_ws_nparams())

    def params(self) -> np.ndarray:
        out = np.zeros(self.nparams, dtype=np.float32)
        _check(lib().rks_ws_get_params(self._h, out.ctypes.data), "rks_ws_get_params")
        return out

    def set_params(self, theta) -> None:
        th = np.ascontiguousarray(theta, dtype=np.float32)
        if th.size != self.nparams:
            raise ValueError(f"expected {self.nparams} parameters, got {th.size}")
        _check(lib().rks_ws_set_params(self._h, th.ctypes.data), "rks_ws_set_params")

    @staticmethod
    def _need(t, shape, name):
        import torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA float32 tensor")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")

    def forward(self, x, out=None):
        import torch
        self._need(x, (3, self.H, self.W), "x")
        if out is None:
            out = torch.empty((self.H, self.W), dtype=torch.float32, device=x.device)
        self._need(out, (self.H, self.W), "out")
        _check(lib().rks_ws_forward(self._h, x.data_ptr(), out.data_ptr()), "rks_ws_forward")
        return out

    def accumulate(self, x, Q) -> float:
        """Add dL/dtheta for one sample; Q: CUDA float32 (q, H W), row j = column j of Q."""
        self._need(x, (3, self.H, self.W), "x")
        q = Q.shape[0]
        self._need(Q, (q, self.H * self.W), "Q")
        loss = C.c_double()
        _check(lib().rks_ws_accumulate(self._h, x.data_ptr(), Q.data_ptr(), int(q), C.byref(loss)),
               "rks_ws_accumulate")
        return loss.value

    def grad(self) -> np.ndarray:
        out = np.zeros(self.nparams, dtype=np.float32)
        _check(lib().rks_ws_get_grad(self._h, out.ctypes.data), "rks_ws_get_grad")
        return out

    def zero_grad(self) -> None:
        _check(lib().rks_ws_zero_grad(self._h), "rks_ws_zero_grad")

    def step(self, lr: float) -> None:
        _check(lib().rks_ws_adam_step(self._h, float(lr)), "rks_ws_adam_step")

    def start_vector(self, x, eps: float = 1e-3, seed: int = 1, out=None):
        """u1 = u / ||u|| + eps g / ||g|| (CUDA float64, H W) for rks_create's u1."""
        import torch
        self._need(x, (3, self.H, self.W), "x")
        if out is None:
            out = torch.empty(self.H * self.W, dtype=torch.float64, device=x.device)
        if not (out.is_cuda and out.dtype == torch.float64 and out.is_contiguous() and out.numel() == self.H * self.W):
            raise ValueError("out must be a contiguous CUDA float64 tensor of H W values")
        _check(lib().rks_ws_start_vector(self._h, x.data_ptr(), float(eps), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                         out.data_ptr()), "rks_ws_start_vector")
        return out

    def close(self):
        if getattr(self, "_h", None):
            lib().rks_ws_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
