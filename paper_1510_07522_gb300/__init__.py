"""Python binding of librsrr.so, the GB300 (sm_103a) resolvent-sampling Rayleigh-Ritz library.

Argument marshalling only: every step of RSRR runs in the library's CUDA kernels.  The
functions keep the C names (rsrr_create_nep, rsrr_sample, rsrr_project, rsrr_solve, ...);
`Nep` is a small convenience wrapper over them.  Importing works without a GPU (the
library only needs the CUDA runtime to load); calls that touch the device fail with
RsrrError when no device is present.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librsrr.so")

RSRR_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ESINGULAR", -4: "ENOTCONVERGED", -5: "ENONFINITE",
          -6: "ETIMEOUT", -7: "ECUDA", -8: "EORDER", -9: "EUNSUPPORTED"}
RSRR_FP64 = 0
RSRR_C64_IR = 1
RSRR_REFINE_FULL = 0x100
RSRR_NATURAL_ORDER = 0x1
RSRR_DENSE_LU = 0x2
RSRR_BAND_CUDA_CORES = 0x4
RSRR_AUTOTUNE = 0x8

F_CONST, F_Z, F_Z2, F_ISQRT_SHIFT, F_EXP_DELAY, F_RATIONAL, F_CALLBACK, F_CHEBYSHEV = range(8)


class RsrrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


# f(z) and f'(z) for m points: (user, m, z_reim, f_reim, df_reim)
RSRR_FN_CB = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double))


class rsrr_fn(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("p", ctypes.c_double * 4),
                ("cb", RSRR_FN_CB), ("user", ctypes.c_void_p)]


def callback_fn(f, df):
    """A RSRR_F_CALLBACK term from Python callables f(z) and df(z) on complex scalars.  Returns the
    (kind, params) pair that rsrr_create_nep / Nep take; the wrapper lives with the returned
    object, which the handle keeps."""
    def cb(user, m, z, fo, dfo):
        for k in range(m):
            zz = complex(z[2 * k], z[2 * k + 1])
            v, d = complex(f(zz)), complex(df(zz))
            fo[2 * k], fo[2 * k + 1] = v.real, v.imag
            dfo[2 * k], dfo[2 * k + 1] = d.real, d.imag
    return (F_CALLBACK, RSRR_FN_CB(cb))


class rsrr_contour(ctypes.Structure):
    _fields_ = [("gamma_re", ctypes.c_double), ("gamma_im", ctypes.c_double),
                ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("shape", ctypes.c_int32), ("side_nodes", ctypes.c_int32)]


RSRR_CONTOUR_ELLIPSE, RSRR_CONTOUR_RECTANGLE = 0, 1


def _contour(gamma, a, b, shape=RSRR_CONTOUR_ELLIPSE, side_nodes=0):
    return rsrr_contour(complex(gamma).real, complex(gamma).imag, float(a), float(b), int(shape), int(side_nodes))


class rsrr_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("J", ctypes.c_int32), ("N", ctypes.c_int32), ("L", ctypes.c_int32),
                ("kl", ctypes.c_int32), ("ku", ctypes.c_int32), ("natural_order", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("refine_sweeps", ctypes.c_int32),
                ("k_S", ctypes.c_int32), ("nbar", ctypes.c_int32),
                ("n_winding", ctypes.c_int32), ("n_gap", ctypes.c_int32),
                ("winding_re", ctypes.c_double), ("winding_im", ctypes.c_double),
                ("max_eta", ctypes.c_double),
                ("ms_sample", ctypes.c_double), ("ms_project", ctypes.c_double),
                ("ms_solve", ctypes.c_double), ("device_bytes", ctypes.c_int64),
                ("ms_factor", ctypes.c_double), ("ms_trsv", ctypes.c_double),
                ("factor_launches", ctypes.c_int32), ("trsv_launches", ctypes.c_int32),
                ("rows_kept", ctypes.c_int32), ("jacobi_sweeps_project", ctypes.c_int32),
                ("jacobi_sweeps_solve", ctypes.c_int32),
                ("ms_project_qr", ctypes.c_double), ("ms_project_svd", ctypes.c_double),
                ("ms_project_basis", ctypes.c_double), ("ms_project_gemm", ctypes.c_double),
                ("ms_solve_inverse", ctypes.c_double), ("ms_solve_svd", ctypes.c_double),
                ("ms_solve_extract", ctypes.c_double), ("ms_zgemm", ctypes.c_double),
                ("zgemm_gflop", ctypes.c_double), ("dense_lu", ctypes.c_int32),
                ("red_terms", ctypes.c_int32), ("proj_cols", ctypes.c_int32),
                ("ms_zgemm_tc", ctypes.c_double), ("zgemm_tc_gflop", ctypes.c_double),
                ("ms_jacobi", ctypes.c_double), ("jacobi_gflop", ctypes.c_double),
                ("band_lu_tc", ctypes.c_int32), ("tune_strategy", ctypes.c_int32),
                ("tune_band", ctypes.c_int32), ("tune_cached", ctypes.c_int32),
                ("iterative_band", ctypes.c_int32)]


_lib = None
EXPORTS = ["rsrr_create_nep", "rsrr_sample", "rsrr_project", "rsrr_solve", "rsrr_get_info",
           "rsrr_get_samples", "rsrr_get_eta", "rsrr_get_sigma", "rsrr_get_basis",
           "rsrr_get_projected", "rsrr_get_hankel_sigma", "rsrr_destroy", "rsrr_last_error",
           "rsrr_version", "rsrr_kernel_launches", "rsrr_band_solve_noalloc", "rsrr_sample_batch",
           "rsrr_project_moments", "rsrr_sample_points", "rsrr_project_chebyshev", "rsrr_create_nep_tz",
           "rsrr_zgemm", "rsrr_set_band_preconditioner", "rsrr_selftest_bounded_wait",
           "rsrr_device_peak_bytes", "rsrr_zinv_batch"]


def lib():
    """Load librsrr.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(or python -m paper_1510_07522_gb300._build)")
    L = ctypes.CDLL(LIB_PATH)
    P, I32, I64, D, U32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint32
    sig = {
        "rsrr_create_nep": ([I64, I32, P, P, P, P, U32, P, P], ctypes.c_int),
        "rsrr_sample": ([P, P, I32, I32, P, I32, D, I32], ctypes.c_int),
        "rsrr_project": ([P, D, P], ctypes.c_int),
        "rsrr_solve": ([P, I32, I32, D, I32, P, P, P, P], ctypes.c_int),
        "rsrr_get_info": ([P, P], ctypes.c_int),
        "rsrr_get_samples": ([P, I32, I32, P], ctypes.c_int),
        "rsrr_get_eta": ([P, P], ctypes.c_int),
        "rsrr_get_sigma": ([P, P], ctypes.c_int),
        "rsrr_get_basis": ([P, P], ctypes.c_int),
        "rsrr_get_projected": ([P, P], ctypes.c_int),
        "rsrr_get_hankel_sigma": ([P, P], ctypes.c_int),
        "rsrr_destroy": ([P], None),
        "rsrr_last_error": ([], ctypes.c_char_p),
        "rsrr_version": ([], ctypes.c_char_p),
        "rsrr_kernel_launches": ([], ctypes.c_int64),
        "rsrr_band_solve_noalloc": ([I64, I32, I32, P, I32, P, P], ctypes.c_int),
        "rsrr_sample_batch": ([P, I32, P, P, P, P, I32, D, I32], ctypes.c_int),
        "rsrr_project_moments": ([P, I32, D, P], ctypes.c_int),
        "rsrr_project_chebyshev": ([P, I32, D, D, D, P], ctypes.c_int),
        "rsrr_create_nep_tz": ([I64, P, P, RSRR_TZ_CB, P, U32, P, P], ctypes.c_int),
        "rsrr_zgemm": ([I32, I32, I32, I32, I32, I32, P, P, I64, I64, P, I64, I64, P, P, I64, I64, I32, P],
                       ctypes.c_int),
        "rsrr_set_band_preconditioner": ([P, I32], ctypes.c_int),
        "rsrr_selftest_bounded_wait": ([I32, P], ctypes.c_int),
        "rsrr_device_peak_bytes": ([I32], ctypes.c_int64),
        "rsrr_zinv_batch": ([I32, I32, I32, P, P, P], ctypes.c_int),
        "rsrr_sample_points": ([P, P, I32, P, I32, P, I32, D, I32], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(rc):
    if rc != RSRR_OK:
        raise RsrrError(rc, lib().rsrr_last_error().decode())


def _ptr(a):
    return None if a is None else a.ctypes.data


def _c128(a, shape=None, order="F"):
    a = np.asarray(a, dtype=np.complex128)
    if shape is not None:
        a = a.reshape(shape, order=order)
    return np.require(a, requirements=["F_CONTIGUOUS", "ALIGNED"] if order == "F" else ["C_CONTIGUOUS"])


def current_stream():
    """The caller's CUDA stream from PyTorch (None = the default stream)."""
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:  # noqa: BLE001 - torch is optional plumbing
        pass
    return None


# ---- the C entry points with their own names (marshalling only) ---------------------------
def rsrr_create_nep(n, rowptr, colind, vals, fns, flags=0, stream=None):
    """vals: complex [J, nnz] on the union CSR pattern; fns: list of (kind, params)."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.complex128)
    J = vals.shape[0]
    farr = (rsrr_fn * J)()
    for i, (kind, params) in enumerate(fns):
        farr[i].kind = int(kind)
        farr[i].reserved = 0
        if int(kind) == F_CALLBACK:
            farr[i].cb = params  # an RSRR_FN_CB from callback_fn
            continue
        p = list(params) + [0.0] * 4
        for t in range(4):
            farr[i].p[t] = float(p[t])
    h = ctypes.c_void_p()
    _check(lib().rsrr_create_nep(int(n), int(J), _ptr(rowptr), _ptr(colind), _ptr(vals), farr,
                                 int(flags), stream if stream is not None else current_stream(),
                                 ctypes.byref(h)))
    return h


# T(z) values for m points: (user, m, z_reim, vals_reim [m][nnz][2])
RSRR_TZ_CB = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_double))


def tz_callback(tz, nnz):
    """An RSRR_TZ_CB from a Python callable tz(z) -> complex values [nnz] of T(z) on the pattern."""
    def cb(user, m, z, out):
        buf = np.ctypeslib.as_array(out, shape=(int(m) * nnz * 2,)).view(np.complex128).reshape(int(m), nnz)
        for k in range(m):
            buf[k] = tz(complex(z[2 * k], z[2 * k + 1]))
    return RSRR_TZ_CB(cb)


def rsrr_create_nep_tz(n, rowptr, colind, cb, flags=0, stream=None):
    """cb: an RSRR_TZ_CB (see tz_callback); the caller keeps it alive with the handle."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(lib().rsrr_create_nep_tz(int(n), _ptr(rowptr), _ptr(colind), cb, None, int(flags),
                                    stream if stream is not None else current_stream(), ctypes.byref(h)))
    return h


def rsrr_sample(h, gamma, a, b, N, L, U=None, precision=RSRR_FP64, tol=1e-10, max_refine=10,
                shape=RSRR_CONTOUR_ELLIPSE, side_nodes=0):
    C = _contour(gamma, a, b, shape, side_nodes)
    Uc = None if U is None else _c128(U)
    _check(lib().rsrr_sample(h, ctypes.byref(C), int(N), int(L), _ptr(Uc), int(precision), float(tol),
                             int(max_refine)))


def rsrr_sample_batch(handles, contours, Ns, Ls, Us=None, precision=RSRR_FP64, tol=1e-10, max_refine=10):
    """rsrr_sample for several handles in one call (contours: list of (gamma, a, b) or
    (gamma, a, b, shape, side_nodes))."""
    count = len(handles)
    H = (ctypes.c_void_p * count)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    C = (rsrr_contour * count)()
    for i, c in enumerate(contours):
        C[i] = _contour(*c)
    Narr = (ctypes.c_int32 * count)(*[int(x) for x in Ns])
    Larr = (ctypes.c_int32 * count)(*[int(x) for x in Ls])
    keep = []
    Uarr = None
    if Us is not None:
        Uarr = (ctypes.c_void_p * count)()
        for i, U in enumerate(Us):
            if U is not None:
                Uc = _c128(U)
                keep.append(Uc)
                Uarr[i] = Uc.ctypes.data
    _check(lib().rsrr_sample_batch(H, count, C, Narr, Larr, Uarr, int(precision), float(tol), int(max_refine)))
    del keep


def rsrr_sample_points(h, gamma, a, b, z, L, U=None, precision=RSRR_FP64, tol=1e-10, max_refine=10,
                       shape=RSRR_CONTOUR_ELLIPSE):
    """rsrr_sample at the points z (complex array); (gamma, a, b, shape) is the contour for rsrr_solve."""
    C = _contour(gamma, a, b, shape)
    zr = np.ascontiguousarray(np.asarray(z, dtype=np.complex128))
    Uc = None if U is None else _c128(U)
    _check(lib().rsrr_sample_points(h, ctypes.byref(C), int(zr.size), _ptr(zr), int(L), _ptr(Uc), int(precision),
                                    float(tol), int(max_refine)))


def zgemm(path, A, B, C, opA=0, opB=0, alpha=1.0, beta=0.0, M=None, N=None, K=None, batch=1, strides=(0, 0, 0),
          lds=None, stream=None):
    """rsrr_zgemm on device buffers A, B, C (objects with data_ptr(), complex128, column-major with
    leading dimensions `lds` = (lda, ldb, ldc)); C = alpha op(A) op(B) + beta C."""
    al = (ctypes.c_double * 2)(complex(alpha).real, complex(alpha).imag)
    be = (ctypes.c_double * 2)(complex(beta).real, complex(beta).imag)
    lda, ldb, ldc = lds
    _check(lib().rsrr_zgemm(int(path), int(opA), int(opB), int(M), int(N), int(K), al,
                            ctypes.c_void_p(A.data_ptr()), int(lda), int(strides[0]),
                            ctypes.c_void_p(B.data_ptr()), int(ldb), int(strides[1]), be,
                            ctypes.c_void_p(C.data_ptr()), int(ldc), int(strides[2]), int(batch),
                            stream if stream is not None else current_stream()))


def zinv_batch(path, A, info, k, batch, stream=None):
    """rsrr_zinv_batch: A (device, batch consecutive k x k complex128 column-major matrices) is
    replaced by its inverse; info (device int32 [batch]) flags matrices with a zero pivot."""
    _check(lib().rsrr_zinv_batch(int(path), int(k), int(batch), ctypes.c_void_p(A.data_ptr()),
                                 ctypes.c_void_p(info.data_ptr()),
                                 stream if stream is not None else current_stream()))


def rsrr_project_chebyshev(h, d, x_lo, x_hi, delta=1e-14):
    k = ctypes.c_int32()
    _check(lib().rsrr_project_chebyshev(h, int(d), float(x_lo), float(x_hi), float(delta), ctypes.byref(k)))
    return k.value


def rsrr_project_moments(h, Kp, delta=1e-14):
    k = ctypes.c_int32()
    _check(lib().rsrr_project_moments(h, int(Kp), float(delta), ctypes.byref(k)))
    return k.value


def rsrr_project(h, delta=1e-14):
    k = ctypes.c_int32()
    _check(lib().rsrr_project(h, float(delta), ctypes.byref(k)))
    return k.value


def rsrr_solve(h, N_S=500, K=2, tol_gap=1e3, cap=None, n=None, vectors=True):
    if cap is None:
        cap = 4096
    lam = np.zeros(cap, dtype=np.complex128)
    V = np.zeros((n, cap), dtype=np.complex128, order="F") if (vectors and n) else None
    res = np.zeros(cap)
    nC = ctypes.c_int32()
    _check(lib().rsrr_solve(h, int(N_S), int(K), float(tol_gap), int(cap), _ptr(lam), _ptr(V), _ptr(res),
                            ctypes.byref(nC)))
    k = nC.value
    return lam[:k].copy(), (None if V is None else V[:, :k].copy()), res[:k].copy()


def rsrr_get_info(h):
    info = rsrr_info()
    _check(lib().rsrr_get_info(h, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in rsrr_info._fields_}


def rsrr_band_solve_noalloc(n, kl, ku, ab_ptr, L, b_ptr, stream=None):
    """Band LU + solve of one system from device pointers, using only the library's fixed
    scratch array (no device allocation); see rsrr.h."""
    _check(lib().rsrr_band_solve_noalloc(int(n), int(kl), int(ku), ctypes.c_void_p(ab_ptr), int(L),
                                         ctypes.c_void_p(b_ptr),
                                         stream if stream is not None else current_stream()))


def rsrr_selftest_bounded_wait(kind, stream=None):
    """Run one bounded device wait made to run out (kind 0: grid barrier, 1: mbarrier) or to
    complete (2, 3); raises RsrrError('ETIMEOUT') when the wait gave up."""
    _check(lib().rsrr_selftest_bounded_wait(int(kind), ctypes.c_void_p(stream) if stream else None))


def rsrr_destroy(h):
    if h:
        lib().rsrr_destroy(h)


def sample_batch(neps, contours, Ns, Ls, Us=None, precision=RSRR_FP64, tol=1e-10, max_refine=10):
    """rsrr_sample_batch over Nep objects (all created on one stream)."""
    rsrr_sample_batch([p.h for p in neps], contours, Ns, Ls, Us, precision, tol, max_refine)
    for p, N, L in zip(neps, Ns, Ls):
        p.N, p.L = int(N), int(L)


class Nep:
    """Handle for T(z) = sum_i f_i(z) A_i on the device (rsrr_create_nep ... rsrr_destroy)."""

    def __init__(self, n, rowptr, colind, vals, fns, flags=0, stream=None):
        self.n = int(n)
        self.J = int(np.asarray(vals).shape[0])
        self._fns = list(fns)  # keeps RSRR_F_CALLBACK wrappers alive as long as the handle
        self.h = rsrr_create_nep(n, rowptr, colind, vals, self._fns, flags, stream)

    @classmethod
    def from_tz(cls, n, rowptr, colind, tz, flags=0, stream=None):
        """rsrr_create_nep_tz: T known only by tz(z) -> complex values [nnz] on the pattern."""
        self = cls.__new__(cls)
        self.n, self.J = int(n), 0
        self._fns = [tz_callback(tz, int(np.asarray(colind).size))]
        self.h = rsrr_create_nep_tz(n, rowptr, colind, self._fns[0], flags, stream)
        return self

    def sample(self, gamma, a, b, N, L, U=None, precision=RSRR_FP64, tol=1e-10, max_refine=10,
               shape=RSRR_CONTOUR_ELLIPSE, side_nodes=0):
        self.N, self.L = int(N), int(L)
        rsrr_sample(self.h, gamma, a, b, N, L, U, precision, tol, max_refine, shape, side_nodes)

    def project(self, delta=1e-14):
        self.kS = rsrr_project(self.h, delta)
        return self.kS

    def sample_points(self, gamma, a, b, z, L, U=None, precision=RSRR_FP64, tol=1e-10, max_refine=10,
                      shape=RSRR_CONTOUR_ELLIPSE):
        """rsrr_sample_points: sample at the points z, keep the contour for rsrr_solve."""
        self.N, self.L = int(np.asarray(z).size), int(L)
        rsrr_sample_points(self.h, gamma, a, b, z, L, U, precision, tol, max_refine, shape)

    def project_moments(self, Kp, delta=1e-14):
        """The SSRR moment scheme: rsrr_project on K' quadrature moments of the samples."""
        self.kS = rsrr_project_moments(self.h, Kp, delta)
        return self.kS

    def set_band_preconditioner(self, band):
        """rsrr_set_band_preconditioner: factor only |i - j| <= band and iterate (-1 = off)."""
        _check(lib().rsrr_set_band_preconditioner(self.h, int(band)))

    def project_chebyshev(self, d, x_lo, x_hi, delta=1e-14):
        """rsrr_project, then the reduced NEP as its degree-d Chebyshev interpolant on [x_lo, x_hi]."""
        self.kS = rsrr_project_chebyshev(self.h, d, x_lo, x_hi, delta)
        return self.kS

    def solve(self, N_S=500, K=2, tol_gap=1e3, cap=4096, vectors=True):
        return rsrr_solve(self.h, N_S, K, tol_gap, cap, self.n, vectors)

    def info(self):
        return rsrr_get_info(self.h)

    def samples(self, j0=0, j1=None):
        j1 = self.N if j1 is None else j1
        out = np.zeros((self.n, (j1 - j0) * self.L), dtype=np.complex128, order="F")
        _check(lib().rsrr_get_samples(self.h, int(j0), int(j1), _ptr(out)))
        return out

    def eta(self):
        out = np.zeros(self.N * self.L)
        _check(lib().rsrr_get_eta(self.h, _ptr(out)))
        return out

    def sigma(self):
        out = np.zeros(min(self.n, self.info()["proj_cols"]))
        _check(lib().rsrr_get_sigma(self.h, _ptr(out)))
        return out

    def basis(self):
        out = np.zeros((self.n, self.kS), dtype=np.complex128, order="F")
        _check(lib().rsrr_get_basis(self.h, _ptr(out)))
        return out

    def projected(self):
        out = np.zeros((self.info()["red_terms"], self.kS, self.kS), dtype=np.complex128)
        _check(lib().rsrr_get_projected(self.h, _ptr(out)))
        # stored column-major per term
        return np.ascontiguousarray(np.transpose(out, (0, 2, 1)))

    def hankel_sigma(self, K):
        out = np.zeros(K * self.kS)
        _check(lib().rsrr_get_hankel_sigma(self.h, _ptr(out)))
        return out

    def close(self):
        if getattr(self, "h", None):
            rsrr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
