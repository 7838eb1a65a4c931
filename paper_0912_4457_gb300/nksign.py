"""ctypes binding of the C ABI in include/nksign.h (argument marshalling only).

Every function here has the name of the C entry point without the ``nk_``
prefix and forwards to ``libnksign.so``; all arithmetic of the method runs in
the library's CUDA kernels.  Device arrays are passed as torch CUDA tensors
(complex128, contiguous) and the current torch stream is used unless one is
given.  There is no CPU fallback: if the library is not built, or no GPU is
present, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnksign.so")

NK_OK = 0
NK_EINVAL = -1
NK_ENOMEM = -2
NK_EBREAKDOWN = -3
NK_ENOTCONV = -4
NK_ERHI = -5
NK_ECUDA = -6
NK_ETIMEOUT = -7
NK_ESTATE = -8

NK_FP64 = 0x0
NK_MIXED = 0x1
NK_DOUBLE_PASS = 0x2
NK_NO_GRAPH = 0x10
NK_PROFILE = 0x20
NK_ASYNC = 0x40
NK_SHARED_P = 0x80
NK_PREFIX_FP64 = 0x100
NK_EPS_EST = 0x200
NK_PREDICT = 0x400
NK_MAX_RHS = 12
NK_NCLASS = 9
CLASS_NAMES = ["dslash", "dslash_df", "step2", "dslash64", "inner", "rhi", "lift", "other", "step2_df"]

ERROR_NAMES = {
    NK_EINVAL: "NK_EINVAL", NK_ENOMEM: "NK_ENOMEM", NK_EBREAKDOWN: "NK_EBREAKDOWN",
    NK_ENOTCONV: "NK_ENOTCONV", NK_ERHI: "NK_ERHI", NK_ECUDA: "NK_ECUDA",
    NK_ETIMEOUT: "NK_ETIMEOUT", NK_ESTATE: "NK_ESTATE",
}

EXPORTED = [
    "nk_create_lattice", "nk_load_links", "nk_load_links_dev", "nk_set_mu_mw", "nk_set_precision", "nk_set_df_recurrence",
    "nk_set_adapt_start", "nk_set_nesting", "nk_set_deflation", "nk_eigs_smallest", "nk_overlap_solve",
    "nk_sign_apply", "nk_sign_apply_dev", "nk_overlap_apply", "nk_overlap_apply_dev",
    "nk_dslash_dev", "nk_stencil32_dev", "nk_outer_lanczos_dev", "nk_inner_sign", "nk_inner_sign_noalloc", "nk_last_error",
    "nk_destroy",
    "nk_mlp_create", "nk_mlp_set_norm", "nk_mlp_set_weight_decay", "nk_mlp_get_params", "nk_mlp_set_params", "nk_mlp_loss_grad",
    "nk_mlp_train", "nk_mlp_forward", "nk_mlp_last_error", "nk_mlp_destroy", "nk_features",
    "nk_predict_sizes", "nk_set_predictor", "nk_set_launch", "nk_get_launch", "nk_autotune", "nk_wait",
]

NK_MLP_IN = 16
NK_MLP_HIDDEN = 64
NK_MLP_OUT = 2
NK_MLP_PARAMS = 64 * 16 + 64 + 64 * 64 + 64 + 2 * 64 + 2


class NkStats(ctypes.Structure):
    _fields_ = [
        ("n_rhs", ctypes.c_int),
        ("k_used", ctypes.c_int),
        ("k_rhs", ctypes.c_int * NK_MAX_RHS),
        ("checks", ctypes.c_int),
        ("ell_used", ctypes.c_int),
        ("rhi_iters", ctypes.c_int * NK_MAX_RHS),
        ("status", ctypes.c_int * NK_MAX_RHS),
        ("p", ctypes.c_double * NK_MAX_RHS),
        ("z_min", ctypes.c_double * NK_MAX_RHS),
        ("z_max", ctypes.c_double * NK_MAX_RHS),
        ("xnorm", ctypes.c_double * NK_MAX_RHS),
        ("t_total_ms", ctypes.c_double),
        ("launches", ctypes.c_int),
        ("t_class_ms", ctypes.c_double * NK_NCLASS),
        ("n_class", ctypes.c_int * NK_NCLASS),
        ("t_basis_ms", ctypes.c_double),
        ("t_inner_ms", ctypes.c_double),
        ("t_lift_ms", ctypes.c_double),
        ("eps_sgn2", ctypes.c_double * NK_MAX_RHS),
        ("k_pred", ctypes.c_int),
        ("ell_pred", ctypes.c_int),
        ("predict_fallback", ctypes.c_int),
        ("defl_m", ctypes.c_int),
        ("defl_gap", ctypes.c_double),
    ]

    def as_dict(self):
        n = self.n_rhs
        return {
            "n_rhs": n, "k_used": self.k_used, "k_rhs": list(self.k_rhs[:n]), "checks": self.checks,
            "ell_used": self.ell_used,
            "rhi_iters": list(self.rhi_iters[:n]), "status": list(self.status[:n]),
            "p": list(self.p[:n]), "z_min": list(self.z_min[:n]), "z_max": list(self.z_max[:n]),
            "xnorm": list(self.xnorm[:n]), "t_total_ms": self.t_total_ms,
            "launches": self.launches,
            "t_class_ms": dict(zip(CLASS_NAMES, list(self.t_class_ms))),
            "n_class": dict(zip(CLASS_NAMES, list(self.n_class))),
            "t_basis_ms": self.t_basis_ms, "t_inner_ms": self.t_inner_ms, "t_lift_ms": self.t_lift_ms,
            "eps_sgn2": list(self.eps_sgn2[:n]), "k_pred": self.k_pred, "ell_pred": self.ell_pred,
            "predict_fallback": bool(self.predict_fallback),
            "defl_m": self.defl_m, "defl_gap": self.defl_gap,
        }


class NkLaunch(ctypes.Structure):
    _fields_ = [("stencil_threads", ctypes.c_int), ("stencil_order", ctypes.c_int), ("step2_blocks", ctypes.c_int),
                ("early_threads", ctypes.c_int), ("early_order", ctypes.c_int), ("stencil_split", ctypes.c_int),
                ("early_split", ctypes.c_int)]

    def as_tuple(self):
        return (self.stencil_threads, self.stencil_order, self.step2_blocks, self.early_threads, self.early_order,
                self.stencil_split, self.early_split)


class NkError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERROR_NAMES.get(code, "NK_?"), code, msg))
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libnksign.so (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libnksign.so is not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    P, I, D, U = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint
    dp = ctypes.POINTER(ctypes.c_double)
    fp = ctypes.POINTER(ctypes.c_float)
    sig = {
        "nk_create_lattice": ([ctypes.POINTER(ctypes.c_int), I, ctypes.POINTER(P)], I),
        "nk_load_links": ([P, dp], I),
        "nk_load_links_dev": ([P, P, P], I),
        "nk_set_mu_mw": ([P, D, D], I),
        "nk_set_precision": ([P, I], I),
        "nk_set_df_recurrence": ([P, I], I),
        "nk_set_adapt_start": ([P, I], I),
        "nk_set_nesting": ([P, I, P], I),
        "nk_set_deflation": ([P, I, P, P, P], I),
        "nk_eigs_smallest": ([P, dp, I, I, D, dp, dp, P, P, P], I),
        "nk_overlap_solve": ([P, P, I, I, I, ctypes.c_double, U, ctypes.c_double, ctypes.c_double, I, P, P, P], I),
        "nk_sign_apply": ([P, dp, I, I, I, D, D, U, dp, ctypes.POINTER(NkStats)], I),
        "nk_sign_apply_dev": ([P, P, I, I, I, D, D, U, P, ctypes.POINTER(NkStats), P], I),
        "nk_overlap_apply": ([P, dp, I, I, I, D, U, dp, ctypes.POINTER(NkStats)], I),
        "nk_overlap_apply_dev": ([P, P, I, I, I, D, U, P, ctypes.POINTER(NkStats), P], I),
        "nk_dslash_dev": ([P, P, P, I, I, I, P], I),
        "nk_stencil32_dev": ([P, P, P, I, P], I),
        "nk_outer_lanczos_dev": ([P, P, I, I, U, dp, dp, dp, dp, P], I),
        "nk_inner_sign": ([P, dp, dp, dp, I, I, I, D, I, dp, ctypes.POINTER(NkStats)], I),
        "nk_inner_sign_noalloc": ([P, P, P, I, I, I, D, I, P, P, ctypes.c_char_p, ctypes.c_size_t], I),
        "nk_last_error": ([P], ctypes.c_char_p),
        "nk_destroy": ([P], None),
        "nk_mlp_create": ([ctypes.c_ulonglong, ctypes.POINTER(P)], I),
        "nk_mlp_set_norm": ([P, fp, fp, fp, fp], I),
        "nk_mlp_set_weight_decay": ([P, ctypes.c_float], I),
        "nk_mlp_get_params": ([P, fp], I),
        "nk_mlp_set_params": ([P, fp], I),
        "nk_mlp_loss_grad": ([P, fp, fp, I, fp, fp], I),
        "nk_mlp_train": ([P, fp, fp, I, I, ctypes.c_float, fp], I),
        "nk_mlp_forward": ([P, fp, I, fp], I),
        "nk_mlp_last_error": ([P], ctypes.c_char_p),
        "nk_mlp_destroy": ([P], None),
        "nk_features": ([P, P, fp, P], I),
        "nk_predict_sizes": ([P, P, P, I, ctypes.POINTER(I), ctypes.POINTER(I), P], I),
        "nk_set_predictor": ([P, P], I),
        "nk_set_launch": ([P, I, U, ctypes.POINTER(NkLaunch)], I),
        "nk_get_launch": ([P, I, U, ctypes.POINTER(NkLaunch)], I),
        "nk_autotune": ([P, I, U, ctypes.c_char_p, ctypes.POINTER(NkLaunch), dp], I),
        "nk_wait": ([P, ctypes.POINTER(NkStats)], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _host_c128(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _dev_ptr(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if t.dtype not in (torch.complex128, torch.float64):
        raise TypeError("tensor must be complex128 (or float64 with interleaved re/im)")
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """Owns an nk_ctx*; each method maps to one C entry point."""

    def __init__(self, dims, bc_t_antiperiodic: bool = True):
        lib = load_library()
        self._lib = lib
        d = (ctypes.c_int * 4)(*[int(x) for x in dims])
        h = ctypes.c_void_p()
        rc = lib.nk_create_lattice(d, 1 if bc_t_antiperiodic else 0, ctypes.byref(h))
        if rc != NK_OK:
            raise NkError(rc, "nk_create_lattice failed (no CUDA device or bad dims)")
        self.h = h
        self.dims = tuple(int(x) for x in dims)
        self.V = int(np.prod(self.dims))
        self.N = 12 * self.V

    def _check(self, rc):
        if rc != NK_OK:
            raise NkError(rc, self._lib.nk_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self._lib.nk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- setup ------------------------------------------------------------
    def load_links(self, U: np.ndarray):
        u = _host_c128(U).reshape(-1)
        if u.size != 36 * self.V:
            raise ValueError("links must have 36*V complex entries")
        self._check(self._lib.nk_load_links(self.h, _dptr(u.view(np.float64))))

    def load_links_dev(self, U_dev, stream=None):
        self._check(self._lib.nk_load_links_dev(self.h, _dev_ptr(U_dev), _stream_ptr(stream)))

    def set_mu_mw(self, mu: float, m_w: float):
        self._check(self._lib.nk_set_mu_mw(self.h, float(mu), float(m_w)))

    def set_precision(self, j0: int):
        self._check(self._lib.nk_set_precision(self.h, int(j0)))

    def set_df_recurrence(self, j1: int):
        self._check(self._lib.nk_set_df_recurrence(self.h, int(j1)))

    def set_adapt_start(self, k_first: int):
        self._check(self._lib.nk_set_adapt_start(self.h, int(k_first)))

    def overlap_solve(self, b, k, ell, mass=0.0, tol_cg=1e-8, maxit=500, tol_sign=0.0, flags=NK_FP64, check=True):
        """nk_overlap_solve: x = (D_ov + mass)^-1 b by CG on the normal
        equations; returns (x, iterations, relative residuals, rc)."""
        b = _host_c128(b)
        if b.ndim == 1:
            b = b[None, :]
        n = b.shape[0]
        x = np.zeros_like(b)
        its = np.zeros(n, np.int32)
        res = np.zeros(n)
        rc = self._lib.nk_overlap_solve(self.h, _dptr(b.view(np.float64)), n, int(k), int(ell), float(tol_sign),
                                        int(flags), float(mass), float(tol_cg), int(maxit),
                                        _dptr(x.view(np.float64)), its.ctypes.data_as(ctypes.c_void_p), _dptr(res))
        if check:
            self._check(rc)
        return x, its, res, rc

    def set_deflation(self, lam=None, R=None, L=None):
        """nk_set_deflation: eigenvalues lam (m,), right eigenvectors R (m, 12 V)
        and left eigenvectors L (m, 12 V) with <l_i, r_j> = delta_ij, or None
        (Hermitian: L = R); lam=None switches deflation off."""
        if lam is None or len(lam) == 0:
            self._check(self._lib.nk_set_deflation(self.h, 0, None, None, None))
            return
        lam = np.ascontiguousarray(lam, dtype=np.complex128)
        R = np.ascontiguousarray(R, dtype=np.complex128).reshape(len(lam), self.N)
        Lp = None
        if L is not None:
            L = np.ascontiguousarray(L, dtype=np.complex128).reshape(len(lam), self.N)
            Lp = _dptr(L.view(np.float64))
        self._check(self._lib.nk_set_deflation(self.h, len(lam), _dptr(lam.view(np.float64)),
                                               _dptr(R.view(np.float64)), Lp))

    def eigs_smallest(self, b, k, m, tol=1e-10, check=True):
        """nk_eigs_smallest: the m eigenpairs of A of smallest |lambda| from a
        k-step Lanczos eigensolver started at b (12 V complex).  Returns
        (lam (found,), R (found, 12 V), L (found, 12 V), resid (found,), rc);
        L = R at mu = 0.  With check, rc != NK_OK raises."""
        b = _host_c128(b).reshape(self.N)
        lam = np.zeros(m, np.complex128)
        R = np.zeros((m, self.N), np.complex128)
        L = np.zeros((m, self.N), np.complex128)
        res = np.zeros(m)
        found = ctypes.c_int(0)
        rc = self._lib.nk_eigs_smallest(self.h, _dptr(b.view(np.float64)), int(k), int(m), float(tol),
                                        _dptr(lam.view(np.float64)), _dptr(R.view(np.float64)),
                                        L.ctypes.data_as(ctypes.c_void_p), res.ctypes.data_as(ctypes.c_void_p),
                                        ctypes.byref(found))
        if check:
            self._check(rc)
        n = found.value
        return lam[:n], R[:n], L[:n], res[:n], rc

    def set_nesting(self, ells=()):
        """nk_set_nesting: sizes l_2 >= l_3 >= ... of the levels below the first
        (multi-level nesting, Sec. 4.5); () restores one level."""
        arr = (ctypes.c_int * max(1, len(ells)))(*[int(v) for v in ells])
        self._check(self._lib.nk_set_nesting(self.h, len(ells), arr if len(ells) else None))

    # -- solves (host arrays) --------------------------------------------------
    def sign_apply(self, b, k, ell, tol=0.0, p=0.0, flags=NK_FP64, check=True):
        b = _host_c128(b)
        if b.ndim == 1:
            b = b[None, :]
        n = b.shape[0]
        y = np.zeros_like(b)
        st = NkStats()
        rc = self._lib.nk_sign_apply(self.h, _dptr(b.view(np.float64)), n, int(k), int(ell), float(tol),
                                     float(p), int(flags), _dptr(y.view(np.float64)), ctypes.byref(st))
        if check:
            self._check(rc)
        return y, st.as_dict(), rc

    def overlap_apply(self, b, k, ell, tol=0.0, flags=NK_FP64, check=True):
        b = _host_c128(b)
        if b.ndim == 1:
            b = b[None, :]
        n = b.shape[0]
        y = np.zeros_like(b)
        st = NkStats()
        rc = self._lib.nk_overlap_apply(self.h, _dptr(b.view(np.float64)), n, int(k), int(ell), float(tol),
                                        int(flags), _dptr(y.view(np.float64)), ctypes.byref(st))
        if check:
            self._check(rc)
        return y, st.as_dict(), rc

    # -- solves (device tensors) -----------------------------------------------
    def sign_apply_dev(self, b_dev, y_dev, n_rhs, k, ell, tol=0.0, p=0.0, flags=NK_FP64, stream=None,
                       check=True):
        st = NkStats()
        rc = self._lib.nk_sign_apply_dev(self.h, _dev_ptr(b_dev), int(n_rhs), int(k), int(ell), float(tol),
                                         float(p), int(flags), _dev_ptr(y_dev), ctypes.byref(st),
                                         _stream_ptr(stream))
        if check:
            self._check(rc)
        return st.as_dict(), rc

    def wait(self, check=True):
        """nk_wait: collect the pending NK_ASYNC solve (statistics dict, rc)."""
        st = NkStats()
        rc = self._lib.nk_wait(self.h, ctypes.byref(st))
        if check:
            self._check(rc)
        return st.as_dict(), rc

    def overlap_apply_dev(self, b_dev, y_dev, n_rhs, k, ell, tol=0.0, flags=NK_FP64, stream=None):
        st = NkStats()
        rc = self._lib.nk_overlap_apply_dev(self.h, _dev_ptr(b_dev), int(n_rhs), int(k), int(ell),
                                            float(tol), int(flags), _dev_ptr(y_dev), ctypes.byref(st),
                                            _stream_ptr(stream))
        self._check(rc)
        return st.as_dict()

    # -- single steps ---------------------------------------------------------
    def dslash_dev(self, in_dev, out_dev, n_vec, dagger=False, precision=64, stream=None):
        self._check(self._lib.nk_dslash_dev(self.h, _dev_ptr(in_dev), _dev_ptr(out_dev), int(n_vec),
                                            1 if dagger else 0, int(precision), _stream_ptr(stream)))

    def stencil32_dev(self, in_dev, out_dev, n_rhs, stream=None):
        """nk_stencil32_dev: A on the first n_rhs and A^dagger on the next n_rhs
        FP32 vectors of in_dev (pair layout, 24 V floats per vector) -> out_dev."""
        import torch
        for t in (in_dev, out_dev):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous() and t.dtype == torch.float32):
                raise TypeError("expected contiguous float32 CUDA tensors")
            if t.numel() < 2 * int(n_rhs) * 24 * self.V:
                raise ValueError("tensor holds fewer than 2 n_rhs vectors")
        self._check(self._lib.nk_stencil32_dev(self.h, ctypes.c_void_p(in_dev.data_ptr()),
                                               ctypes.c_void_p(out_dev.data_ptr()), int(n_rhs),
                                               _stream_ptr(stream)))

    def outer_lanczos_dev(self, b_dev, n_rhs, k, flags=NK_FP64, stream=None):
        a = np.zeros((n_rhs, k), np.complex128)
        be = np.zeros((n_rhs, k), np.complex128)
        ga = np.zeros((n_rhs, k), np.complex128)
        xn = np.zeros(n_rhs)
        self._check(self._lib.nk_outer_lanczos_dev(
            self.h, _dev_ptr(b_dev), int(n_rhs), int(k), int(flags), _dptr(a.view(np.float64)),
            _dptr(be.view(np.float64)), _dptr(ga.view(np.float64)), _dptr(xn), _stream_ptr(stream)))
        return a, be, ga, xn

    def inner_sign(self, alpha, beta, gamma, ell, p=0.0, hermitian=True, check=True):
        alpha = _host_c128(alpha)
        if alpha.ndim == 1:
            alpha = alpha[None, :]
        n, k = alpha.shape
        beta = _host_c128(beta, (n, k)) if np.asarray(beta).size == n * k else _pad(beta, n, k)
        gamma = _host_c128(gamma, (n, k)) if np.asarray(gamma).size == n * k else _pad(gamma, n, k)
        c = np.zeros((n, k), np.complex128)
        st = NkStats()
        rc = self._lib.nk_inner_sign(self.h, _dptr(alpha.view(np.float64)), _dptr(beta.view(np.float64)),
                                     _dptr(gamma.view(np.float64)), n, k, int(ell), float(p),
                                     1 if hermitian else 0, _dptr(c.view(np.float64)), ctypes.byref(st))
        if check:
            self._check(rc)
        return c, st.as_dict(), rc

    # -- launch shape / autotuner -------------------------------------------
    def set_launch(self, n_rhs, flags, stencil_threads, stencil_order, step2_blocks, early_threads=128,
                   early_order=0, stencil_split=1, early_split=1):
        lc = NkLaunch(int(stencil_threads), int(stencil_order), int(step2_blocks), int(early_threads),
                      int(early_order), int(stencil_split), int(early_split))
        self._check(self._lib.nk_set_launch(self.h, int(n_rhs), int(flags), ctypes.byref(lc)))

    def get_launch(self, n_rhs, flags=NK_FP64):
        lc = NkLaunch()
        self._check(self._lib.nk_get_launch(self.h, int(n_rhs), int(flags), ctypes.byref(lc)))
        return lc.as_tuple()

    def autotune(self, n_rhs, flags=NK_FP64, cache_path=None):
        """nk_autotune: returns ((stencil_threads, stencil_order, step2_blocks, early_threads, early_order,
        stencil_split, early_split), ms per outer step)."""
        lc = NkLaunch()
        ms = ctypes.c_double()
        path = cache_path.encode() if cache_path else None
        self._check(self._lib.nk_autotune(self.h, int(n_rhs), int(flags), path, ctypes.byref(lc), ctypes.byref(ms)))
        return lc.as_tuple(), ms.value

    # -- learned subspace sizes ---------------------------------------------
    def features(self, b_dev, stream=None):
        """nk_features: the NK_MLP_IN predictor features of one device source."""
        f = np.zeros(NK_MLP_IN, np.float32)
        self._check(self._lib.nk_features(self.h, _dev_ptr(b_dev), _fptr(f), _stream_ptr(stream)))
        return f

    def predict_sizes(self, mlp, b_dev, k_max, stream=None):
        """nk_predict_sizes: (k, l) for one device source from a trained Mlp."""
        k = ctypes.c_int()
        ell = ctypes.c_int()
        self._check(self._lib.nk_predict_sizes(self.h, mlp.h, _dev_ptr(b_dev), int(k_max), ctypes.byref(k),
                                               ctypes.byref(ell), _stream_ptr(stream)))
        return k.value, ell.value

    def set_predictor(self, mlp):
        """nk_set_predictor: the Mlp that NK_PREDICT solves use (None: none).
        The context keeps a reference so the predictor outlives its use."""
        self._predictor = mlp
        self._check(self._lib.nk_set_predictor(self.h, mlp.h if mlp is not None else None))


def _fptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _f32(a, cols):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a.reshape(-1, cols)


class Mlp:
    """Owns an nk_mlp* (the 16 -> 64 -> 64 -> 2 size predictor)."""

    def __init__(self, seed: int = 0):
        lib = load_library()
        self._lib = lib
        h = ctypes.c_void_p()
        rc = lib.nk_mlp_create(ctypes.c_ulonglong(int(seed)), ctypes.byref(h))
        if rc != NK_OK:
            raise NkError(rc, "nk_mlp_create failed")
        self.h = h

    def _check(self, rc):
        if rc != NK_OK:
            raise NkError(rc, self._lib.nk_mlp_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self._lib.nk_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_norm(self, xmu, xsd, ymu, ysd):
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (xmu, xsd, ymu, ysd)]
        self._check(self._lib.nk_mlp_set_norm(self.h, *[_fptr(a) for a in arrs]))

    def set_weight_decay(self, wd):
        self._check(self._lib.nk_mlp_set_weight_decay(self.h, float(wd)))

    def get_params(self):
        w = np.zeros(NK_MLP_PARAMS, np.float32)
        self._check(self._lib.nk_mlp_get_params(self.h, _fptr(w)))
        return w

    def set_params(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        if w.size != NK_MLP_PARAMS:
            raise ValueError("expected %d parameters" % NK_MLP_PARAMS)
        self._check(self._lib.nk_mlp_set_params(self.h, _fptr(w)))

    def loss_grad(self, X, Y):
        X, Y = _f32(X, NK_MLP_IN), _f32(Y, NK_MLP_OUT)
        loss = np.zeros(1, np.float32)
        g = np.zeros(NK_MLP_PARAMS, np.float32)
        self._check(self._lib.nk_mlp_loss_grad(self.h, _fptr(X), _fptr(Y), X.shape[0], _fptr(loss), _fptr(g)))
        return float(loss[0]), g

    def train(self, X, Y, epochs, lr=1e-3):
        X, Y = _f32(X, NK_MLP_IN), _f32(Y, NK_MLP_OUT)
        hist = np.zeros(int(epochs), np.float32)
        self._check(self._lib.nk_mlp_train(self.h, _fptr(X), _fptr(Y), X.shape[0], int(epochs), float(lr),
                                           _fptr(hist)))
        return hist

    def forward(self, X):
        X = _f32(X, NK_MLP_IN)
        Y = np.zeros((X.shape[0], NK_MLP_OUT), np.float32)
        self._check(self._lib.nk_mlp_forward(self.h, _fptr(X), X.shape[0], _fptr(Y)))
        return Y


def _check_complex_extent(name, t, need):
    """Raises ValueError unless tensor t holds at least `need` complex128
    entries (a float64 tensor counts two of its entries per complex)."""
    per = 2 if str(getattr(t, "dtype", "")) == "torch.float64" else 1
    have = int(t.numel()) // per
    if need > 0 and have < need:
        raise ValueError("%s holds %d complex entries, the call needs %d" % (name, have, need))


def inner_sign_noalloc(alpha_dev, beta_dev, gamma_dev, c_dev, n_rhs, k, ell, p=0.0, hermitian=True,
                       stream=None):
    """nk_inner_sign_noalloc on caller-owned device tensors (complex128, shape
    (n_rhs, k)); returns (rc, message).  The library allocates nothing.

    The C entry point reads n_rhs * k complex entries of alpha, beta and gamma
    and writes as many to c, so a tensor holding fewer is refused here with
    ValueError before anything is launched."""
    need = int(n_rhs) * int(k)
    for name, t in (("alpha", alpha_dev), ("beta", beta_dev), ("gamma", gamma_dev), ("c", c_dev)):
        _check_complex_extent(name, t, need)
    lib = load_library()
    buf = ctypes.create_string_buffer(256)
    rc = lib.nk_inner_sign_noalloc(_dev_ptr(alpha_dev), _dev_ptr(beta_dev), _dev_ptr(gamma_dev), int(n_rhs),
                                   int(k), int(ell), float(p), 1 if hermitian else 0, _dev_ptr(c_dev),
                                   _stream_ptr(stream), buf, 256)
    return rc, buf.value.decode()


def _pad(x, n, k):
    """(n, k-1) off-diagonals -> (n, k) with a zero last entry."""
    x = np.asarray(x, dtype=np.complex128).reshape(n, -1)
    out = np.zeros((n, k), np.complex128)
    out[:, : x.shape[1]] = x
    return out
