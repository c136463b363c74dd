"""ctypes binding of libzolo_csd.so (include/zolo_csd.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Arrays are column-major.  Accepted inputs are torch tensors
(CUDA or CPU) and numpy arrays; CUDA tensors are passed by device pointer on
torch's current stream, host arrays by host pointer (the library stages them
through device memory itself).  Outputs are allocated like the inputs
(torch CUDA tensors stay on the device, numpy arrays stay on the host).

There is no fallback: if the shared library is missing or fails to load,
importing this module raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libzolo_csd.so")

CSD_F64 = 0
CSD_C128 = 1
STATUS_OK = 0
WARN_ALG2_RCHECK = 3


class csd_info(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("rank", ctypes.c_int),
        ("mu", ctypes.c_double),
        ("zolo_iters", ctypes.c_int),
        ("r_terms", ctypes.c_int * 4),
        ("ell", ctypes.c_double * 4),
        ("chol_fallback", ctypes.c_int),
        ("alg2_used", ctypes.c_int * 2),
        ("orth_err", ctypes.c_double * 2),
        ("rdiff", ctypes.c_double * 2),
        ("eig_splits", ctypes.c_int),
        ("eig_retries", ctypes.c_int),
        ("eig_leaves", ctypes.c_int),
        ("eig_offblock", ctypes.c_double),
        ("ms_total", ctypes.c_double),
    ]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out


class csd_profile(ctypes.Structure):
    _fields_ = [("count", ctypes.c_longlong * 5), ("ms", ctypes.c_double * 5), ("flops", ctypes.c_double * 5),
                ("site_count", ctypes.c_longlong * 24), ("site_ms", ctypes.c_double * 24),
                ("site_flops", ctypes.c_double * 24)]

    SITES = ["other", "qr_W", "qr_W2", "qr_update", "formq_W", "formq_W2", "formq_update", "zolo_combine",
             "gram", "chol_row", "chol_trailing", "trsm_f_update", "trsm_f_diag", "trsm_b_update",
             "trsm_b_diag", "H", "orth", "eig", "assembly", "alg2", "tmerge", "qr_update_x", "grad"]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing; build it with paper_1804_09002_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.csd_create.argtypes = [ctypes.POINTER(vp), ci, vp]
    lib.csd_set_stream.argtypes = [vp, vp]
    lib.csd_destroy.argtypes = [vp]
    lib.csd_workspace_bytes.argtypes = [vp]
    lib.csd_workspace_bytes.restype = ctypes.c_longlong
    lib.csd_polar.argtypes = [vp, ci, ci, vp, ci, vp, ci, vp, ci, vp, ci, vp, ci, vp,
                              ctypes.POINTER(ci), ctypes.POINTER(csd_info)]
    lib.polar.argtypes = [vp, ci, ci, vp, ci, vp, ci, vp, ci, ctypes.POINTER(csd_info)]
    lib.heig.argtypes = [vp, ci, ci, vp, ci, vp, vp, ci, ctypes.POINTER(csd_info)]
    lib.polar_noalloc.argtypes = [ci, ci, vp, ci, vp, ci, vp, ci, vp]
    lib.zolo_coeffs.argtypes = [cd, ci, vp, vp, ctypes.POINTER(cd), ctypes.POINTER(cd)]
    lib.zolo_plan.argtypes = [cd, ci, ci, vp, vp]
    lib.csd_profile_enable.argtypes = [vp, ci]
    lib.csd_set_tensor_cores.argtypes = [vp, ci]
    lib.csd_set_theta_mode.argtypes = [vp, ci]
    lib.csd_polar_rect.argtypes = [vp, ci, ci, ci, ci, vp, ci, vp, ci, vp, ci, vp, ci, vp, ci, vp,
                                   ctypes.POINTER(ci), ctypes.POINTER(csd_info)]
    lib.csd_complete_v2.argtypes = [vp, ci, ci, vp, ci, vp, ci, vp, ci, vp, ci, vp, vp, ci,
                                    ctypes.POINTER(csd_info)]
    lib.csd_profile_read.argtypes = [vp, ctypes.POINTER(csd_profile)]
    lib.csd_set_zolo_control.argtypes = [vp, ci, ci]
    lib.csd_set_test_hooks.argtypes = [vp, ctypes.c_uint, ctypes.c_longlong, ci]
    lib.csd_gemm.argtypes = [vp, ci, ci, ci, ci, ci, cd, vp, ci, vp, ci, cd, vp, ci, ci]
    lib.csd_fp64_peak.argtypes = [ci, ci, ctypes.POINTER(cd), ctypes.POINTER(cd)]
    lib.csd_set_sign_convention.argtypes = [vp, ci]
    lib.csd_set_alg2_fallback.argtypes = [vp, cd]
    lib.csd_set_mixed_precision.argtypes = [vp, ci, ctypes.c_uint]
    lib.csd_set_eig_leaf.argtypes = [vp, ci]
    lib.csd_batch_create.argtypes = [vp, ci, vp, ctypes.POINTER(vp)]
    lib.csd_batch_run.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.csd_batch_destroy.argtypes = [vp]
    lib.csd_batch_stats.argtypes = [vp, ctypes.POINTER(ci), ctypes.POINTER(ci), ctypes.POINTER(ci), vp]
    lib.csd_polar_backward.argtypes = [vp, ci, ci, vp, ci, vp, ci, vp, ci, vp, vp, ci, vp, ci, vp, ci, vp, vp, ci,
                                       vp, ci, ctypes.POINTER(csd_info)]
    lib.csd_launch_count.argtypes = []
    lib.csd_launch_count.restype = ctypes.c_longlong
    lib.csd_status_str.argtypes = [ci]
    lib.csd_status_str.restype = ctypes.c_char_p
    for f in ("csd_create", "csd_set_stream", "csd_destroy", "csd_polar", "polar", "heig", "zolo_coeffs",
              "zolo_plan", "csd_profile_enable", "csd_profile_read", "polar_noalloc", "csd_set_tensor_cores",
              "csd_set_theta_mode", "csd_complete_v2", "csd_polar_rect", "csd_set_zolo_control",
              "csd_set_test_hooks", "csd_gemm", "csd_fp64_peak", "csd_set_sign_convention",
              "csd_polar_backward", "csd_set_alg2_fallback", "csd_set_mixed_precision", "csd_set_eig_leaf",
              "csd_batch_create", "csd_batch_run", "csd_batch_destroy", "csd_batch_stats"):
        getattr(lib, f).restype = ci
    return lib


lib = _load()

EXPORTED = ["csd_create", "csd_set_stream", "csd_destroy", "csd_workspace_bytes", "csd_polar", "polar", "heig",
            "zolo_coeffs", "zolo_plan", "csd_status_str", "csd_profile_enable", "csd_profile_read",
            "csd_launch_count", "polar_noalloc", "csd_set_tensor_cores", "csd_set_theta_mode", "csd_complete_v2",
            "csd_polar_rect", "csd_set_zolo_control", "csd_set_test_hooks", "csd_gemm", "csd_fp64_peak",
            "csd_set_sign_convention", "csd_polar_backward", "csd_set_alg2_fallback", "csd_set_mixed_precision",
            "csd_set_eig_leaf", "csd_batch_create", "csd_batch_run", "csd_batch_destroy", "csd_batch_stats"]

STATUS_NOT_CONVERGED = 2
TEST_REJECT_EIG_SPLITS = 1


class CSDError(RuntimeError):
    def __init__(self, status, where, info=None):
        super().__init__(f"{where}: status {status} ({lib.csd_status_str(status).decode()})")
        self.status = status
        self.info = info


# ------------------------------------------------------------------ host-only
def zolo_coeffs(ell, r):
    """Zolotarev coefficients computed by the library's host code:
    (c[2r], a[r], mhat, ell_next)."""
    c = np.zeros(2 * r)
    a = np.zeros(r)
    m = ctypes.c_double()
    en = ctypes.c_double()
    st = lib.zolo_coeffs(float(ell), int(r), c.ctypes.data, a.ctypes.data, ctypes.byref(m), ctypes.byref(en))
    if st != 0:
        raise CSDError(st, "zolo_coeffs")
    return c, a, m.value, en.value


def zolo_plan(ell0=1e-15, rmax=8, max_iter=4):
    r = np.zeros(max_iter, dtype=np.int32)
    ell = np.zeros(max_iter)
    k = lib.zolo_plan(float(ell0), int(rmax), int(max_iter), r.ctypes.data, ell.ctypes.data)
    if k < 0:
        raise CSDError(k, "zolo_plan")
    return r[:k].tolist(), ell[:k].tolist()


def fp64_peak(kind=0, device=0):
    """Measured FP64 rate (TFLOP/s, best launch ms): kind 0 = DFMA loop,
    1 = mma.sync f64 loop."""
    t = ctypes.c_double()
    ms = ctypes.c_double()
    st = lib.csd_fp64_peak(int(device), int(kind), ctypes.byref(t), ctypes.byref(ms))
    if st != 0:
        raise CSDError(st, "csd_fp64_peak")
    return t.value, ms.value


# ------------------------------------------------------------------ arrays
def _torch():
    import torch
    return torch


def _is_torch(x):
    try:
        import torch
    except ImportError:
        return False
    return isinstance(x, torch.Tensor)


def _dtype_code(x):
    if _is_torch(x):
        torch = _torch()
        if x.dtype == torch.float64:
            return CSD_F64
        if x.dtype == torch.complex128:
            return CSD_C128
    else:
        if x.dtype == np.float64:
            return CSD_F64
        if x.dtype == np.complex128:
            return CSD_C128
    raise TypeError("inputs must be float64 or complex128")


def _colmajor(x):
    """(array, pointer, ld) of a column-major view of the 2-D array x."""
    # a single column has no meaningful column stride: its ld is m
    if _is_torch(x):
        if x.dim() != 2:
            raise ValueError("expected a 2-D tensor")
        m, n = x.shape
        if not (x.stride(0) == 1 and (n == 1 or x.stride(1) >= max(m, 1))):
            x = x.t().contiguous().t()
        return x, x.data_ptr(), max(m, 1) if n == 1 else max(x.stride(1), 1)
    x = np.asfortranarray(x)
    if x.ndim != 2:
        raise ValueError("expected a 2-D array")
    m, n = x.shape
    return x, x.ctypes.data, max(m, 1) if n == 1 else max(x.strides[1] // x.itemsize, 1)


def _empty_like2(x, m, n, dtype=None):
    if _is_torch(x):
        torch = _torch()
        t = torch.empty((n, m), dtype=dtype or x.dtype, device=x.device).t()
        return t
    return np.empty((m, n), dtype=dtype or x.dtype, order="F")


def _empty_vec(x, n):
    if _is_torch(x):
        torch = _torch()
        return torch.empty(n, dtype=torch.float64, device=x.device)
    return np.empty(n, dtype=np.float64)


def _ptr(v):
    return v.data_ptr() if _is_torch(v) else v.ctypes.data


class Context:
    """A library context: device workspace plus the CUDA stream it issues on."""

    def __init__(self, device=0):
        self._h = ctypes.c_void_p()
        st = lib.csd_create(ctypes.byref(self._h), int(device), None)
        if st != 0:
            raise CSDError(st, "csd_create")
        self.device = device

    def close(self):
        if self._h:
            lib.csd_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _bind_stream(self, x):
        if _is_torch(x) and x.is_cuda:
            torch = _torch()
            lib.csd_set_stream(self._h, ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream))
        else:
            lib.csd_set_stream(self._h, None)

    def set_tensor_cores(self, enable=True, sites=-1):
        """Run real FP64 products on the tcgen05 tensor cores (sliced BF16,
        FP64-accurate) instead of the FP64 FMA pipe; `sites` is a bit mask
        over the GEMM call sites (csd_profile.SITES), -1 = all."""
        st = lib.csd_set_tensor_cores(self._h, (sites if sites else 0) if enable else 0)
        if st != 0:
            raise CSDError(st, "csd_set_tensor_cores")

    def workspace_bytes(self):
        return lib.csd_workspace_bytes(self._h)

    def set_theta_mode(self, mode):
        """0: theta = atan2(S, C) (remark (iii), default); 1: theta from the
        eigenvalues of B, sin(theta) - cos(theta) = Lambda (remark (iv))."""
        st = lib.csd_set_theta_mode(self._h, int(mode))
        if st != 0:
            raise CSDError(st, "csd_set_theta_mode")

    def set_eig_leaf(self, leaf):
        """Zolo-eig blocks of at most `leaf` rows go to the batched Jacobi
        leaf solver."""
        st = lib.csd_set_eig_leaf(self._h, int(leaf))
        if st != 0:
            raise CSDError(st, "csd_set_eig_leaf")

    def set_mixed_precision(self, slices=6, scope=1):
        """Cholesky-iteration products of Zolo-pd with 5 or 6 BF16 slices
        (scope bit 0: the CSD's polars, bit 1: Zolo-eig's); 7 = off."""
        st = lib.csd_set_mixed_precision(self._h, int(slices), int(scope))
        if st != 0:
            raise CSDError(st, "csd_set_mixed_precision")

    def set_alg2_fallback(self, factor=1e3):
        """SVD polar fallback of Algorithm 2 when ||R~ - R|| / ||R|| reaches
        factor n u (0: always; negative: never, warn instead)."""
        st = lib.csd_set_alg2_fallback(self._h, float(factor))
        if st != 0:
            raise CSDError(st, "csd_set_alg2_fallback")

    def set_sign_convention(self, mode=1):
        """1: each column of V1 (with U1, U2) has its largest-magnitude entry
        real positive, so the factors are unique for distinct angles."""
        st = lib.csd_set_sign_convention(self._h, int(mode))
        if st != 0:
            raise CSDError(st, "csd_set_sign_convention")

    def csd_backward(self, U1, U2, V1, theta, gU1=None, gU2=None, gV1=None, gtheta=None):
        """(gA1, gA2) of a loss with gradients gU1, gU2, gV1, gtheta (None =
        zero) at the outputs of csd_polar (real, full rank)."""
        U1, p1, l1 = _colmajor(U1)
        U2, p2, l2 = _colmajor(U2)
        V1, pv, lv = _colmajor(V1)
        n = V1.shape[1]
        if _dtype_code(V1) != CSD_F64:
            raise TypeError("csd_backward is defined for real float64 factors")

        def opt(x):
            if x is None:
                return None, None, n
            x, p, ld = _colmajor(x)
            return x, p, ld

        def vec(x):
            if x is None:
                return None, None
            x = x.contiguous() if _is_torch(x) else np.ascontiguousarray(x, dtype=np.float64)
            return x, _ptr(x)

        gU1, pg1, lg1 = opt(gU1)
        gU2, pg2, lg2 = opt(gU2)
        gV1, pgv, lgv = opt(gV1)
        theta, pth = vec(theta)
        gtheta, pgt = vec(gtheta)
        gA1 = _empty_like2(V1, n, n)
        gA2 = _empty_like2(V1, n, n)
        info = csd_info()
        self._bind_stream(V1)
        st = lib.csd_polar_backward(self._h, CSD_F64, n, p1, l1, p2, l2, pv, lv, pth, pg1, lg1, pg2, lg2, pgv, lgv,
                                    pgt, _ptr(gA1), n, _ptr(gA2), n, ctypes.byref(info))
        if st != 0:
            raise CSDError(st, "csd_polar_backward", info.as_dict())
        return gA1, gA2

    def set_zolo_control(self, max_extra_passes=1, stop_after=0):
        """polar(): further plan passes when the iterate has not converged
        (default 1); stop_after = k > 0 returns the k-th Zolo-pd iterate."""
        st = lib.csd_set_zolo_control(self._h, int(max_extra_passes), int(stop_after))
        if st != 0:
            raise CSDError(st, "csd_set_zolo_control")

    def set_test_hooks(self, flags=0, tc_probe_wait=0, tc_flush_every=0):
        """Failure-path test hooks (host-side split rejection, a tensor-core
        wait that runs out, int64 write-outs every few drains); 0 = off."""
        st = lib.csd_set_test_hooks(self._h, int(flags), int(tc_probe_wait), int(tc_flush_every))
        if st != 0:
            raise CSDError(st, "csd_set_test_hooks")

    def gemm(self, A, B, C=None, alpha=1.0, beta=0.0, opA=0, opB=0, engine=1):
        """C = alpha op(A) op(B) + beta C on the library's FP64 product
        kernels (engine 0: FP64 pipe, 1: tensor cores); float64 CUDA tensors."""
        if not (_is_torch(A) and A.is_cuda):
            raise TypeError("csd_gemm takes CUDA tensors")
        A, pa, la = _colmajor(A)
        B, pb, lb = _colmajor(B)
        m = A.shape[0] if opA == 0 else A.shape[1]
        k = A.shape[1] if opA == 0 else A.shape[0]
        n = B.shape[1] if opB == 0 else B.shape[0]
        if C is None:
            C = _empty_like2(A, m, n)
            C.zero_()
        C, pc, lc = _colmajor(C)
        self._bind_stream(A)
        st = lib.csd_gemm(self._h, int(opA), int(opB), m, n, k, float(alpha), pa, la, pb, lb, float(beta), pc, lc,
                          int(engine))
        if st != 0:
            raise CSDError(st, "csd_gemm")
        return C

    def complete_v2(self, A3, A4, U1, U2, theta):
        """V2 of the complete 2 x 2 CSD of a unitary [A1 A3; A2 A4] from the
        U1, U2, theta of [A1; A2] (remark (viii))."""
        dt = _dtype_code(A3)
        A3, p3, l3 = _colmajor(A3)
        A4, p4, l4 = _colmajor(A4)
        U1, pu1, lu1 = _colmajor(U1)
        U2, pu2, lu2 = _colmajor(U2)
        n = A3.shape[1]
        if _is_torch(theta):
            theta = theta.contiguous()
        else:
            theta = np.ascontiguousarray(theta, dtype=np.float64)
        V2 = _empty_like2(A3, n, n)
        info = csd_info()
        self._bind_stream(A3)
        st = lib.csd_complete_v2(self._h, dt, n, p3, l3, p4, l4, pu1, lu1, pu2, lu2, _ptr(theta), _ptr(V2), n,
                                 ctypes.byref(info))
        if st != STATUS_OK:
            raise CSDError(st, "csd_complete_v2")
        return V2

    def csd_polar(self, A1, A2, out=None):
        """CS decomposition of [A1; A2].  Returns dict(U1, U2, V1, theta,
        rank, info); columns/entries beyond `rank` are unspecified/zero."""
        dt = _dtype_code(A1)
        if _dtype_code(A2) != dt:
            raise TypeError("A1 and A2 must share a dtype")
        A1, p1, l1 = _colmajor(A1)
        A2, p2, l2 = _colmajor(A2)
        n = A1.shape[1]
        if tuple(A1.shape) != (n, n) or tuple(A2.shape) != (n, n):
            raise ValueError("A1 and A2 must be n x n")
        if out is None:
            out = dict(U1=_empty_like2(A1, n, n), U2=_empty_like2(A1, n, n), V1=_empty_like2(A1, n, n),
                       theta=_empty_vec(A1, n))
        U1, pu1, lu1 = _colmajor(out["U1"])
        U2, pu2, lu2 = _colmajor(out["U2"])
        V1, pv1, lv1 = _colmajor(out["V1"])
        theta = out["theta"]
        rank = ctypes.c_int()
        info = csd_info()
        self._bind_stream(A1)
        st = lib.csd_polar(self._h, dt, n, p1, l1, p2, l2, pu1, lu1, pu2, lu2, pv1, lv1, _ptr(theta),
                           ctypes.byref(rank), ctypes.byref(info))
        if st not in (STATUS_OK, WARN_ALG2_RCHECK):
            raise CSDError(st, "csd_polar", info.as_dict())
        return dict(U1=U1, U2=U2, V1=V1, theta=theta, rank=rank.value, info=info.as_dict(), status=st)

    def csd_polar_rect(self, A1, A2):
        """CS decomposition of [A1; A2] with A1 m1 x n, A2 m2 x n (m_i >= n).
        Returns dict(U1 (m1 x n), U2 (m2 x n), V1, theta, rank, info)."""
        dt = _dtype_code(A1)
        if _dtype_code(A2) != dt:
            raise TypeError("A1 and A2 must share a dtype")
        A1, p1, l1 = _colmajor(A1)
        A2, p2, l2 = _colmajor(A2)
        m1, n = A1.shape
        m2 = A2.shape[0]
        if A2.shape[1] != n:
            raise ValueError("A1 and A2 must have the same number of columns")
        U1 = _empty_like2(A1, m1, n)
        U2 = _empty_like2(A1, m2, n)
        V1 = _empty_like2(A1, n, n)
        theta = _empty_vec(A1, n)
        rank = ctypes.c_int()
        info = csd_info()
        self._bind_stream(A1)
        st = lib.csd_polar_rect(self._h, dt, m1, m2, n, p1, l1, p2, l2, _ptr(U1), m1, _ptr(U2), m2, _ptr(V1), n,
                                _ptr(theta), ctypes.byref(rank), ctypes.byref(info))
        if st not in (STATUS_OK, WARN_ALG2_RCHECK):
            raise CSDError(st, "csd_polar_rect")
        return dict(U1=U1, U2=U2, V1=V1, theta=theta, rank=rank.value, info=info.as_dict(), status=st)

    def polar(self, A, want_h=True, allow_not_converged=False):
        """(W, H, info).  CSD_ERR_NOT_CONVERGED raises unless
        allow_not_converged, in which case the last iterate is returned and
        info["status"] says so."""
        dt = _dtype_code(A)
        A, pa, la = _colmajor(A)
        n = A.shape[1]
        W = _empty_like2(A, n, n)
        H = _empty_like2(A, n, n) if want_h else None
        info = csd_info()
        self._bind_stream(A)
        st = lib.polar(self._h, dt, n, pa, la, _ptr(W), n, _ptr(H) if want_h else None, n, ctypes.byref(info))
        if st != STATUS_OK and not (allow_not_converged and st == STATUS_NOT_CONVERGED):
            raise CSDError(st, "polar", info.as_dict())
        return W, H, info.as_dict()

    def heig(self, B):
        dt = _dtype_code(B)
        B, pb, lb = _colmajor(B)
        n = B.shape[1]
        V = _empty_like2(B, n, n)
        lam = _empty_vec(B, n)
        info = csd_info()
        self._bind_stream(B)
        st = lib.heig(self._h, dt, n, pb, lb, _ptr(lam), _ptr(V), n, ctypes.byref(info))
        if st != STATUS_OK:
            raise CSDError(st, "heig", info.as_dict())
        return lam, V, info.as_dict()


class Batch:
    """A plan for many real FP64 CSDs of the given sizes (csd_batch_*):
    the first run autotunes and captures a CUDA graph, later runs on the
    same packed buffers replay it."""

    def __init__(self, ctx, sizes):
        import torch
        self.ctx = ctx
        self.sizes = [int(v) for v in sizes]
        self._h = ctypes.c_void_p()
        n = (ctypes.c_int * len(self.sizes))(*self.sizes)
        st = lib.csd_batch_create(ctx._h, len(self.sizes), ctypes.cast(n, ctypes.c_void_p), ctypes.byref(self._h))
        if st != 0:
            raise CSDError(st, "csd_batch_create")
        self.off = np.concatenate([[0], np.cumsum([v * v for v in self.sizes])]).astype(np.int64)
        self.toff = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        dev = torch.device("cuda", ctx.device)
        tot, ttot = int(self.off[-1]), int(self.toff[-1])
        self.A1 = torch.empty(tot, dtype=torch.float64, device=dev)
        self.A2 = torch.empty(tot, dtype=torch.float64, device=dev)
        self.U1 = torch.empty(tot, dtype=torch.float64, device=dev)
        self.U2 = torch.empty(tot, dtype=torch.float64, device=dev)
        self.V1 = torch.empty(tot, dtype=torch.float64, device=dev)
        self.theta = torch.empty(ttot, dtype=torch.float64, device=dev)
        self.status = np.zeros(len(self.sizes), dtype=np.int32)

    def _view(self, buf, i):
        n = self.sizes[i]
        return buf[int(self.off[i]):int(self.off[i + 1])].view(n, n).t()  # column-major n x n

    def load(self, A1s, A2s):
        """Copy the inputs (column-major views or any 2-D tensors) into the
        packed input buffers."""
        for i, (a1, a2) in enumerate(zip(A1s, A2s)):
            self._view(self.A1, i).copy_(a1)
            self._view(self.A2, i).copy_(a2)

    def run(self):
        self.ctx._bind_stream(self.A1)
        st = lib.csd_batch_run(self._h, self.A1.data_ptr(), self.A2.data_ptr(), self.U1.data_ptr(),
                               self.U2.data_ptr(), self.V1.data_ptr(), self.theta.data_ptr(), self.status.ctypes.data)
        if st != 0:
            raise CSDError(st, "csd_batch_run")
        return self.status

    def result(self, i):
        return dict(U1=self._view(self.U1, i), U2=self._view(self.U2, i), V1=self._view(self.V1, i),
                    theta=self.theta[int(self.toff[i]):int(self.toff[i + 1])], status=int(self.status[i]))

    def stats(self):
        g, nb, tcb = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        t = (ctypes.c_double * 3)()
        lib.csd_batch_stats(self._h, ctypes.byref(g), ctypes.byref(nb), ctypes.byref(tcb), ctypes.cast(t, ctypes.c_void_p))
        return dict(granularity=g.value, buckets=nb.value, tc_buckets=tcb.value,
                    tune_ms={16: t[0], 32: t[1], 64: t[2]})

    def close(self):
        if self._h:
            lib.csd_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default = {}


def default_context(device=0):
    if device not in _default:
        _default[device] = Context(device)
    return _default[device]


def csd_polar(A1, A2, device=0):
    return default_context(device).csd_polar(A1, A2)


def polar(A, device=0, want_h=True):
    return default_context(device).polar(A, want_h)


def heig(B, device=0):
    return default_context(device).heig(B)
