"""ctypes binding of libchebfd.so: argument marshalling only.

The functions below carry the names of the C ABI (include/chebfd.h) and pass
device pointers (torch tensors on the current CUDA device), host numpy arrays
and the current torch stream through unchanged.  Every computation runs inside
the library; if it is missing this module raises instead of falling back.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libchebfd.so")

R64, C128, R32, C64 = 0, 1, 2, 3
KERNEL_NONE, KERNEL_FEJER, KERNEL_JACKSON, KERNEL_LANCZOS = 0, 1, 2, 3
LATTICE_TOPI, LATTICE_GRAPHENE, LATTICE_TOPI_SLAB = 0, 1, 2
LATTICES = {"topi": LATTICE_TOPI, "graphene": LATTICE_GRAPHENE, "topi_slab": LATTICE_TOPI_SLAB}
KERNEL_IDS = {"none": KERNEL_NONE, "fejer": KERNEL_FEJER, "jackson": KERNEL_JACKSON,
              "lanczos": KERNEL_LANCZOS}
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENUMERIC", 5: "ENOCONV",
          6: "ETIMEOUT", 7: "EUNSUPPORTED"}

PRECISION = {"fp64": 0, "mixed": 1, "mixed_df": 2}

c_i64p = ctypes.POINTER(ctypes.c_int64)
c_i32p = ctypes.POINTER(ctypes.c_int32)
c_dp = ctypes.POINTER(ctypes.c_double)
c_vp = ctypes.c_void_p


class LatticeDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("Lx", ctypes.c_int32), ("Ly", ctypes.c_int32),
                ("Lz", ctypes.c_int32), ("t", ctypes.c_double), ("m", ctypes.c_double),
                ("W", ctypes.c_double), ("seed", ctypes.c_uint64), ("sell_C", ctypes.c_int32),
                ("sell_sigma", ctypes.c_int32), ("also_single", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class MatrixInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("nnz_padded", ctypes.c_int64),
                ("nchunks", ctypes.c_int64), ("C", ctypes.c_int32), ("sigma", ctypes.c_int32),
                ("max_row_len", ctypes.c_int32), ("is_complex", ctypes.c_int32),
                ("has_single", ctypes.c_int32), ("blocked_width", ctypes.c_int32)]


# name -> (restype, argtypes); every function returns chebfd_status unless noted
SIGNATURES = {
    "chebfd_abi_version": (ctypes.c_int, []),
    "chebfd_last_error": (ctypes.c_char_p, []),
    "chebfd_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "chebfd_matrix_create_csr": (ctypes.c_int, [ctypes.c_int64, c_i64p, c_i32p, c_vp, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_int, c_vp,
                                                ctypes.POINTER(c_vp)]),
    "chebfd_matrix_create_lattice": (ctypes.c_int, [ctypes.POINTER(LatticeDesc), c_vp,
                                                    ctypes.POINTER(c_vp)]),
    "chebfd_matrix_get_info": (ctypes.c_int, [c_vp, ctypes.POINTER(MatrixInfo)]),
    "chebfd_matrix_export_sell": (ctypes.c_int, [c_vp, c_i64p, c_i32p, c_i32p, c_vp, c_i64p]),
    "chebfd_matrix_destroy": (ctypes.c_int, [c_vp]),
    "chebfd_matrix_set_blocked": (ctypes.c_int, [c_vp, ctypes.c_int]),
    "chebfd_matrix_set_matrix_free": (ctypes.c_int, [c_vp, ctypes.c_int]),
    "chebfd_spmv": (ctypes.c_int, [c_vp, ctypes.c_double, ctypes.c_double, c_vp, c_vp,
                                   ctypes.c_int64, ctypes.c_int, ctypes.c_int, c_vp]),
    "chebfd_scale_bounds": (ctypes.c_int, [c_vp, ctypes.c_int, ctypes.c_uint64, c_dp, c_dp, c_dp,
                                           c_dp, c_vp]),
    "chebfd_window_coeffs": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_double, c_dp]),
    "chebfd_filter_block": (ctypes.c_int, [c_vp, ctypes.c_double, ctypes.c_double, c_dp,
                                           ctypes.c_int, c_vp, ctypes.c_int64, ctypes.c_int,
                                           ctypes.c_int, c_dp, c_vp]),
    "chebfd_filter_block_noalloc": (ctypes.c_int, [c_vp, ctypes.c_double, ctypes.c_double, c_dp,
                                                   ctypes.c_int, c_vp, ctypes.c_int64,
                                                   ctypes.c_int, ctypes.c_int, c_dp, c_vp]),
    "chebfd_filter_block_df": (ctypes.c_int, [c_vp, ctypes.c_double, ctypes.c_double, c_dp,
                                              ctypes.c_int, c_vp, ctypes.c_int64, ctypes.c_int,
                                              ctypes.c_int, c_vp]),
    "chebfd_filter_block_host": (ctypes.c_int, [c_vp, ctypes.c_double, ctypes.c_double, c_dp,
                                                ctypes.c_int, c_vp, ctypes.c_int64, ctypes.c_int,
                                                ctypes.c_int, c_vp]),
    "chebfd_chebyshev_step": (ctypes.c_int, [c_vp, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, c_vp, c_vp, c_vp, ctypes.c_int64,
                                             ctypes.c_int, ctypes.c_int, c_vp]),
    "chebfd_kpm_moments": (ctypes.c_int, [c_vp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_uint64, c_dp, c_vp]),
    "chebfd_random_block": (ctypes.c_int, [c_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                           ctypes.c_int, c_vp]),
    "chebfd_orthonormalize": (ctypes.c_int, [c_vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int64,
                                             ctypes.c_int, ctypes.c_uint64, c_i64p, c_i32p, c_vp]),
    "chebfd_rayleigh_ritz": (ctypes.c_int, [c_vp, c_vp, ctypes.c_int64, ctypes.c_int,
                                            ctypes.c_int, c_dp, c_dp, c_vp, c_vp]),
    "chebfd_harmonic_ritz": (ctypes.c_int, [c_vp, c_vp, ctypes.c_int64, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_double, c_dp, c_dp, c_vp]),
    "chebfd_residuals": (ctypes.c_int, [c_vp, c_vp, c_dp, ctypes.c_int64, ctypes.c_int,
                                        ctypes.c_int, c_dp, c_vp]),
    "chebfd_convert_block": (ctypes.c_int, [c_vp, ctypes.c_int, ctypes.c_int64, c_vp,
                                            ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                            ctypes.c_int, c_vp]),
    "chebfd_solve": (ctypes.c_int, [c_vp, c_vp, c_vp, ctypes.POINTER(c_vp)]),
    "chebfd_result_get": (ctypes.c_int, [c_vp, c_vp]),
    "chebfd_result_destroy": (ctypes.c_int, [c_vp]),
    "chebfd_result_copy_vectors": (ctypes.c_int, [c_vp, c_vp, ctypes.c_int64, c_vp]),
    "chebfd_result_iterations": (ctypes.c_int, [c_vp, c_vp, ctypes.c_int, c_i32p]),
    "chebfd_gram": (ctypes.c_int, [c_vp, ctypes.c_int64, c_vp, ctypes.c_int64, ctypes.c_int64,
                                   ctypes.c_int, ctypes.c_int, c_vp, ctypes.c_int, c_vp]),
    "chebfd_block_update": (ctypes.c_int, [c_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                           c_vp, ctypes.c_int, ctypes.c_int, c_vp,
                                           ctypes.c_int64, ctypes.c_int, ctypes.c_int, c_vp]),
    "chebfd_ensemble_create": (ctypes.c_int, [ctypes.POINTER(c_vp), ctypes.c_int, ctypes.c_int,
                                              c_vp, ctypes.POINTER(c_vp)]),
    "chebfd_ensemble_info": (ctypes.c_int, [c_vp, c_i64p, c_i32p, c_i64p, c_i32p, c_i32p,
                                            c_i32p]),
    "chebfd_ensemble_set_coeffs": (ctypes.c_int, [c_vp, c_dp, c_dp, c_dp, ctypes.c_int, c_vp]),
    "chebfd_ensemble_set_launch": (ctypes.c_int, [c_vp, ctypes.c_int, ctypes.c_int]),
    "chebfd_ensemble_filter": (ctypes.c_int, [c_vp, c_vp, ctypes.c_int64, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_int, c_vp]),
    "chebfd_ensemble_autotune": (ctypes.c_int, [ctypes.POINTER(c_vp), ctypes.c_int, c_vp,
                                                ctypes.c_int64, ctypes.c_int, ctypes.c_int, c_vp,
                                                ctypes.POINTER(c_vp), c_dp]),
    "chebfd_ensemble_destroy": (ctypes.c_int, [c_vp]),
    "chebfd_param_features": (ctypes.c_int, [c_vp, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_uint64, c_dp, c_dp, c_vp]),
    "chebfd_choose_params": (ctypes.c_int, [c_vp, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double, c_vp, ctypes.c_int,
                                            ctypes.c_uint64, c_i32p, c_i32p, c_i32p, c_dp, c_vp]),
    "chebfd_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(c_vp)]),
    "chebfd_mlp_num_params": (ctypes.c_int, [c_vp, c_i64p]),
    "chebfd_mlp_set_params": (ctypes.c_int, [c_vp, ctypes.POINTER(ctypes.c_float),
                                             ctypes.c_int64]),
    "chebfd_mlp_get_params": (ctypes.c_int, [c_vp, ctypes.POINTER(ctypes.c_float),
                                             ctypes.POINTER(ctypes.c_float), ctypes.c_int64]),
    "chebfd_mlp_forward": (ctypes.c_int, [c_vp, c_vp, ctypes.c_int, c_vp, c_vp]),
    "chebfd_mlp_loss_grad": (ctypes.c_int, [c_vp, c_vp, c_vp, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_float), c_vp]),
    "chebfd_mlp_adam": (ctypes.c_int, [c_vp, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_float, c_vp]),
    "chebfd_mlp_destroy": (ctypes.c_int, [c_vp]),
    "chebfd_solve_batched": (ctypes.c_int, [c_vp, ctypes.POINTER(c_vp), c_dp, c_dp, c_vp, c_vp,
                                            ctypes.POINTER(c_vp), c_i32p]),
}

KERNEL_NAMES = {v: k for k, v in KERNEL_IDS.items()}


class Params(ctypes.Structure):
    _fields_ = [("lam_lo", ctypes.c_double), ("lam_hi", ctypes.c_double), ("eps", ctypes.c_double),
                ("a", ctypes.c_double), ("b", ctypes.c_double), ("mu", ctypes.c_double),
                ("ns", ctypes.c_int32), ("Np", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("nb", ctypes.c_int32), ("precision", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("lanczos_steps", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("window_inset", ctypes.c_double)]


class ResultInfo(ctypes.Structure):
    _fields_ = [("nev", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("fp64_iterations", ctypes.c_int32),
                ("n_mvm", ctypes.c_int64), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("seconds_filter", ctypes.c_double), ("seconds_dense", ctypes.c_double),
                ("seconds_total", ctypes.c_double), ("lambda_", c_dp), ("res", c_dp),
                ("V", c_vp)]


class IterationInfo(ctypes.Structure):
    _fields_ = [("iteration", ctypes.c_int32), ("fp64_filter", ctypes.c_int32),
                ("in_window", ctypes.c_int32), ("ghosts", ctypes.c_int32),
                ("accepted", ctypes.c_int32), ("converged_pairs", ctypes.c_int32),
                ("Np", ctypes.c_int32), ("locked", ctypes.c_int32),
                ("res_min", ctypes.c_double), ("res_max", ctypes.c_double),
                ("seconds_filter", ctypes.c_double), ("seconds_dense", ctypes.c_double),
                ("seconds_gram", ctypes.c_double), ("seconds_block_gemm", ctypes.c_double),
                ("seconds_eigensolve", ctypes.c_double), ("seconds_hy", ctypes.c_double),
                ("seconds_residuals", ctypes.c_double), ("seconds_other", ctypes.c_double)]


class ChebFDError(RuntimeError):
    def __init__(self, status, where, message):
        super().__init__("%s: %s (%s)" % (where, STATUS.get(status, status), message))
        self.status = status


_lib = None


def lib():
    """Load libchebfd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libchebfd.so not built: run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status, where):
    if status != 0:
        msg = lib().chebfd_last_error()
        raise ChebFDError(status, where, msg.decode() if msg else "")


def _ptr(t):
    """Device or host pointer of a torch tensor / numpy array (None -> NULL)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(t.ctypes.data)


def _stream(stream=None):
    if stream is not None:
        return ctypes.c_void_p(stream)
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def dtype_of(t):
    import torch
    return {torch.float64: R64, torch.complex128: C128, torch.float32: R32,
            torch.complex64: C64}[t.dtype]


class Matrix:
    """Owner of a chebfd_matrix handle (device SELL-C-sigma)."""

    def __init__(self, handle):
        self.handle = handle
        info = MatrixInfo()
        _check(lib().chebfd_matrix_get_info(handle, ctypes.byref(info)), "chebfd_matrix_get_info")
        self.info = info

    @property
    def n(self):
        return self.info.n

    @property
    def is_complex(self):
        return bool(self.info.is_complex)

    @property
    def blocked_width(self):
        """Block columns per 4-row block of the blocked copy (0: no copy)."""
        return self.info.blocked_width

    def set_blocked(self, enable):
        """Use (True) or bypass (False) the blocked copy in the complex64 step."""
        _check(lib().chebfd_matrix_set_blocked(self.handle, 1 if enable else 0),
               "chebfd_matrix_set_blocked")

    def set_matrix_free(self, enable, pairs=False):
        """Rebuild the insulator's entries in registers in the complex64 step
        and in the double-float step; pairs=True also runs the complex64
        filter two Chebyshev steps per pass (16-column panels)."""
        mode = (2 if pairs else 1) if enable else 0
        _check(lib().chebfd_matrix_set_matrix_free(self.handle, mode),
               "chebfd_matrix_set_matrix_free")

    def close(self):
        if self.handle:
            _check(lib().chebfd_matrix_destroy(self.handle), "chebfd_matrix_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def export_sell(self):
        i = self.info
        chunk_ptr = np.zeros(i.nchunks + 1, np.int64)
        chunk_len = np.zeros(i.nchunks, np.int32)
        col = np.zeros(i.nnz_padded, np.int32)
        val = np.zeros(i.nnz_padded, np.complex128 if i.is_complex else np.float64)
        perm = np.zeros(i.n, np.int64)
        _check(lib().chebfd_matrix_export_sell(
            self.handle, chunk_ptr.ctypes.data_as(c_i64p), chunk_len.ctypes.data_as(c_i32p),
            col.ctypes.data_as(c_i32p), ctypes.c_void_p(val.ctypes.data),
            perm.ctypes.data_as(c_i64p)), "chebfd_matrix_export_sell")
        return dict(n=i.n, C=i.C, sigma=i.sigma, nchunks=i.nchunks, chunk_ptr=chunk_ptr,
                    chunk_len=chunk_len, col=col, val=val, perm=perm)


def chebfd_matrix_create_csr(rowptr, col, val, sell_C=1, sell_sigma=1, also_single=False,
                             stream=None):
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    cplx = np.iscomplexobj(val)
    val = np.ascontiguousarray(val, np.complex128 if cplx else np.float64)
    h = c_vp()
    _check(lib().chebfd_matrix_create_csr(
        len(rowptr) - 1, rowptr.ctypes.data_as(c_i64p), col.ctypes.data_as(c_i32p),
        ctypes.c_void_p(val.ctypes.data), C128 if cplx else R64, sell_C, sell_sigma,
        1 if also_single else 0, _stream(stream), ctypes.byref(h)), "chebfd_matrix_create_csr")
    return Matrix(h)


def chebfd_matrix_create_lattice(kind, Lx, Ly, Lz=1, t=1.0, m=1.0, W=0.0, seed=0, sell_C=1,
                                 sell_sigma=1, also_single=False, stream=None):
    d = LatticeDesc(kind=LATTICES[kind] if isinstance(kind, str) else int(kind),
                    Lx=Lx, Ly=Ly, Lz=Lz, t=t, m=m, W=W, seed=seed, sell_C=sell_C,
                    sell_sigma=sell_sigma, also_single=1 if also_single else 0, reserved=0)
    h = c_vp()
    _check(lib().chebfd_matrix_create_lattice(ctypes.byref(d), _stream(stream), ctypes.byref(h)),
           "chebfd_matrix_create_lattice")
    return Matrix(h)


def chebfd_spmv(H, alpha, beta, X, Y, stream=None):
    n, nb = X.shape[0], X.shape[1]
    ld = X.stride(0)
    assert Y.stride(0) == ld and X.dtype == Y.dtype
    _check(lib().chebfd_spmv(H.handle, alpha, beta, _ptr(X), _ptr(Y), ld, nb, dtype_of(X),
                             _stream(stream)), "chebfd_spmv")


def chebfd_scale_bounds(H, lanczos_steps=30, seed=0, stream=None):
    a, b, al, be = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().chebfd_scale_bounds(H.handle, lanczos_steps, seed, ctypes.byref(a),
                                     ctypes.byref(b), ctypes.byref(al), ctypes.byref(be),
                                     _stream(stream)), "chebfd_scale_bounds")
    return a.value, b.value, al.value, be.value


def chebfd_window_coeffs(a, b, lam_lo, lam_hi, Np, kernel="lanczos", mu=2.0):
    gc = np.zeros(Np + 1)
    k = KERNEL_IDS[kernel] if isinstance(kernel, str) else int(kernel)
    _check(lib().chebfd_window_coeffs(a, b, lam_lo, lam_hi, Np, k, mu, gc.ctypes.data_as(c_dp)),
           "chebfd_window_coeffs")
    return gc


def chebfd_filter_block(H, alpha, beta, gc, X, moments=None, stream=None):
    """In place: X <- p[H] X for a device tensor X (N x nb, row stride ld)."""
    gc = np.ascontiguousarray(gc, np.float64)
    Np = len(gc) - 1
    n, nb = X.shape[0], X.shape[1]
    mp = ctypes.cast(ctypes.c_void_p(moments.data_ptr()), c_dp) if moments is not None else None
    _check(lib().chebfd_filter_block(H.handle, alpha, beta, gc.ctypes.data_as(c_dp), Np, _ptr(X),
                                     X.stride(0), nb, dtype_of(X), mp, _stream(stream)),
           "chebfd_filter_block")


def chebfd_filter_block_noalloc(H, alpha, beta, gc, X, moments=None, stream=None):
    """As chebfd_filter_block, with the library's fixed device scratch instead of
    allocated work vectors (for callers that cannot allocate device memory)."""
    gc = np.ascontiguousarray(gc, np.float64)
    Np = len(gc) - 1
    n, nb = X.shape[0], X.shape[1]
    mp = ctypes.cast(ctypes.c_void_p(moments.data_ptr()), c_dp) if moments is not None else None
    _check(lib().chebfd_filter_block_noalloc(H.handle, alpha, beta, gc.ctypes.data_as(c_dp), Np,
                                             _ptr(X), X.stride(0), nb, dtype_of(X), mp,
                                             _stream(stream)), "chebfd_filter_block_noalloc")


def chebfd_filter_block_host(H, alpha, beta, gc, X, stream=None):
    """In place: X <- p[H] X for a HOST tensor or array X (N x nb, row-major;
    page-locked for asynchronous copies), streamed through the device panel
    by panel with the copies overlapping the filter.  Asynchronous on
    `stream`: synchronise it before reading X."""
    gc = np.ascontiguousarray(gc, np.float64)
    Np = len(gc) - 1
    n, nb = X.shape[0], X.shape[1]
    if hasattr(X, "device"):
        assert X.device.type == "cpu", "chebfd_filter_block_host takes a host block"
        ld = X.stride(0)
        dt = dtype_of(X)
    else:
        ld = X.strides[0] // X.itemsize
        dt = {np.dtype(np.complex64): C64, np.dtype(np.complex128): C128,
              np.dtype(np.float32): R32, np.dtype(np.float64): R64}[X.dtype]
    _check(lib().chebfd_filter_block_host(H.handle, alpha, beta, gc.ctypes.data_as(c_dp), Np,
                                          _ptr(X), ld, nb, dt, _stream(stream)),
           "chebfd_filter_block_host")


def chebfd_filter_block_df(H, alpha, beta, gc, X, stream=None):
    """In place, double-float arithmetic: X <- p[H] X for an FP64 device block X."""
    gc = np.ascontiguousarray(gc, np.float64)
    Np = len(gc) - 1
    n, nb = X.shape[0], X.shape[1]
    _check(lib().chebfd_filter_block_df(H.handle, alpha, beta, gc.ctypes.data_as(c_dp), Np,
                                        _ptr(X), X.stride(0), nb, dtype_of(X), _stream(stream)),
           "chebfd_filter_block_df")


GRAM_METHODS = {"fp64": 0, "double_float": 1, "tensor": 2}


def chebfd_gram(A, B=None, method="tensor", stream=None):
    """A^H B (m x m device tensor) for device blocks A, B (N x m, R64/C128):
    the tall Gram product of steps 6-7 by cuBLAS FP64 ("fp64"), the
    double-float kernel ("double_float") or the bf16 tensor-core split
    ("tensor")."""
    import torch
    B = A if B is None else B
    n, m = A.shape[0], A.shape[1]
    assert B.shape[0] == n and B.shape[1] == m and A.dtype == B.dtype
    C = torch.empty((m, m), dtype=A.dtype, device=A.device)
    _check(lib().chebfd_gram(_ptr(A), A.stride(0), _ptr(B), B.stride(0), n, m, dtype_of(A),
                             _ptr(C), GRAM_METHODS[method], _stream(stream)), "chebfd_gram")
    # the library stores C[p + q m] = sum_i A[i,p] conj(B[i,q]) column-major: read
    # row-major that is C_rm[q, p]; A^H B [p, q] = conj(C_rm[q, p])
    return torch.conj_physical(C.T) if C.is_complex() else C.T


def chebfd_block_update(Y, M, method="tensor", stream=None):
    """Y @ M for a device block Y (N x k) and a device k x r matrix M (R64/C128):
    the tall block update of steps 6-7 by cuBLAS FP64 ("fp64"), the
    double-float kernel ("double_float") or the bf16 tensor-core split
    ("tensor").  Returns a new N x r device tensor."""
    import torch
    n, k = Y.shape[0], Y.shape[1]
    r = M.shape[1]
    assert M.shape[0] == k and M.dtype == Y.dtype
    # the library takes conj(M) column-major: that is M^H stored row-major
    # (conj_physical: a lazy conj() would hand the library unconjugated memory)
    Mc = torch.conj_physical(M).T.contiguous() if M.is_complex() else M.T.contiguous()
    T = torch.empty((n, r), dtype=Y.dtype, device=Y.device)
    _check(lib().chebfd_block_update(_ptr(Y), Y.stride(0), n, k, _ptr(Mc), k, r, _ptr(T),
                                     T.stride(0), dtype_of(Y), GRAM_METHODS[method],
                                     _stream(stream)), "chebfd_block_update")
    return T


def chebfd_chebyshev_step(H, alpha, beta, c, U, W, Y, stream=None):
    """W <- 2(alpha H + beta) U - W ; Y <- Y + c W (one fused step)."""
    n, nb = U.shape[0], U.shape[1]
    ld = U.stride(0)
    assert W.stride(0) == ld and Y.stride(0) == ld
    _check(lib().chebfd_chebyshev_step(H.handle, alpha, beta, c, _ptr(U), _ptr(W), _ptr(Y), ld, nb,
                                       dtype_of(U), _stream(stream)), "chebfd_chebyshev_step")


def chebfd_kpm_moments(H, alpha, beta, M, R, seed=0, stream=None):
    mu = np.zeros(M)
    _check(lib().chebfd_kpm_moments(H.handle, alpha, beta, M, R, seed, mu.ctypes.data_as(c_dp),
                                    _stream(stream)), "chebfd_kpm_moments")
    return mu


def chebfd_orthonormalize(Y, seed=0, refill_counter=0, stream=None):
    """In place SVQB of a device FP64 block; returns (rank, new refill counter)."""
    n, ns = Y.shape[0], Y.shape[1]
    cnt = ctypes.c_int64(refill_counter)
    rank = ctypes.c_int32(0)
    _check(lib().chebfd_orthonormalize(_ptr(Y), n, ns, Y.stride(0), dtype_of(Y), seed,
                                       ctypes.byref(cnt), ctypes.byref(rank), _stream(stream)),
           "chebfd_orthonormalize")
    return rank.value, cnt.value


def chebfd_rayleigh_ritz(H, Y, HV=None, stream=None):
    """In place: Y <- Ritz vectors; returns (theta, residuals) as numpy arrays."""
    ns = Y.shape[1]
    theta = np.zeros(ns)
    res = np.zeros(ns)
    _check(lib().chebfd_rayleigh_ritz(H.handle, _ptr(Y), Y.stride(0), ns, dtype_of(Y),
                                      theta.ctypes.data_as(c_dp), res.ctypes.data_as(c_dp),
                                      _ptr(HV), _stream(stream)), "chebfd_rayleigh_ritz")
    return theta, res


def chebfd_harmonic_ritz(H, Y, tau, stream=None):
    """In place: Y (orthonormal) <- unit harmonic Ritz vectors for the target
    tau; returns (Rayleigh quotients, residuals) as numpy arrays."""
    ns = Y.shape[1]
    theta = np.zeros(ns)
    res = np.zeros(ns)
    _check(lib().chebfd_harmonic_ritz(H.handle, _ptr(Y), Y.stride(0), ns, dtype_of(Y), float(tau),
                                      theta.ctypes.data_as(c_dp), res.ctypes.data_as(c_dp),
                                      _stream(stream)), "chebfd_harmonic_ritz")
    return theta, res


def chebfd_residuals(H, V, theta, stream=None):
    k = V.shape[1]
    theta = np.ascontiguousarray(theta, np.float64)
    res = np.zeros(k)
    _check(lib().chebfd_residuals(H.handle, _ptr(V), theta.ctypes.data_as(c_dp), V.stride(0), k,
                                  dtype_of(V), res.ctypes.data_as(c_dp), _stream(stream)),
           "chebfd_residuals")
    return res


def chebfd_convert_block(X, Y, stream=None):
    """Y <- X with a change of precision (device blocks of equal shape)."""
    _check(lib().chebfd_convert_block(_ptr(X), dtype_of(X), X.stride(0), _ptr(Y), dtype_of(Y),
                                      Y.stride(0), X.shape[0], X.shape[1], _stream(stream)),
           "chebfd_convert_block")


EXTRACTION = {"ritz": 0, "harmonic": 1}


def chebfd_solve(H, lam_lo, lam_hi, ns, Np, eps=1e-9, kernel="lanczos", mu=2.0, nb=0,
                 precision="fp64", max_iter=50, seed=0, a=0.0, b=0.0, lanczos_steps=30,
                 stream=None, extraction="ritz", window_inset=0.0, adaptive=False,
                 locking=False):
    """Run ChebFD; returns a dict with lambda, res (numpy), V (torch, device) and the log.
    extraction="harmonic" uses harmonic Ritz pairs for the window centre;
    window_inset=f filters with the window narrowed by f of the half-width;
    adaptive=True sets N_p from the first filter's moments (the log shows it);
    locking=True locks converged pairs out of the search block."""
    p = Params(lam_lo=lam_lo, lam_hi=lam_hi, eps=eps, a=a, b=b, mu=mu, ns=ns, Np=Np,
               kernel=KERNEL_IDS[kernel] if isinstance(kernel, str) else int(kernel), nb=nb,
               precision=PRECISION[precision], max_iter=max_iter,
               lanczos_steps=lanczos_steps,
               flags=EXTRACTION[extraction] | (2 if adaptive else 0) | (4 if locking else 0),
               seed=seed, window_inset=window_inset)
    h = c_vp()
    st = lib().chebfd_solve(H.handle, ctypes.byref(p), _stream(stream), ctypes.byref(h))
    if st not in (0, 5) or not h:
        _check(st, "chebfd_solve")
    try:
        return _result_dict(h, H.n, H.is_complex, st=st, stream=stream)
    finally:
        lib().chebfd_result_destroy(h)


def _iterations(h):
    """The per-iteration records of a result handle, as a list of dicts."""
    cnt = ctypes.c_int32()
    _check(lib().chebfd_result_iterations(h, None, 0, ctypes.byref(cnt)),
           "chebfd_result_iterations")
    recs = (IterationInfo * max(cnt.value, 1))()
    _check(lib().chebfd_result_iterations(h, recs, cnt.value, ctypes.byref(cnt)),
           "chebfd_result_iterations")
    return [{f: getattr(recs[i], f) for f, _ in IterationInfo._fields_}
            for i in range(cnt.value)]


class Ensemble:
    """Owner of a chebfd_ensemble handle (block-diagonal ensemble of matrices)."""

    def __init__(self, handle):
        self.handle = handle
        self._refresh()

    def _refresh(self):
        n = ctypes.c_int64()
        cnt = ctypes.c_int32()
        C, panel, tile = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().chebfd_ensemble_info(self.handle, ctypes.byref(n), ctypes.byref(cnt), None,
                                          ctypes.byref(C), ctypes.byref(panel),
                                          ctypes.byref(tile)), "chebfd_ensemble_info")
        offs = np.zeros(cnt.value + 1, np.int64)
        _check(lib().chebfd_ensemble_info(self.handle, None, None, offs.ctypes.data_as(c_i64p),
                                          None, None, None), "chebfd_ensemble_info")
        self.n, self.count, self.offsets = n.value, cnt.value, offs
        self.sell_C, self.panel, self.tile = C.value, panel.value, tile.value

    def set_coeffs(self, alpha, beta, gc, stream=None):
        alpha = np.ascontiguousarray(alpha, np.float64)
        beta = np.ascontiguousarray(beta, np.float64)
        gc = np.ascontiguousarray(gc, np.float64)
        Np = gc.shape[1] - 1
        _check(lib().chebfd_ensemble_set_coeffs(self.handle, alpha.ctypes.data_as(c_dp),
                                                beta.ctypes.data_as(c_dp), gc.ctypes.data_as(c_dp),
                                                Np, _stream(stream)), "chebfd_ensemble_set_coeffs")

    def set_launch(self, panel=0, tile=0):
        _check(lib().chebfd_ensemble_set_launch(self.handle, panel, tile),
               "chebfd_ensemble_set_launch")
        self._refresh()

    def filter(self, X, use_graph=True, stream=None):
        _check(lib().chebfd_ensemble_filter(self.handle, _ptr(X), X.stride(0), X.shape[1],
                                            dtype_of(X), 1 if use_graph else 0, _stream(stream)),
               "chebfd_ensemble_filter")

    def close(self):
        if self.handle:
            _check(lib().chebfd_ensemble_destroy(self.handle), "chebfd_ensemble_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def chebfd_ensemble_create(matrices, sell_C=1, stream=None):
    arr = (c_vp * len(matrices))(*[m.handle for m in matrices])
    h = c_vp()
    _check(lib().chebfd_ensemble_create(arr, len(matrices), sell_C, _stream(stream),
                                        ctypes.byref(h)), "chebfd_ensemble_create")
    return Ensemble(h)


def chebfd_ensemble_autotune(matrices, X, stream=None):
    """Returns (ensemble with the fastest layout and launch shape, ms per step)."""
    arr = (c_vp * len(matrices))(*[m.handle for m in matrices])
    h = c_vp()
    ms = ctypes.c_double()
    _check(lib().chebfd_ensemble_autotune(arr, len(matrices), _ptr(X), X.stride(0), X.shape[1],
                                          dtype_of(X), _stream(stream), ctypes.byref(h),
                                          ctypes.byref(ms)), "chebfd_ensemble_autotune")
    return Ensemble(h), ms.value


def _result_dict(h, n, is_complex, st=0, vectors=True, stream=None):
    import torch
    info = ResultInfo()
    _check(lib().chebfd_result_get(h, ctypes.byref(info)), "chebfd_result_get")
    nev = info.nev
    lam = np.ctypeslib.as_array(info.lambda_, (nev,)).copy() if nev else np.zeros(0)
    res = np.ctypeslib.as_array(info.res, (nev,)).copy() if nev else np.zeros(0)
    V = None
    if vectors:
        dt = torch.complex128 if is_complex else torch.float64
        V = torch.empty((n, max(nev, 1)), dtype=dt, device="cuda")[:, :nev]
        if nev:
            _check(lib().chebfd_result_copy_vectors(h, _ptr(V), V.stride(0), _stream(stream)),
                   "chebfd_result_copy_vectors")
    return dict(lam=lam, res=res, V=V, nev=nev, iterations=info.iterations,
                converged=bool(info.converged), fp64_iterations=info.fp64_iterations,
                n_mvm=info.n_mvm, a=info.a, b=info.b, seconds_filter=info.seconds_filter,
                seconds_dense=info.seconds_dense, seconds_total=info.seconds_total,
                status=STATUS[st], log=_iterations(h))


def chebfd_solve_batched(E, matrices, a, b, lam_lo, lam_hi, ns, Np, eps=1e-9, kernel="lanczos",
                         mu=2.0, precision="fp64", max_iter=50, seed=0, vectors=False,
                         stream=None, window_inset=0.0):
    """ChebFD on every ensemble member; returns (list of per-member dicts, iterations)."""
    cnt = len(matrices)
    arr = (c_vp * cnt)(*[m.handle for m in matrices])
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    p = Params(lam_lo=lam_lo, lam_hi=lam_hi, eps=eps, a=0.0, b=0.0, mu=mu, ns=ns, Np=Np,
               kernel=KERNEL_IDS[kernel] if isinstance(kernel, str) else int(kernel), nb=0,
               precision=PRECISION[precision], max_iter=max_iter, lanczos_steps=0,
               flags=0, seed=seed, window_inset=window_inset)
    outs = (c_vp * cnt)()
    its = ctypes.c_int32()
    _check(lib().chebfd_solve_batched(E.handle, arr, a.ctypes.data_as(c_dp),
                                      b.ctypes.data_as(c_dp), ctypes.byref(p), _stream(stream),
                                      outs, ctypes.byref(its)), "chebfd_solve_batched")
    results = []
    try:
        for i in range(cnt):
            results.append(_result_dict(outs[i], matrices[i].n, matrices[i].is_complex,
                                        vectors=vectors))
    finally:
        for i in range(cnt):
            if outs[i]:
                lib().chebfd_result_destroy(outs[i])
    return results, its.value


def chebfd_param_features(H, lam_lo, lam_hi, m_feat=64, a=0.0, b=0.0, seed=0, stream=None):
    f = np.zeros(m_feat + 3)
    nt = ctypes.c_double()
    _check(lib().chebfd_param_features(H.handle, a, b, lam_lo, lam_hi, m_feat, seed,
                                       f.ctypes.data_as(c_dp), ctypes.byref(nt), _stream(stream)),
           "chebfd_param_features")
    return f, nt.value


def chebfd_choose_params(H, lam_lo, lam_hi, mlp=None, m_feat=64, a=0.0, b=0.0, seed=0,
                         stream=None):
    """(n_s, N_p, kernel name, N_T estimate) from the paper's rules or the MLP."""
    ns, Np, k = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    nt = ctypes.c_double()
    _check(lib().chebfd_choose_params(H.handle, a, b, lam_lo, lam_hi,
                                      mlp.handle if mlp is not None else None, m_feat, seed,
                                      ctypes.byref(ns), ctypes.byref(Np), ctypes.byref(k),
                                      ctypes.byref(nt), _stream(stream)), "chebfd_choose_params")
    return ns.value, Np.value, KERNEL_NAMES[k.value], nt.value


class MLP:
    """Device MLP (n_in -> n_h -> n_h -> 3) trained by the library's kernels."""

    def __init__(self, n_in, n_hidden=128):
        h = c_vp()
        _check(lib().chebfd_mlp_create(n_in, n_hidden, 3, ctypes.byref(h)), "chebfd_mlp_create")
        self.handle = h
        self.n_in, self.n_hidden = n_in, n_hidden
        c = ctypes.c_int64()
        _check(lib().chebfd_mlp_num_params(h, ctypes.byref(c)), "chebfd_mlp_num_params")
        self.count = c.value

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, np.float32)
        assert flat.size == self.count
        _check(lib().chebfd_mlp_set_params(self.handle, flat.ctypes.data_as(
            ctypes.POINTER(ctypes.c_float)), self.count), "chebfd_mlp_set_params")

    def get_params(self):
        p = np.zeros(self.count, np.float32)
        g = np.zeros(self.count, np.float32)
        fp = ctypes.POINTER(ctypes.c_float)
        _check(lib().chebfd_mlp_get_params(self.handle, p.ctypes.data_as(fp),
                                           g.ctypes.data_as(fp), self.count),
               "chebfd_mlp_get_params")
        return p, g

    def forward(self, X, stream=None):
        import torch
        Z = torch.empty((X.shape[0], 3), dtype=torch.float32, device=X.device)
        _check(lib().chebfd_mlp_forward(self.handle, _ptr(X), X.shape[0], _ptr(Z),
                                        _stream(stream)), "chebfd_mlp_forward")
        return Z

    def loss_grad(self, X, T, stream=None):
        loss = ctypes.c_float()
        _check(lib().chebfd_mlp_loss_grad(self.handle, _ptr(X), _ptr(T), X.shape[0],
                                          ctypes.byref(loss), _stream(stream)),
               "chebfd_mlp_loss_grad")
        return loss.value

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        _check(lib().chebfd_mlp_adam(self.handle, lr, beta1, beta2, eps, _stream(stream)),
               "chebfd_mlp_adam")

    def close(self):
        if self.handle:
            _check(lib().chebfd_mlp_destroy(self.handle), "chebfd_mlp_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pack_params(P):
    """Packed parameter vector (W1, b1, W2, b2, W3, b3) of a dict of arrays."""
    return np.concatenate([np.asarray(P[k], np.float64).reshape(-1)
                           for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def unpack_params(flat, n_in, n_h, n_out=3):
    shapes = [("W1", (n_h, n_in)), ("b1", (n_h,)), ("W2", (n_h, n_h)), ("b2", (n_h,)),
              ("W3", (n_out, n_h)), ("b3", (n_out,))]
    out, o = {}, 0
    for k, s in shapes:
        n = int(np.prod(s))
        out[k] = np.asarray(flat[o:o + n], np.float64).reshape(s)
        o += n
    return out


def chebfd_random_block(X, col0=0, ns_total=None, seed=0, stream=None):
    n, nb = X.shape[0], X.shape[1]
    ns_total = nb if ns_total is None else ns_total
    _check(lib().chebfd_random_block(_ptr(X), n, X.stride(0), nb, col0, ns_total, seed,
                                     dtype_of(X), _stream(stream)), "chebfd_random_block")
