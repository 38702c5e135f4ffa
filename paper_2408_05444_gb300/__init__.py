"""Python binding of the grbk C ABI (include/grbk.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Matrices may
be numpy arrays (host), or torch tensors on the host or on a CUDA device; they
must be row-major with unit column stride.  The library (``_build/libgrbk.so``)
must have been built with ``paper_2408_05444_gb300.build.build()``; without it
every call raises, there is no fallback path.

Solver: greedy randomized block Kaczmarz for A X B = C (arXiv 2408.05444,
Algorithms 1-5).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgrbk.so")

GRBK_OK, GRBK_EINVAL, GRBK_ENOMEM, GRBK_ECUDA, GRBK_ENOTCONV, GRBK_ETIMEOUT, GRBK_ENONFINITE = range(7)
GRBK_GRBK, GRBK_RGRBK, GRBK_MWRBK, GRBK_RBK, GRBK_BK = range(5)
VARIANTS = {"grbk": GRBK_GRBK, "rgrbk": GRBK_RGRBK, "mwrbk": GRBK_MWRBK, "rbk": GRBK_RBK, "bk": GRBK_BK}
GRBK_F64, GRBK_F32 = 0, 1
GRBK_DT_F64, GRBK_DT_F32 = 0, 1
GRBK_STOP_NONE, GRBK_STOP_RELRES, GRBK_STOP_RSE = 0, 1, 2
GRBK_FORM_FULL, GRBK_FORM_ROWSPACE = 0, 1


class grbk_mat(ctypes.Structure):
    _fields_ = [("ptr", ctypes.c_void_p), ("rows", ctypes.c_int64), ("cols", ctypes.c_int64),
                ("ld", ctypes.c_int64), ("dtype", ctypes.c_int32), ("on_device", ctypes.c_int32)]


class grbk_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("refresh_T", ctypes.c_int32), ("alpha", ctypes.c_double),
                ("stop_kind", ctypes.c_int32), ("split_terms", ctypes.c_int32),
                ("x_ref", ctypes.POINTER(grbk_mat)), ("row_trace", ctypes.POINTER(ctypes.c_int32)),
                ("s_trace", ctypes.POINTER(ctypes.c_double)), ("trace_len", ctypes.c_int64),
                ("stream", ctypes.c_void_p), ("grid_ctas", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("use_gram", ctypes.c_int32), ("form", ctypes.c_int32), ("rank_tol", ctypes.c_double),
                ("band_limit", ctypes.c_int32), ("alphas", ctypes.POINTER(ctypes.c_double)),
                ("extended", ctypes.c_int32), ("tune", ctypes.c_int32), ("deferred", ctypes.c_int32)]


class grbk_csr(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("colind", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class grbk_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("relres", ctypes.c_double), ("rse", ctypes.c_double),
                ("seconds", ctypes.c_double), ("alpha", ctypes.c_double), ("iter_kernel_ms", ctypes.c_double),
                ("iter_kernel_launches", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("gram", ctypes.c_int32), ("x0_rejected", ctypes.c_int32), ("status", ctypes.c_int32),
                ("deferred", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class GrbkError(RuntimeError):
    def __init__(self, status, where):
        super().__init__(f"{where}: {grbk_strerror(status)} (status {status})")
        self.status = status


EXPORTS = ["grbk_default_opts", "grbk_create", "grbk_solve", "grbk_residual", "grbk_get_residual",
           "grbk_get_rownorms", "grbk_info", "grbk_destroy", "grbk_batch_create", "grbk_batch_solve",
           "grbk_batch_destroy", "grbk_strerror", "grbk_solve_small_noalloc", "grbk_unet_create",
           "grbk_unet_num_params", "grbk_unet_set_params", "grbk_unet_get_params", "grbk_unet_forward",
           "grbk_unet_loss_grad", "grbk_unet_train_step", "grbk_unet_destroy", "grbk_barrier_selftest",
           "grbk_form_info", "grbk_batch_info", "grbk_trim_cache", "grbk_fp64_probe", "grbk_fp64_issue_probe", "grbk_sparse_create", "grbk_sparse_cluster",
           "grbk_sparse_solve", "grbk_sparse_info", "grbk_sparse_get_residual", "grbk_sparse_destroy",
           "grbk_tune_num_variants", "grbk_tune_variant_info", "grbk_tune_choose", "grbk_tune_lookup",
           "grbk_tune_store", "grbk_tune_clear", "grbk_batch_variant", "grbk_unet_use_tensor_cores"]
GRBK_NOALLOC_MAX_SIDE = 512

_lib = None


def lib():
    """Load libgrbk.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgrbk.so is not built ({LIB_PATH}); run paper_2408_05444_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        vp, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        L.grbk_default_opts.argtypes = [P(grbk_opts)]
        L.grbk_default_opts.restype = None
        L.grbk_create.argtypes = [P(vp), P(grbk_mat), P(grbk_mat), P(grbk_mat), P(grbk_opts)]
        L.grbk_create.restype = i32
        L.grbk_solve.argtypes = [vp, i32, dbl, P(grbk_mat), dbl, i64, u64, P(grbk_mat), P(grbk_result)]
        L.grbk_solve.restype = i32
        L.grbk_residual.argtypes = [vp, P(grbk_mat), P(grbk_mat)]
        L.grbk_residual.restype = i32
        L.grbk_get_residual.argtypes = [vp, P(grbk_mat)]
        L.grbk_get_residual.restype = i32
        L.grbk_get_rownorms.argtypes = [vp, vp, i32]
        L.grbk_get_rownorms.restype = i32
        L.grbk_info.argtypes = [vp, P(i64), P(dbl)]
        L.grbk_info.restype = i32
        L.grbk_trim_cache.argtypes = []
        L.grbk_trim_cache.restype = None
        L.grbk_form_info.argtypes = [vp, P(i32), P(i64)]
        L.grbk_form_info.restype = i32
        L.grbk_destroy.argtypes = [vp]
        L.grbk_destroy.restype = None
        L.grbk_batch_create.argtypes = [P(vp), i32, P(grbk_mat), P(grbk_mat), P(grbk_mat), P(grbk_opts)]
        L.grbk_batch_create.restype = i32
        L.grbk_batch_solve.argtypes = [vp, i32, dbl, P(grbk_mat), dbl, P(dbl), i64, u64, P(grbk_mat),
                                       P(grbk_result)]
        L.grbk_batch_solve.restype = i32
        L.grbk_batch_info.argtypes = [vp, i32, P(i32), P(i32)]
        L.grbk_batch_info.restype = i32
        L.grbk_batch_destroy.argtypes = [vp]
        L.grbk_batch_destroy.restype = None
        L.grbk_solve_small_noalloc.argtypes = [vp, vp, vp, i32, i32, i32, i32, i32, dbl, dbl, dbl, i64, u64, vp,
                                               P(i64), P(dbl), vp]
        L.grbk_solve_small_noalloc.restype = i32
        L.grbk_unet_create.argtypes = [P(vp), i32, vp]
        L.grbk_unet_create.restype = i32
        L.grbk_unet_num_params.argtypes = [vp]
        L.grbk_unet_num_params.restype = i64
        L.grbk_unet_set_params.argtypes = [vp, vp, i32]
        L.grbk_unet_set_params.restype = i32
        L.grbk_unet_get_params.argtypes = [vp, vp, i32]
        L.grbk_unet_get_params.restype = i32
        L.grbk_unet_forward.argtypes = [vp, vp, i32, i32, i32, vp]
        L.grbk_unet_forward.restype = i32
        L.grbk_unet_loss_grad.argtypes = [vp, vp, vp, i32, i32, i32, P(dbl), vp, i32]
        L.grbk_unet_loss_grad.restype = i32
        L.grbk_unet_train_step.argtypes = [vp, vp, vp, i32, i32, i32, ctypes.c_float, P(dbl)]
        L.grbk_unet_train_step.restype = i32
        L.grbk_unet_use_tensor_cores.argtypes = [vp, i32]
        L.grbk_unet_use_tensor_cores.restype = i32
        L.grbk_unet_destroy.argtypes = [vp]
        L.grbk_unet_destroy.restype = None
        L.grbk_barrier_selftest.argtypes = [i32, vp]
        L.grbk_barrier_selftest.restype = i32
        L.grbk_sparse_create.argtypes = [P(vp), i32, P(grbk_csr), P(grbk_csr), P(grbk_mat), P(grbk_opts)]
        L.grbk_sparse_create.restype = i32
        L.grbk_sparse_solve.argtypes = [vp, i32, dbl, dbl, P(dbl), i64, u64, P(grbk_mat), P(grbk_result)]
        L.grbk_sparse_solve.restype = i32
        L.grbk_sparse_info.argtypes = [vp, i32, P(i64), P(dbl)]
        L.grbk_sparse_info.restype = i32
        L.grbk_sparse_cluster.argtypes = [vp, P(i32)]
        L.grbk_sparse_cluster.restype = i32
        L.grbk_sparse_get_residual.argtypes = [vp, i32, vp, vp]
        L.grbk_sparse_get_residual.restype = i32
        L.grbk_sparse_destroy.argtypes = [vp]
        L.grbk_sparse_destroy.restype = None
        L.grbk_tune_num_variants.argtypes = []
        L.grbk_tune_num_variants.restype = i32
        L.grbk_tune_variant_info.argtypes = [i32, P(i32), P(i32)]
        L.grbk_tune_variant_info.restype = i32
        L.grbk_tune_choose.argtypes = [P(dbl), i32]
        L.grbk_tune_choose.restype = i32
        L.grbk_tune_lookup.argtypes = [i32, i32, i32, i32, i32, i32, P(i32)]
        L.grbk_tune_lookup.restype = i32
        L.grbk_tune_store.argtypes = [i32, i32, i32, i32, i32, i32, i32]
        L.grbk_tune_store.restype = i32
        L.grbk_tune_clear.argtypes = []
        L.grbk_tune_clear.restype = None
        L.grbk_batch_variant.argtypes = [vp, i32, P(i32), P(dbl)]
        L.grbk_batch_variant.restype = i32
        L.grbk_fp64_probe.argtypes = [i64, i32, P(dbl), P(dbl), vp]
        L.grbk_fp64_probe.restype = i32
        L.grbk_fp64_issue_probe.argtypes = [i32, i32, i32, i64, P(dbl), vp]
        L.grbk_fp64_issue_probe.restype = i32
        L.grbk_strerror.argtypes = [i32]
        L.grbk_strerror.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def mat(x, out=False) -> grbk_mat:
    """Describe a 2-D FP32 or FP64 numpy array or torch tensor for the C ABI.

    The library trusts a descriptor (pointer, rows, cols, row stride), so
    everything it cannot express is refused here, before a pointer leaves
    Python: other ranks or dtypes, a column stride other than 1, a row stride
    below the column count (flipped views, broadcast or expanded rows), and,
    for an output (out=True), a read-only numpy array."""
    if _is_torch(x):
        import torch
        if x.dim() != 2:
            raise ValueError(f"need a 2-D tensor, got {x.dim()}-D")
        if x.dtype not in (torch.float64, torch.float32):
            raise TypeError(f"need a float32 or float64 tensor, got {x.dtype}")
        rows, cols = x.shape
        rs, cs = x.stride()
        ptr, f64, dev = x.data_ptr(), x.dtype == torch.float64, 1 if x.is_cuda else 0
    elif isinstance(x, np.ndarray):
        if x.ndim != 2:
            raise ValueError(f"need a 2-D array, got {x.ndim}-D")
        if x.dtype not in (np.dtype(np.float64), np.dtype(np.float32)):
            raise TypeError(f"need a native float32 or float64 array, got {x.dtype}")
        if out and not x.flags.writeable:
            raise ValueError("output array is read-only")
        rows, cols = x.shape
        it = x.itemsize
        if x.strides[0] % it or x.strides[1] % it:
            raise ValueError("strides are not whole elements")
        rs, cs = x.strides[0] // it, x.strides[1] // it
        ptr, f64, dev = x.ctypes.data, x.dtype == np.float64, 0
    else:
        raise TypeError(f"need a numpy array or a torch tensor, got {type(x).__name__}")
    if cols > 1 and cs != 1:
        raise ValueError("need unit column stride (row-major rows)")
    if rows > 1 and rs < cols:
        raise ValueError(f"row stride {rs} is below the column count {cols} (flipped, broadcast or expanded rows)")
    ld = rs if rows > 1 else cols
    return grbk_mat(ptr, rows, cols, max(ld, cols), GRBK_DT_F64 if f64 else GRBK_DT_F32, dev)


def _stream_ptr(stream):
    return 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)


def _cuda_f32_tensor(t, name, ndim):
    """Pointer of a contiguous FP32 CUDA tensor of rank ndim (raises otherwise)."""
    if not _is_torch(t):
        raise TypeError(f"{name}: need a torch tensor, got {type(t).__name__}")
    import torch
    if t.dtype != torch.float32:
        raise TypeError(f"{name}: need float32, got {t.dtype}")
    if not t.is_cuda:
        raise ValueError(f"{name}: need a CUDA tensor")
    if t.dim() != ndim or not t.is_contiguous():
        raise ValueError(f"{name}: need a contiguous {ndim}-D tensor, got shape {tuple(t.shape)}")
    return t.data_ptr()


def grbk_strerror(status: int) -> str:
    return lib().grbk_strerror(int(status)).decode()


def grbk_default_opts(**kw) -> grbk_opts:
    o = grbk_opts()
    lib().grbk_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class _Keep:
    """Holds Python objects that back pointers inside an opts struct."""


def _make_opts(opts, precision=None, refresh_T=None, alpha=None, stop_kind=None, split_terms=None,
               x_ref=None, trace_len=0, stream=None, grid_ctas=None, check_every=None, use_gram=None,
               form=None, rank_tol=None, band_limit=None, alphas=None, extended=None, tune=None, deferred=None):
    o = grbk_default_opts() if opts is None else opts
    keep = _Keep()
    if precision is not None:
        o.precision = {"f64": GRBK_F64, "f32": GRBK_F32}.get(precision, precision)
    if refresh_T is not None:
        o.refresh_T = refresh_T
    if alpha is not None:
        o.alpha = alpha
    if stop_kind is not None:
        o.stop_kind = {"none": GRBK_STOP_NONE, "relres": GRBK_STOP_RELRES, "rse": GRBK_STOP_RSE}.get(stop_kind, stop_kind)
    if split_terms is not None:
        o.split_terms = split_terms
    if grid_ctas is not None:
        o.grid_ctas = grid_ctas
    if check_every is not None:
        o.check_every = check_every
    if use_gram is not None:
        o.use_gram = {True: 1, False: -1}.get(use_gram, use_gram)
    if form is not None:
        o.form = {"full": GRBK_FORM_FULL, "rowspace": GRBK_FORM_ROWSPACE}.get(form, form)
    if rank_tol is not None:
        o.rank_tol = rank_tol
    if band_limit is not None:
        o.band_limit = band_limit
    if extended is not None:
        o.extended = int(bool(extended))
    if tune is not None:
        o.tune = int(bool(tune))
    if deferred is not None:
        o.deferred = {True: 1, False: -1}.get(deferred, deferred)
    if alphas is not None:
        keep.alphas = np.ascontiguousarray(alphas, dtype=np.float64)
        o.alphas = keep.alphas.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    if stream is not None:
        o.stream = stream if isinstance(stream, int) else stream.cuda_stream
    if x_ref is not None:
        keep.xr_arr = x_ref
        keep.xr = mat(x_ref)
        o.x_ref = ctypes.pointer(keep.xr)
    if trace_len > 0:
        keep.rows = np.full(trace_len, -1, dtype=np.int32)
        keep.S = np.zeros(trace_len, dtype=np.float64)
        o.row_trace = keep.rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        o.s_trace = keep.S.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        o.trace_len = trace_len
    return o, keep


class Context:
    """Owns a grbk_ctx* and the host buffers its opts point to."""

    def __init__(self, handle, keep, opts):
        self.handle = handle
        self.keep = keep
        self.opts = opts

    @property
    def row_trace(self):
        return getattr(self.keep, "rows", None)

    @property
    def s_trace(self):
        return getattr(self.keep, "S", None)

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                lib().grbk_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def grbk_create(A, B, C, opts=None, **kw) -> Context:
    """grbk_create(A, B, C, opts) -- set up one system; keyword options fill
    grbk_opts (precision='f64'|'f32', refresh_T, alpha, stop_kind, split_terms,
    x_ref, trace_len, stream, grid_ctas, check_every, use_gram, form='full'|'rowspace',
    rank_tol, deferred)."""
    o, keep = _make_opts(opts, **kw)
    h = ctypes.c_void_p()
    mA, mB, mC = mat(A), mat(B), mat(C)
    st = lib().grbk_create(ctypes.byref(h), ctypes.byref(mA), ctypes.byref(mB), ctypes.byref(mC), ctypes.byref(o))
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_create")
    return Context(h.value, keep, o)


def grbk_solve(ctx: Context, variant, theta=0.5, X0=None, tol=0.0, maxit=1000, seed=0, X_out=None):
    """grbk_solve -> (status, result dict).  X_out (p x q) is written in place."""
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    res = grbk_result()
    m0 = mat(X0) if X0 is not None else None
    mo = mat(X_out, out=True) if X_out is not None else None
    st = lib().grbk_solve(ctx.handle, v, float(theta), ctypes.byref(m0) if m0 is not None else None, float(tol),
                          int(maxit), int(seed), ctypes.byref(mo) if mo is not None else None, ctypes.byref(res))
    if st not in (GRBK_OK, GRBK_ENOTCONV):
        raise GrbkError(st, "grbk_solve")
    return st, res.as_dict()


def grbk_residual(ctx: Context, X, R_out):
    mx, mr = mat(X), mat(R_out, out=True)
    st = lib().grbk_residual(ctx.handle, ctypes.byref(mx), ctypes.byref(mr))
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_residual")


def grbk_get_residual(ctx: Context, R_out):
    mr = mat(R_out, out=True)
    st = lib().grbk_get_residual(ctx.handle, ctypes.byref(mr))
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_get_residual")


def grbk_get_rownorms(ctx: Context, s_out):
    """s_out <- s_i = ||R_i||^2 (i < m): a contiguous FP64 array or tensor
    (host or CUDA) with at least m entries."""
    m = grbk_info(ctx)[0][0]
    if _is_torch(s_out):
        import torch
        if s_out.dtype != torch.float64 or not s_out.is_contiguous() or s_out.numel() < m:
            raise ValueError(f"s_out: need a contiguous float64 tensor of at least {m} entries")
        ptr, dev = s_out.data_ptr(), 1 if s_out.is_cuda else 0
    elif isinstance(s_out, np.ndarray):
        if (s_out.dtype != np.float64 or not s_out.flags.c_contiguous or not s_out.flags.writeable
                or s_out.size < m):
            raise ValueError(f"s_out: need a writable contiguous float64 array of at least {m} entries")
        ptr, dev = s_out.ctypes.data, 0
    else:
        raise TypeError(f"s_out: need a numpy array or a torch tensor, got {type(s_out).__name__}")
    st = lib().grbk_get_rownorms(ctx.handle, ptr, dev)
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_get_rownorms")


def grbk_info(ctx: Context):
    dims = (ctypes.c_int64 * 4)()
    al = ctypes.c_double()
    st = lib().grbk_info(ctx.handle, dims, ctypes.byref(al))
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_info")
    return tuple(dims), al.value


def grbk_form_info(ctx: Context):
    """-> ('full' | 'rowspace', columns of the kept residual: n or rank B)."""
    f = ctypes.c_int32()
    cols = ctypes.c_int64()
    st = lib().grbk_form_info(ctx.handle, ctypes.byref(f), ctypes.byref(cols))
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_form_info")
    return ("full", "rowspace")[f.value], cols.value


def grbk_trim_cache():
    """Return the device blocks kept from destroyed contexts to the driver."""
    lib().grbk_trim_cache()


def grbk_destroy(ctx: Context):
    if ctx.handle:
        lib().grbk_destroy(ctx.handle)
        ctx.handle = None


class Batch:
    def __init__(self, handle, keep):
        self.handle = handle
        self.keep = keep

    @property
    def row_trace(self):
        return getattr(self.keep, "rows_view", None)

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                lib().grbk_batch_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def _mat_array(xs, out=False):
    arr = (grbk_mat * len(xs))()
    for i, x in enumerate(xs):
        arr[i] = mat(x, out=out)
    return arr


def grbk_batch_create(As, Bs, Cs, opts=None, trace_len=0, **kw) -> Batch:
    """Batched systems; trace_len > 0 records each system's first trace_len rows
    (available as batch.row_trace, shape nsys x trace_len); alphas: one step per
    system (grbk_opts.alphas)."""
    if kw.get("alphas") is not None and len(kw["alphas"]) != len(As):
        raise ValueError(f"alphas needs {len(As)} entries, got {len(kw['alphas'])}")
    o, keep = _make_opts(opts, trace_len=trace_len * len(As), **kw)
    if trace_len > 0:
        o.trace_len = trace_len
        keep.rows_view = keep.rows.reshape(len(As), trace_len)
    h = ctypes.c_void_p()
    a, b, c = _mat_array(As), _mat_array(Bs), _mat_array(Cs)
    st = lib().grbk_batch_create(ctypes.byref(h), len(As), a, b, c, ctypes.byref(o))
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_batch_create")
    return Batch(h.value, keep)


def grbk_batch_info(batch: Batch, sys: int):
    """-> (half-bandwidth of A, of B) of a system on the banded path, (-1, -1) on the dense path."""
    ba, bb = ctypes.c_int32(), ctypes.c_int32()
    st = lib().grbk_batch_info(batch.handle, int(sys), ctypes.byref(ba), ctypes.byref(bb))
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_batch_info")
    return ba.value, bb.value


def grbk_batch_solve(batch: Batch, variant, theta=0.5, X0s=None, tol=0.0, targets=None, maxit=1000, seed=0,
                     X_outs=None):
    """grbk_batch_solve -> (status, list of result dicts)."""
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    n = len(X_outs) if X_outs is not None else (len(X0s) if X0s is not None else None)
    x0 = _mat_array(X0s) if X0s is not None else None
    xo = _mat_array(X_outs, out=True) if X_outs is not None else None
    tg = None
    if targets is not None:
        tgt = np.ascontiguousarray(targets, dtype=np.float64)
        tg = tgt.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        n = len(tgt)
    if n is None:
        raise ValueError("need X_outs, X0s or targets to size the results")
    res = (grbk_result * n)()
    st = lib().grbk_batch_solve(batch.handle, v, float(theta), x0, float(tol), tg, int(maxit), int(seed), xo, res)
    if st not in (GRBK_OK, GRBK_ENOTCONV):
        raise GrbkError(st, "grbk_batch_solve")
    return st, [r.as_dict() for r in res]


def grbk_batch_destroy(batch: Batch):
    if batch.handle:
        lib().grbk_batch_destroy(batch.handle)
        batch.handle = None


def grbk_solve_small_noalloc(A, B, C, X_out, variant="grbk", theta=0.5, alpha=0.0, tol=0.0, maxit=1000, seed=0,
                             stream=None):
    """grbk_solve_small_noalloc -> (status, iters, relres).  A (m x p), B (q x n),
    C (m x n) and X_out (p x q) are contiguous FP32 CUDA tensors; nothing is
    allocated by the library."""
    ptrs = [_cuda_f32_tensor(t, name, 2) for t, name in ((A, "A"), (B, "B"), (C, "C"), (X_out, "X_out"))]
    m, p = A.shape
    q, n = B.shape
    if tuple(C.shape) != (m, n) or tuple(X_out.shape) != (p, q):
        raise ValueError(f"need C {m}x{n} and X_out {p}x{q}, got {tuple(C.shape)} and {tuple(X_out.shape)}")
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    it = ctypes.c_int64(0)
    rr = ctypes.c_double(0.0)
    st = lib().grbk_solve_small_noalloc(ptrs[0], ptrs[1], ptrs[2], m, p, q, n, v, float(theta), float(alpha),
                                        float(tol), int(maxit), int(seed), ptrs[3], ctypes.byref(it),
                                        ctypes.byref(rr), _stream_ptr(stream))
    return st, it.value, rr.value


# ---------------------------------------------------------------------------
# learned warm start (U-Net)
# ---------------------------------------------------------------------------
class UNetHandle:
    def __init__(self, handle, width):
        self.handle = handle
        self.width = width

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                lib().grbk_unet_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def grbk_unet_create(width=20, stream=None) -> UNetHandle:
    h = ctypes.c_void_p()
    st = lib().grbk_unet_create(ctypes.byref(h), int(width), _stream_ptr(stream))
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_unet_create")
    return UNetHandle(h.value, width)


def grbk_unet_num_params(net: UNetHandle) -> int:
    return int(lib().grbk_unet_num_params(net.handle))


def grbk_unet_set_params(net: UNetHandle, params):
    """params: the network's flat FP32 parameter vector (grbk_unet_num_params
    entries), a host array or a host or CUDA tensor."""
    npar = grbk_unet_num_params(net)
    if _is_torch(params):
        import torch
        if params.dtype != torch.float32 or not params.is_contiguous() or params.numel() != npar:
            raise ValueError(f"params: need a contiguous float32 tensor of {npar} entries")
        st = lib().grbk_unet_set_params(net.handle, params.data_ptr(), 1 if params.is_cuda else 0)
    else:
        a = np.ascontiguousarray(params, dtype=np.float32)
        if a.size != npar:
            raise ValueError(f"params: need {npar} entries, got {a.size}")
        st = lib().grbk_unet_set_params(net.handle, a.ctypes.data, 0)
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_unet_set_params")


def grbk_unet_get_params(net: UNetHandle) -> np.ndarray:
    out = np.zeros(grbk_unet_num_params(net), dtype=np.float32)
    st = lib().grbk_unet_get_params(net.handle, out.ctypes.data, 0)
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_unet_get_params")
    return out


def _same_shape(C, T, name):
    if tuple(T.shape) != tuple(C.shape):
        raise ValueError(f"{name}: need shape {tuple(C.shape)}, got {tuple(T.shape)}")


def grbk_unet_forward(net: UNetHandle, C, X0):
    """C, X0: contiguous FP32 CUDA tensors [n, h, w]."""
    pc, px = _cuda_f32_tensor(C, "C", 3), _cuda_f32_tensor(X0, "X0", 3)
    _same_shape(C, X0, "X0")
    n, h, w = C.shape
    st = lib().grbk_unet_forward(net.handle, pc, n, h, w, px)
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_unet_forward")


def grbk_unet_loss_grad(net: UNetHandle, C, T, want_grad=True):
    pc, pt = _cuda_f32_tensor(C, "C", 3), _cuda_f32_tensor(T, "T", 3)
    _same_shape(C, T, "T")
    n, h, w = C.shape
    loss = ctypes.c_double(0.0)
    g = np.zeros(grbk_unet_num_params(net), dtype=np.float32) if want_grad else None
    st = lib().grbk_unet_loss_grad(net.handle, pc, pt, n, h, w, ctypes.byref(loss),
                                   g.ctypes.data if g is not None else None, 0)
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_unet_loss_grad")
    return loss.value, g


def grbk_unet_train_step(net: UNetHandle, C, T, lr) -> float:
    pc, pt = _cuda_f32_tensor(C, "C", 3), _cuda_f32_tensor(T, "T", 3)
    _same_shape(C, T, "T")
    n, h, w = C.shape
    loss = ctypes.c_double(0.0)
    st = lib().grbk_unet_train_step(net.handle, pc, pt, n, h, w, float(lr), ctypes.byref(loss))
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_unet_train_step")
    return loss.value


def grbk_unet_use_tensor_cores(net: UNetHandle, on=True):
    """on: True/1 tensor cores (row-halo tiles where the image allows), 2 tensor cores with
    one load per tap, False/0 SIMT."""
    st = lib().grbk_unet_use_tensor_cores(net.handle, int(on))
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_unet_use_tensor_cores")


def grbk_unet_destroy(net: UNetHandle):
    if net.handle:
        lib().grbk_unet_destroy(net.handle)
        net.handle = None


def grbk_barrier_selftest(absent_cta=-1, stream=None) -> int:
    """Status of one bounded grid barrier; absent_cta >= 0 leaves that CTA out."""
    return int(lib().grbk_barrier_selftest(int(absent_cta), _stream_ptr(stream)))


def grbk_fp64_probe(iters=1 << 16, blocks_per_sm=8, stream=None):
    """grbk_fp64_probe -> (FP64 FMAs per second, milliseconds of the timed launch)."""
    r, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = lib().grbk_fp64_probe(int(iters), int(blocks_per_sm), ctypes.byref(r), ctypes.byref(ms), _stream_ptr(stream))
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_fp64_probe")
    return r.value, ms.value


FP64_OPS = {"add": 0, "fma": 1, "mul": 2, "div": 3, "cvt": 4}


def grbk_fp64_issue_probe(op="add", warps=1, active_lanes=32, iters=2048, stream=None) -> float:
    """grbk_fp64_issue_probe -> SM clock cycles per FP64 operation per warp."""
    c = ctypes.c_double(0.0)
    st = lib().grbk_fp64_issue_probe(int(FP64_OPS[op]), int(warps), int(active_lanes), int(iters), ctypes.byref(c),
                                     _stream_ptr(stream))
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_fp64_issue_probe")
    return c.value


# ---------------------------------------------------------------------------
# sparse A and B (CSR)
# ---------------------------------------------------------------------------
def csr_arrays(M):
    """(rows, cols, rowptr int64, colind int32, val float64) of a scipy.sparse
    matrix or a dense 2-D array (its nonzeros, row by row, ascending columns)."""
    if hasattr(M, "tocsr"):
        M = M.tocsr()
        M.sum_duplicates()
        M.sort_indices()
        return (int(M.shape[0]), int(M.shape[1]), np.ascontiguousarray(M.indptr, dtype=np.int64),
                np.ascontiguousarray(M.indices, dtype=np.int32), np.ascontiguousarray(M.data, dtype=np.float64))
    D = np.asarray(M, dtype=np.float64)
    if D.ndim != 2:
        raise ValueError("need a 2-D matrix")
    nz = D != 0
    rowptr = np.concatenate([[0], np.cumsum(nz.sum(axis=1))]).astype(np.int64)
    r, c = np.nonzero(nz)
    return (D.shape[0], D.shape[1], rowptr, np.ascontiguousarray(c, dtype=np.int32),
            np.ascontiguousarray(D[r, c], dtype=np.float64))


def _csr(M, keep):
    rows, cols, rp, ci, v = csr_arrays(M)
    keep.append((rp, ci, v))
    return grbk_csr(rows, cols, len(v), rp.ctypes.data, ci.ctypes.data if len(ci) else None,
                    v.ctypes.data if len(v) else None)


class Sparse:
    def __init__(self, handle, keep, nsys, trace_len):
        self.handle = handle
        self.keep = keep
        self.nsys = nsys
        self.trace_len = trace_len

    @property
    def row_trace(self):
        rows = getattr(self.keep, "rows", None)
        return None if rows is None else rows.reshape(self.nsys, self.trace_len)

    @property
    def s_trace(self):
        S = getattr(self.keep, "S", None)
        return None if S is None else S.reshape(self.nsys, self.trace_len)

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                lib().grbk_sparse_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def grbk_sparse_create(As, Bs, Cs, opts=None, trace_len=0, **kw) -> Sparse:
    """Systems with sparse A_s, B_s (scipy.sparse or dense arrays, sent as CSR)
    and dense C_s; trace_len > 0 records each system's first trace_len rows
    and ||R^k||_F^2 (sparse.row_trace, sparse.s_trace: nsys x trace_len)."""
    n = len(As)
    if kw.get("alphas") is not None and len(kw["alphas"]) != n:
        raise ValueError(f"alphas needs {n} entries, got {len(kw['alphas'])}")
    o, keep = _make_opts(opts, trace_len=trace_len * n, **kw)
    if trace_len > 0:
        o.trace_len = trace_len
    held = []
    a = (grbk_csr * n)(*[_csr(M, held) for M in As])
    b = (grbk_csr * n)(*[_csr(M, held) for M in Bs])
    keep.csr = held
    c = _mat_array(Cs)
    h = ctypes.c_void_p()
    st = lib().grbk_sparse_create(ctypes.byref(h), n, a, b, c, ctypes.byref(o))
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_sparse_create")
    return Sparse(h.value, keep, n, trace_len)


def grbk_sparse_solve(sp: Sparse, variant, theta=0.5, tol=0.0, targets=None, maxit=1000, seed=0, X_outs=None):
    """grbk_sparse_solve -> (status, list of result dicts); X_outs written in place."""
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    xo = _mat_array(X_outs, out=True) if X_outs is not None else None
    tg = None
    if targets is not None:
        tgt = np.ascontiguousarray(targets, dtype=np.float64)
        if len(tgt) != sp.nsys:
            raise ValueError(f"targets needs {sp.nsys} entries")
        tg = tgt.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    res = (grbk_result * sp.nsys)()
    st = lib().grbk_sparse_solve(sp.handle, v, float(theta), float(tol), tg, int(maxit), int(seed), xo, res)
    if st not in (GRBK_OK, GRBK_ENOTCONV):
        raise GrbkError(st, "grbk_sparse_solve")
    return st, [r.as_dict() for r in res]


def grbk_sparse_cluster(sp: Sparse) -> int:
    """-> CTAs per system (thread-block cluster size) of the last solve."""
    c = ctypes.c_int32(0)
    st = lib().grbk_sparse_cluster(sp.handle, ctypes.byref(c))
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_sparse_cluster")
    return c.value


def grbk_sparse_info(sp: Sparse, sys: int):
    """-> (entries of A_s A_s^T, step alpha_s)."""
    nnz, al = ctypes.c_int64(), ctypes.c_double()
    st = lib().grbk_sparse_info(sp.handle, int(sys), ctypes.byref(nnz), ctypes.byref(al))
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_sparse_info")
    return nnz.value, al.value


def grbk_sparse_get_residual(sp: Sparse, sys: int, m: int, n: int):
    """-> (R (m x n), row norms (m)) of system `sys` after a solve."""
    R = np.empty((m, n))
    s = np.empty(m)
    st = lib().grbk_sparse_get_residual(sp.handle, int(sys), R.ctypes.data, s.ctypes.data)
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_sparse_get_residual")
    return R, s


def grbk_sparse_destroy(sp: Sparse):
    if sp.handle:
        lib().grbk_sparse_destroy(sp.handle)
        sp.handle = None


# ---------------------------------------------------------------------------
# batch autotuner
# ---------------------------------------------------------------------------
def grbk_tune_variants():
    """-> list of (threads per CTA, rows per warp) of the compiled batched-kernel variants."""
    out = []
    for v in range(lib().grbk_tune_num_variants()):
        t, r = ctypes.c_int32(), ctypes.c_int32()
        lib().grbk_tune_variant_info(v, ctypes.byref(t), ctypes.byref(r))
        out.append((t.value, r.value))
    return out


def grbk_tune_choose(ms):
    a = np.ascontiguousarray(ms, dtype=np.float64)
    return int(lib().grbk_tune_choose(a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(a)))


def grbk_tune_lookup(m, p, q, n, bandA=-1, bandB=-1):
    v = ctypes.c_int32()
    st = lib().grbk_tune_lookup(m, p, q, n, bandA, bandB, ctypes.byref(v))
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_tune_lookup")
    return v.value


def grbk_tune_store(m, p, q, n, bandA, bandB, variant):
    st = lib().grbk_tune_store(m, p, q, n, bandA, bandB, int(variant))
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_tune_store")


def grbk_tune_clear():
    lib().grbk_tune_clear()


def grbk_batch_variant(batch: Batch, sys: int):
    """-> (variant index of system `sys`, seconds the batch's tuning took)."""
    v, t = ctypes.c_int32(), ctypes.c_double()
    st = lib().grbk_batch_variant(batch.handle, int(sys), ctypes.byref(v), ctypes.byref(t))
    if st != GRBK_OK:
        raise GrbkError(st, "grbk_batch_variant")
    return v.value, t.value
