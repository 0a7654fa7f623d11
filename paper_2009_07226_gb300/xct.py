"""ctypes binding of libxct.so.

Each function here has the name of the C entry point it calls (declared in
``include/xct.h``) and only marshals arguments: tensors and arrays become
pointers, torch streams become cudaStream_t handles, status codes become
``XctError``.  All computation happens in the library's CUDA kernels; there
is no fallback: if ``libxct.so`` is missing or does not load, the functions
raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libxct.so")

XCT_OK, XCT_ERR_INVALID, XCT_ERR_OOM, XCT_ERR_CUDA = 0, 1, 2, 3
XCT_ERR_TIMEOUT, XCT_ERR_BREAKDOWN, XCT_ERR_UNSUPPORTED = 4, 5, 6
XCT_F32, XCT_F16, XCT_BF16, XCT_F16A, XCT_BF16A = 0, 1, 2, 3, 4
XCT_PLAN_KEEP_F64, XCT_PLAN_AUTOTUNE, XCT_PLAN_FEW_SLICES, XCT_PLAN_NARROW_TILES = 1, 2, 4, 8
XCT_PLAN_PAIRED_ROWS = 16
XCT_CGLS_X0, XCT_CGLS_NO_GRAPH, XCT_CGLS_TIMING = 1, 2, 4
XCT_CGLS_SAVE, XCT_CGLS_RESUME = 32, 64
XCT_EXPORT_A_F64, XCT_EXPORT_AT_F64, XCT_EXPORT_A_STORED, XCT_EXPORT_AT_STORED = 0, 1, 2, 3
XCT_EXPORT_A_PAIRED, XCT_EXPORT_AT_PAIRED = 4, 5

STORAGE = {"f32": XCT_F32, "f16": XCT_F16, "bf16": XCT_BF16, "f16a": XCT_F16A,
           "bf16a": XCT_BF16A}
_STATUS = {0: "XCT_OK", 1: "XCT_ERR_INVALID", 2: "XCT_ERR_OOM", 3: "XCT_ERR_CUDA",
           4: "XCT_ERR_TIMEOUT", 5: "XCT_ERR_BREAKDOWN", 6: "XCT_ERR_UNSUPPORTED"}


class XctError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class xct_geometry(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_angles", ctypes.c_int32), ("n_det", ctypes.c_int32),
                ("hilbert_tile", ctypes.c_int32), ("cos_sin", ctypes.c_void_p),
                ("det_spacing", ctypes.c_double), ("det_offset", ctypes.c_double),
                ("min_seg", ctypes.c_double)]


class xct_stats(ctypes.Structure):
    _fields_ = [("n_rays", ctypes.c_int64), ("n_pix", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("storage", ctypes.c_int32), ("rows_per_block", ctypes.c_int32),
                ("stage_capacity", ctypes.c_int32), ("stage_capacity_at", ctypes.c_int32),
                ("stages_a", ctypes.c_int64), ("stages_at", ctypes.c_int64),
                ("slots_a", ctypes.c_int64), ("slots_at", ctypes.c_int64),
                ("bytes_a", ctypes.c_int64), ("bytes_at", ctypes.c_int64),
                ("plan_ms", ctypes.c_double), ("t_project_ms", ctypes.c_double),
                ("t_backproject_ms", ctypes.c_double), ("t_other_ms", ctypes.c_double),
                ("n_project", ctypes.c_int64), ("n_backproject", ctypes.c_int64),
                ("t_stage_ms", ctypes.c_double), ("t_vector_ms", ctypes.c_double),
                ("t_scalar_ms", ctypes.c_double), ("slots_a_paired", ctypes.c_int64),
                ("slots_at_paired", ctypes.c_int64), ("gathers_a_paired", ctypes.c_int64),
                ("gathers_at_paired", ctypes.c_int64)]


class xct_job(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("y", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("S", ctypes.c_int32), ("reserved", ctypes.c_int32), ("resid", ctypes.c_void_p)]


XCT_BATCH_AUTOTUNE = 8

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

# (name, restype, argtypes) for every entry point of include/xct.h
_SIGNATURES = [
    ("xct_plan", ctypes.c_int, [ctypes.POINTER(xct_geometry), ctypes.c_int, ctypes.c_uint32,
                                ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    ("xct_free", None, [ctypes.c_void_p]),
    ("xct_project", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_int32, ctypes.c_void_p]),
    ("xct_backproject", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int32, ctypes.c_void_p]),
    ("xct_cgls", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                ctypes.c_int32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]),
    ("xct_tv", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                              ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("xct_adam", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_int32, ctypes.c_void_p]),
    ("xct_tv_reconstruct", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_uint32,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    ("xct_datafit", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                   ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    ("xct_cgls_batch", ctypes.c_int, [ctypes.POINTER(xct_job), ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_uint32, ctypes.c_void_p]),
    ("xct_plan_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(xct_stats)]),
    ("xct_plan_export", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_int64)]),
    ("xct_plan_order", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("xct_project_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int32, ctypes.c_void_p]),
    ("xct_set_allocator", ctypes.c_int, [ALLOC_FN, FREE_FN, ctypes.c_void_p]),
    ("xct_last_error", ctypes.c_char_p, []),
    ("xct_launch_count", ctypes.c_int64, []),
    ("xct_cgls_state_bytes", ctypes.c_int64, [ctypes.c_void_p, ctypes.c_int32]),
    ("xct_project_matfree", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int32, ctypes.c_void_p]),
    ("xct_backproject_matfree", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_int32, ctypes.c_void_p]),
    ("xct_cgls_matfree", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    ("xct_cgls_state", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    ("xct_project_f64", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int32, ctypes.c_void_p]),
    ("xct_backproject_f64", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int32, ctypes.c_void_p]),
    ("xct_cgls_f64", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    ("xct_set_wait_limit", ctypes.c_int, [ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]),
    ("xct_plan_check", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("xct_version", ctypes.c_char_p, []),
    ("xct_roof_probe", ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
]

_lib = None


def lib():
    """Load libxct.so (raises if it is missing: there is no other path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != XCT_OK:
        raise XctError(status, lib().xct_last_error().decode(errors="replace"))


def _ptr(a) -> int | None:
    """Address of a tensor / array / raw integer pointer (None for None)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"cannot pass {type(a)} to libxct")


def _stream(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# --------------------------------------------------------------------------
# the C entry points
# --------------------------------------------------------------------------

def make_geometry(n: int, n_angles: int, n_det: int, cos_sin=None, det_spacing: float = 1.0,
                  det_offset: float = 0.0, min_seg: float = 1e-9, hilbert_tile: int = 0):
    """An xct_geometry; the angle table (if any) is kept alive on the struct."""
    g = xct_geometry(n, n_angles, n_det, hilbert_tile, None, det_spacing, det_offset, min_seg)
    if cos_sin is not None:
        cs = np.ascontiguousarray(cos_sin, dtype=np.float64).reshape(n_angles, 2)
        g._cs = cs
        g.cos_sin = cs.ctypes.data
    return g


def xct_plan(geometry: xct_geometry, storage, flags: int = 0, stream=None) -> int:
    st = STORAGE[storage] if isinstance(storage, str) else int(storage)
    out = ctypes.c_void_p()
    _check(lib().xct_plan(ctypes.byref(geometry), st, flags, _stream(stream), ctypes.byref(out)))
    return out.value


def xct_free(plan: int) -> None:
    lib().xct_free(plan)


def xct_project(plan: int, x, y, S: int, stream=None) -> None:
    _check(lib().xct_project(plan, _ptr(x), _ptr(y), S, _stream(stream)))


def xct_project_noalloc(plan: int, x, y, S: int, stream=None) -> None:
    """y = A x without allocating: working memory is the library's fixed
    32 MiB device array (device pointers only; overlapping calls race)."""
    _check(lib().xct_project_noalloc(plan, _ptr(x), _ptr(y), S, _stream(stream)))


def xct_backproject(plan: int, y, x, S: int, stream=None) -> None:
    _check(lib().xct_backproject(plan, _ptr(y), _ptr(x), S, _stream(stream)))


def xct_cgls(plan: int, y, x, S: int, iters: int, flags: int = 0, resid=None, stream=None) -> None:
    _check(lib().xct_cgls(plan, _ptr(y), _ptr(x), S, iters, flags, _ptr(resid), _stream(stream)))


def xct_project_matfree(plan: int, x, y, S: int, stream=None) -> None:
    _check(lib().xct_project_matfree(plan, _ptr(x), _ptr(y), S, _stream(stream)))


def xct_project_f64(plan: int, x, y, S: int, stream=None) -> None:
    _check(lib().xct_project_f64(plan, _ptr(x), _ptr(y), S, _stream(stream)))


def xct_backproject_f64(plan: int, y, x, S: int, stream=None) -> None:
    _check(lib().xct_backproject_f64(plan, _ptr(y), _ptr(x), S, _stream(stream)))


def xct_cgls_f64(plan: int, y, x, S: int, iters: int, flags: int = 0, resid=None,
                 stream=None) -> None:
    _check(lib().xct_cgls_f64(plan, _ptr(y), _ptr(x), S, iters, flags, _ptr(resid),
                              _stream(stream)))


def xct_backproject_matfree(plan: int, y, x, S: int, stream=None) -> None:
    _check(lib().xct_backproject_matfree(plan, _ptr(y), _ptr(x), S, _stream(stream)))


def xct_cgls_matfree(plan: int, y, x, S: int, iters: int, flags: int = 0, resid=None,
                     stream=None) -> None:
    _check(lib().xct_cgls_matfree(plan, _ptr(y), _ptr(x), S, iters, flags, _ptr(resid),
                                  _stream(stream)))


def xct_cgls_state_bytes(plan: int, S: int) -> int:
    return lib().xct_cgls_state_bytes(plan, S)


def xct_cgls_state(plan: int, y, x, S: int, iters: int, flags: int, state, resid=None,
                   stream=None) -> None:
    """CGLS with a checkpoint (flags include XCT_CGLS_SAVE and/or
    XCT_CGLS_RESUME); state: uint8 buffer of xct_cgls_state_bytes bytes."""
    _check(lib().xct_cgls_state(plan, _ptr(y), _ptr(x), S, iters, flags, _ptr(resid), _ptr(state),
                                _stream(stream)))


def xct_tv(x, n: int, S: int, eps: float, weight: float, grad=None, value=None, stream=None) -> None:
    _check(lib().xct_tv(_ptr(x), n, S, eps, weight, _ptr(grad), _ptr(value), _stream(stream)))


def xct_adam(x, g, m, v, count: int, lr: float, beta1: float, beta2: float, eps: float, step: int,
             stream=None) -> None:
    _check(lib().xct_adam(_ptr(x), _ptr(g), _ptr(m), _ptr(v), count, lr, beta1, beta2, eps, step,
                          _stream(stream)))


def xct_datafit(q, y, r, length: int, S: int, value=None, stream=None) -> None:
    _check(lib().xct_datafit(_ptr(q), _ptr(y), _ptr(r), length, S, _ptr(value), _stream(stream)))


def xct_tv_reconstruct(plan: int, y, x, S: int, steps: int, lr: float, lam: float, eps: float,
                       flags: int = 0, loss=None, stream=None) -> None:
    _check(lib().xct_tv_reconstruct(plan, _ptr(y), _ptr(x), S, steps, lr, lam, eps, flags,
                                    _ptr(loss), _stream(stream)))


def xct_cgls_batch(jobs, iters: int, flags: int = 0, stream=None) -> None:
    """jobs: sequence of (plan handle, y, x, S[, resid]) with device buffers."""
    arr = (xct_job * max(len(jobs), 1))()
    for i, jb in enumerate(jobs):
        plan, y, x, S = jb[:4]
        resid = jb[4] if len(jb) > 4 else None
        arr[i] = xct_job(plan, _ptr(y), _ptr(x), S, 0, _ptr(resid))
    _check(lib().xct_cgls_batch(arr, len(jobs), iters, flags, _stream(stream)))


def xct_plan_stats(plan: int) -> dict:
    s = xct_stats()
    _check(lib().xct_plan_stats(plan, ctypes.byref(s)))
    return {name: getattr(s, name) for name, _ in xct_stats._fields_}


def xct_plan_export(plan: int, what: int):
    """(rowptr int64, col int32, val float64) host arrays, natural order."""
    nnz = ctypes.c_int64()
    _check(lib().xct_plan_export(plan, what, None, None, None, ctypes.byref(nnz)))
    st = xct_plan_stats(plan)
    nrows = st["n_pix"] if what in (XCT_EXPORT_AT_F64, XCT_EXPORT_AT_STORED, XCT_EXPORT_AT_PAIRED) else st["n_rays"]
    rowptr = np.zeros(nrows + 1, dtype=np.int64)
    col = np.zeros(max(nnz.value, 1), dtype=np.int32)
    val = np.zeros(max(nnz.value, 1), dtype=np.float64)
    _check(lib().xct_plan_export(plan, what, rowptr.ctypes.data, col.ctypes.data, val.ctypes.data,
                                 ctypes.byref(nnz)))
    return rowptr, col[:nnz.value], val[:nnz.value]


def xct_plan_order(plan: int):
    st = xct_plan_stats(plan)
    pix = np.zeros(st["n_pix"], dtype=np.int32)
    ray = np.zeros(st["n_rays"], dtype=np.int32)
    _check(lib().xct_plan_order(plan, pix.ctypes.data, ray.ctypes.data))
    return pix, ray


_hooks = []


def xct_set_allocator(alloc, release, ctx=None) -> None:
    """alloc(bytes, stream) -> int pointer (0 on failure); release(ptr,
    bytes, stream).  None, None restores the library default."""
    if alloc is None and release is None:
        _check(lib().xct_set_allocator(ALLOC_FN(), FREE_FN(), None))
        _hooks.clear()
        return

    def _a(nbytes, stream, _ctx):
        try:
            return alloc(nbytes, stream) or None
        except Exception:
            return None

    def _f(ptr, nbytes, stream, _ctx):
        try:
            release(ptr, nbytes, stream)
        except Exception:
            pass

    fa, ff = ALLOC_FN(_a), FREE_FN(_f)
    _hooks[:] = [fa, ff]
    _check(lib().xct_set_allocator(fa, ff, ctx))


def xct_last_error() -> str:
    return lib().xct_last_error().decode(errors="replace")


def xct_launch_count() -> int:
    return lib().xct_launch_count()


def xct_set_wait_limit(ns: int) -> int:
    """Set the limit of the waits inside the persistent kernels; returns the
    previous limit (nanoseconds)."""
    prev = ctypes.c_uint64()
    _check(lib().xct_set_wait_limit(ns, ctypes.byref(prev)))
    return prev.value


def xct_plan_check(plan: int, stream=None) -> None:
    """Raise XctError(XCT_ERR_TIMEOUT) if a product of this plan gave up a
    wait since the last check."""
    _check(lib().xct_plan_check(plan, _stream(stream)))


def xct_roof_probe(kind: int, iters: int, ctas_per_sm: int = 2, stream=None) -> float:
    """Launch the roof probe (asynchronous); returns its operation count."""
    ops = ctypes.c_double()
    _check(lib().xct_roof_probe(kind, iters, ctas_per_sm, ctypes.byref(ops), _stream(stream)))
    return ops.value


def xct_version() -> str:
    return lib().xct_version().decode()


def use_torch_allocator() -> None:
    """Route the library's device allocations through PyTorch's caching
    allocator (stream-ordered on the stream the library passes)."""
    import torch

    def _alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                  stream if stream else 0)

    def _free(ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(ptr)

    xct_set_allocator(_alloc, _free)


# --------------------------------------------------------------------------
# convenience: a plan object over torch tensors
# --------------------------------------------------------------------------

class Plan:
    """Owns one xct plan; methods call the entry points above on tensors."""

    def __init__(self, n: int, n_angles: int, n_det: int | None = None, storage: str = "f32",
                 cos_sin=None, det_spacing: float = 1.0, det_offset: float = 0.0,
                 min_seg: float = 1e-9, hilbert_tile: int = 0, keep_f64: bool = False,
                 autotune: bool = False, few_slices: bool = False, narrow_tiles: bool = False,
                 paired_rows: bool = False, stream=None):
        self.n, self.m = n, n_angles
        self.nd = n if n_det is None else n_det
        self.storage = storage
        self.geometry = make_geometry(n, n_angles, self.nd, cos_sin, det_spacing, det_offset,
                                      min_seg, hilbert_tile)
        flags = ((XCT_PLAN_KEEP_F64 if keep_f64 else 0) | (XCT_PLAN_AUTOTUNE if autotune else 0)
                 | (XCT_PLAN_FEW_SLICES if few_slices else 0) | (XCT_PLAN_NARROW_TILES if narrow_tiles else 0)
                 | (XCT_PLAN_PAIRED_ROWS if paired_rows else 0))
        self.handle = xct_plan(self.geometry, storage, flags, stream)

    def close(self):
        if getattr(self, "handle", None):
            xct_free(self.handle)
            self.handle = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def npix(self):
        return self.n * self.n

    @property
    def nrays(self):
        return self.m * self.nd

    def stats(self) -> dict:
        return xct_plan_stats(self.handle)

    def project(self, x, out=None, stream=None):
        """y = A x; x [S, n, n] float32 -> y [S, M, N_d]."""
        import torch
        S = x.shape[0]
        y = out if out is not None else torch.empty((S, self.m, self.nd), dtype=torch.float32,
                                                    device=x.device)
        xct_project(self.handle, x, y, S, stream)
        return y

    def backproject(self, y, out=None, stream=None):
        """x = A^T y; y [S, M, N_d] float32 -> x [S, n, n]."""
        import torch
        S = y.shape[0]
        x = out if out is not None else torch.empty((S, self.n, self.n), dtype=torch.float32,
                                                    device=y.device)
        xct_backproject(self.handle, y, x, S, stream)
        return x

    def project_f64(self, x, out=None, stream=None):
        """y = A x in FP64 (plan built with keep_f64); x [S, n, n] float64."""
        import torch
        S = x.shape[0]
        y = out if out is not None else torch.empty((S, self.m, self.nd), dtype=torch.float64,
                                                    device=x.device)
        xct_project_f64(self.handle, x, y, S, stream)
        return y

    def backproject_f64(self, y, out=None, stream=None):
        """x = A^T y in FP64 (plan built with keep_f64); y [S, M, N_d] float64."""
        import torch
        S = y.shape[0]
        x = out if out is not None else torch.empty((S, self.n, self.n), dtype=torch.float64,
                                                    device=y.device)
        xct_backproject_f64(self.handle, y, x, S, stream)
        return x

    def cgls_f64(self, y, iters: int, x0=None, resid: bool = False, stream=None):
        """FP64 CGLS (plan built with keep_f64); y [S, M, N_d] float64."""
        import torch
        S = y.shape[0]
        flags = 0
        if x0 is not None:
            x = x0.clone()
            flags |= XCT_CGLS_X0
        else:
            x = torch.empty((S, self.n, self.n), dtype=torch.float64, device=y.device)
        log = torch.zeros((iters + 1, S, 2), dtype=torch.float64, device=y.device) if resid else None
        xct_cgls_f64(self.handle, y, x, S, iters, flags, log, stream)
        return (x, log) if resid else x

    def cgls(self, y, iters: int, x0=None, resid: bool = False, flags: int = 0, stream=None):
        """CGLS from x0 (or 0); returns x [S, n, n] (and the residual log
        [iters+1, S, 2] as float64 when resid=True)."""
        import torch
        S = y.shape[0]
        if x0 is not None:
            x = x0.clone()
            flags |= XCT_CGLS_X0
        else:
            x = torch.empty((S, self.n, self.n), dtype=torch.float32, device=y.device)
        log = torch.zeros((iters + 1, S, 2), dtype=torch.float64, device=y.device) if resid else None
        xct_cgls(self.handle, y, x, S, iters, flags, log, stream)
        return (x, log) if resid else x
