"""Python binding of the GB300 multi-trait GWAS library (``include/gwas.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library ``libgwas_gb300.so`` built in-tree by :mod:`.build`.  The first call
into the library fails loudly when it has not been built; there is no CPU
fallback.

Array arguments may be numpy arrays (host memory) or torch tensors (host or
CUDA); their dtype, shape and contiguity are checked here and their addresses
are passed to the C functions, which tell host from device memory themselves.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgwas_gb300.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "gwas.h")


def _status_codes():
    codes = {}
    with open(HEADER) as f:
        for line in f:
            mt = re.match(r"#define (GWAS_[A-Z0-9_]+)\s+(\d+)", line)
            if mt:
                codes[mt.group(1)] = int(mt.group(2))
    return codes


_CODES = _status_codes()
globals().update(_CODES)
_NAMES = {v: k for k, v in _CODES.items() if k.startswith("GWAS_ERR") or k == "GWAS_OK"}


class GwasError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class gwas_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("output", C.c_int), ("trait_block", C.c_int), ("device", C.c_int),
                ("profile", C.c_int), ("hbm_budget", C.c_size_t), ("stream", C.c_void_p),
                ("tune_cache", C.c_char_p)]


# void (*)(void* user, int j0, int nb, const void* host_block)
GWAS_BLOCK_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_int, C.c_int, C.c_void_p)
GWAS_SLAB_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_int64, C.c_int64, C.c_int, C.c_int, C.c_void_p)


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1210_7683_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i64, ci = C.c_void_p, C.c_int64, C.c_int
    lib.gwas_default_opts.argtypes = [C.POINTER(gwas_opts)]
    lib.gwas_default_opts.restype = None
    lib.gwas_setup.argtypes = [C.POINTER(vp), ci, ci, vp, vp, ci, vp, C.POINTER(gwas_opts)]
    lib.gwas_setup.restype = ci
    lib.gwas_load_snps.argtypes = [vp, i64, vp]
    lib.gwas_load_snps.restype = ci
    lib.gwas_solve.argtypes = [vp, vp, i64, i64, vp]
    lib.gwas_solve.restype = ci
    lib.gwas_autotune.argtypes = [vp, vp, ci, i64, C.POINTER(C.c_double)]
    lib.gwas_autotune.restype = ci
    lib.gwas_tune_shape.argtypes = [vp, C.POINTER(C.c_int)]
    lib.gwas_tune_shape.restype = ci
    lib.gwas_serve_stats.argtypes = [vp, C.POINTER(i64), C.POINTER(i64)]
    lib.gwas_serve_stats.restype = ci
    lib.gwas_set_h2.argtypes = [vp, ci, vp]
    lib.gwas_set_h2.restype = ci
    lib.gwas_singular_count.argtypes = [vp]
    lib.gwas_singular_count.restype = i64
    lib.gwas_kernel_launches.argtypes = [vp]
    lib.gwas_kernel_launches.restype = i64
    lib.gwas_last_error.argtypes = [vp]
    lib.gwas_last_error.restype = C.c_char_p
    lib.gwas_kernel_time.argtypes = [vp, C.c_char_p, C.POINTER(C.c_double), C.POINTER(i64)]
    lib.gwas_kernel_time.restype = ci
    lib.gwas_reset_timers.argtypes = [vp]
    lib.gwas_reset_timers.restype = None
    lib.gwas_solve_fp64_noalloc.argtypes = [ci, ci, vp, vp, vp, i64, vp, vp, ci, ci, vp, vp, C.POINTER(i64)]
    lib.gwas_solve_fp64_noalloc.restype = ci
    lib.gwas_solve_stream.argtypes = [vp, vp, i64, i64, ci, vp, vp, GWAS_BLOCK_FN, vp]
    lib.gwas_solve_stream.restype = ci
    lib.gwas_solve_ooc.argtypes = [vp, i64, vp, i64, vp, ci, vp, vp, GWAS_SLAB_FN, vp]
    lib.gwas_solve_ooc.restype = ci
    lib.gwas_submit.argtypes = [vp, vp, ci, vp, i64, i64, vp, C.POINTER(C.c_uint64)]
    lib.gwas_submit.restype = ci
    lib.gwas_poll.argtypes = [vp, C.c_uint64, C.POINTER(ci)]
    lib.gwas_poll.restype = ci
    lib.gwas_wait.argtypes = [vp, C.c_uint64, C.c_double]
    lib.gwas_wait.restype = ci
    lib.gwas_request_times.argtypes = [vp, C.c_uint64, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                       C.POINTER(C.c_double)]
    lib.gwas_request_times.restype = ci
    lib.gwas_sbr_info.argtypes = [vp, C.POINTER(ci), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                  C.POINTER(C.c_double)]
    lib.gwas_sbr_info.restype = ci
    lib.gwas_cheb_plan.argtypes = [ci, vp, vp, C.c_double, C.c_double, C.c_double, C.POINTER(ci),
                                   C.POINTER(C.c_double)]
    lib.gwas_cheb_plan.restype = ci
    lib.gwas_check_bounded_wait.argtypes = [ci, C.c_double, C.POINTER(C.c_double)]
    lib.gwas_check_epilogue_math.argtypes = [ci, vp, ci, vp]
    lib.gwas_check_epilogue_math.restype = ci
    lib.gwas_check_bounded_wait.restype = ci
    lib.gwas_destroy.argtypes = [vp]
    lib.gwas_destroy.restype = None
    lib.gwas_eig_info.argtypes = [vp, C.POINTER(ci)]
    lib.gwas_eig_info.restype = ci
    lib.gwas_fp4_info.argtypes = [vp, C.POINTER(ci), C.POINTER(C.c_int64)]
    lib.gwas_fp4_info.restype = ci
    lib.gwas_pool_info.argtypes = [ci, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
    lib.gwas_pool_info.restype = ci
    lib.gwas_pool_trim.argtypes = [ci, C.c_uint64]
    lib.gwas_pool_trim.restype = ci
    return lib


_lib = None


class _LazyLib:
    """Loads the CUDA library on first use and raises if it has not been built."""

    def __getattr__(self, name):
        global _lib
        if _lib is None:
            _lib = _load()
        return getattr(_lib, name)


lib = _LazyLib()


def _addr(x, dtype, shape=None, name="array"):
    """Address of a C-contiguous numpy array or torch tensor of the given dtype."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != np.dtype(dtype):
            raise TypeError(f"{name}: dtype {x.dtype}, expected {np.dtype(dtype)}")
        if not x.flags.c_contiguous:
            raise ValueError(f"{name} must be C-contiguous")
        if shape is not None and tuple(x.shape) != tuple(shape):
            raise ValueError(f"{name}: shape {x.shape}, expected {tuple(shape)}")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):  # torch tensor
        import torch
        tmap = {np.float64: torch.float64, np.float32: torch.float32, np.int8: torch.int8}
        if x.dtype != tmap[np.dtype(dtype).type]:
            raise TypeError(f"{name}: dtype {x.dtype}, expected {dtype}")
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if shape is not None and tuple(x.shape) != tuple(shape):
            raise ValueError(f"{name}: shape {tuple(x.shape)}, expected {tuple(shape)}")
        return x.data_ptr()
    raise TypeError(f"{name}: expected a numpy array or a torch tensor")


# context address -> (n, p, t, output mode): the sizes the binding checks arrays against.  The
# C calls take bare pointers and trust the caller for sizes; from Python the array sizes are
# known, so an array too small for what a call reads or writes is refused before the call.
_CTX = {}


def _key(ctx):
    return getattr(ctx, "value", ctx)


def _nbytes(x):
    if isinstance(x, np.ndarray):
        return x.nbytes
    if hasattr(x, "data_ptr"):
        return x.numel() * x.element_size()
    return None


def _need(x, nbytes, name):
    have = _nbytes(x)
    if have is not None and have < nbytes:
        raise ValueError(f"{name}: {have} bytes, the call needs {nbytes}")


def _out_pair_bytes(p, output):
    return 8 if output == GWAS_OUT_LAST_SE else 8 * p


def _check(rc: int, ctx=None, allow=()):
    if rc != GWAS_OK and rc not in allow:
        raise GwasError(rc, lib.gwas_last_error(ctx).decode())
    return rc


def gwas_default_opts(**kw) -> gwas_opts:
    o = gwas_opts()
    lib.gwas_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "tune_cache" and isinstance(v, str):
            v = v.encode()
        setattr(o, k, v)
    return o


def gwas_autotune(ctx, Y, t_sample=0, m_sample=0) -> float:
    """Choose the fused-kernel launch shape by timing candidates on a sample (see
    include/gwas.h); returns the sample's solve time in ms with the chosen shape."""
    best = C.c_double()
    _check(lib.gwas_autotune(ctx, _addr(Y, np.float64, None, "Y"), int(t_sample), int(m_sample), C.byref(best)), ctx)
    return best.value


def gwas_serve_stats(ctx):
    """(rounds, rounds replayed from the captured CUDA graph) of the serving loop."""
    r, gr = C.c_int64(), C.c_int64()
    _check(lib.gwas_serve_stats(ctx, C.byref(r), C.byref(gr)), ctx)
    return r.value, gr.value


def gwas_tune_shape(ctx) -> dict:
    """The context's launch shape: cluster CTAs along SNPs and traits, epilogue warps,
    CTA-pair mode, SNP tiles per traversal group."""
    v = (C.c_int * 5)()
    _check(lib.gwas_tune_shape(ctx, v), ctx)
    return dict(zip(("cs", "ct", "epw", "pair", "group"), list(v)))


def gwas_setup(n, pm1, phi, XL, t, h2, opts: gwas_opts | None = None):
    """Create a context (see include/gwas.h).  phi: (n, n); XL: (p-1, n); h2: (t,)."""
    ctx = C.c_void_p()
    rc = lib.gwas_setup(C.byref(ctx), n, pm1, _addr(phi, np.float64, (n, n), "phi"),
                        _addr(XL, np.float64, (pm1, n), "XL") if pm1 > 0 else None, t,
                        _addr(h2, np.float64, (t,), "h2"), C.byref(opts) if opts is not None else None)
    _check(rc, None)
    _CTX[_key(ctx)] = (int(n), int(pm1) + 1, int(t), opts.output if opts is not None else GWAS_OUT_LAST_SE)
    return ctx


def gwas_load_snps(ctx, m, XR, n=None):
    """XR: (m, n) int8, SNP-major."""
    shape = None if n is None else (m, n)
    info = _CTX.get(_key(ctx))
    if info is not None:
        _need(XR, int(m) * info[0], "XR")
    return _check(lib.gwas_load_snps(ctx, m, _addr(XR, np.int8, shape, "XR")), ctx)


def gwas_solve(ctx, Y, i0, i1, out):
    """Y: (t, n) float64; out: FULL_B (t, i1-i0, p) float64 or LAST_SE (2, t, i1-i0) float32.

    Returns GWAS_OK or GWAS_ERR_SINGULAR_PAIRS (a warning); raises on errors.
    """
    info = _CTX.get(_key(ctx))
    if info is not None:
        n, p, t, output = info
        _need(Y, 8 * t * n, "Y")
        _need(out, _out_pair_bytes(p, output) * t * max(int(i1) - int(i0), 0), "out")
    yv = _addr(Y, np.float64, None, "Y")
    dt = np.float64 if getattr(out, "dtype", None) in (np.float64, getattr(_torch(), "float64", None)) else np.float32
    return _check(lib.gwas_solve(ctx, yv, int(i0), int(i1), _addr(out, dt, None, "out")), ctx,
                  allow=(GWAS_ERR_SINGULAR_PAIRS,))


def gwas_solve_stream(ctx, Y, i0, i1, block_traits, buf0, buf1, fn):
    """Blocked solve into two host buffers; fn(j0, nb, address) is called per finished block.

    buf0/buf1: host numpy arrays or (pinned) torch tensors large enough for one block
    (see include/gwas.h).  Returns GWAS_OK or GWAS_ERR_SINGULAR_PAIRS; raises otherwise.
    """
    cb = GWAS_BLOCK_FN(lambda user, j0, nb, ptr: fn(j0, nb, ptr))
    dt = np.float64 if getattr(buf0, "dtype", None) in (np.float64, getattr(_torch(), "float64", None)) else np.float32
    rc = lib.gwas_solve_stream(ctx, _addr(Y, np.float64, None, "Y"), int(i0), int(i1), int(block_traits),
                               _addr(buf0, dt, None, "buf0"), _addr(buf1, dt, None, "buf1"), cb, None)
    return _check(rc, ctx, allow=(GWAS_ERR_SINGULAR_PAIRS,))


def gwas_solve_ooc(ctx, m, XR, slab, Y, block_traits, buf0, buf1, fn, n=None):
    """Out-of-core solve: XR (m, n) int8 SNP-major in host (or device) memory is streamed in
    slabs of `slab` SNPs; fn(i0, i1, j0, nb, address) is called per finished piece of SNPs
    [i0, i1) x traits [j0, j0+nb), the piece in gwas_solve's layout at `address` (one of the
    two host buffers).  Returns GWAS_OK or GWAS_ERR_SINGULAR_PAIRS; raises otherwise.
    """
    cb = GWAS_SLAB_FN(lambda user, i0, i1, j0, nb, ptr: fn(i0, i1, j0, nb, ptr))
    dt = np.float64 if getattr(buf0, "dtype", None) in (np.float64, getattr(_torch(), "float64", None)) else np.float32
    shape = None if n is None else (m, n)
    rc = lib.gwas_solve_ooc(ctx, int(m), _addr(XR, np.int8, shape, "XR"), int(slab), _addr(Y, np.float64, None, "Y"),
                            int(block_traits), _addr(buf0, dt, None, "buf0"), _addr(buf1, dt, None, "buf1"), cb, None)
    return _check(rc, ctx, allow=(GWAS_ERR_SINGULAR_PAIRS,))


def gwas_submit(ctx, Y, tk, h2k, i0, i1, out) -> int:
    """Queue a serving request (see include/gwas.h); returns its id."""
    rid = C.c_uint64()
    info = _CTX.get(_key(ctx))
    if info is not None:
        n, p, _, output = info
        _need(Y, 8 * int(tk) * n, "Y")
        _need(out, _out_pair_bytes(p, output) * int(tk) * max(int(i1) - int(i0), 0), "out")
    dt = np.float64 if getattr(out, "dtype", None) in (np.float64, getattr(_torch(), "float64", None)) else np.float32
    _check(lib.gwas_submit(ctx, _addr(Y, np.float64, None, "Y"), int(tk), _addr(h2k, np.float64, (tk,), "h2k"),
                           int(i0), int(i1), _addr(out, dt, None, "out"), C.byref(rid)), ctx)
    return rid.value


def gwas_poll(ctx, req_id):
    """(done, status) of a serving request."""
    done = C.c_int()
    rc = lib.gwas_poll(ctx, req_id, C.byref(done))
    return bool(done.value), rc


def gwas_wait(ctx, req_id, timeout_s=-1.0) -> int:
    return _check(lib.gwas_wait(ctx, req_id, float(timeout_s)), ctx, allow=(GWAS_ERR_SINGULAR_PAIRS,))


def gwas_request_times(ctx, req_id):
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    _check(lib.gwas_request_times(ctx, req_id, C.byref(a), C.byref(b), C.byref(c)), ctx)
    return a.value, b.value, c.value


def gwas_set_h2(ctx, t, h2):
    return _check(lib.gwas_set_h2(ctx, t, _addr(h2, np.float64, (t,), "h2")), ctx)


def gwas_singular_count(ctx) -> int:
    return lib.gwas_singular_count(ctx)


def gwas_kernel_launches(ctx) -> int:
    return lib.gwas_kernel_launches(ctx)


def gwas_kernel_time(ctx, kernel: str):
    """(milliseconds, launches) of one kernel family (profiling contexts only)."""
    ms, n = C.c_double(), C.c_int64()
    _check(lib.gwas_kernel_time(ctx, kernel.encode(), C.byref(ms), C.byref(n)), ctx)
    return ms.value, n.value


def gwas_reset_timers(ctx) -> None:
    lib.gwas_reset_timers(ctx)


def gwas_solve_fp64_noalloc(n, pm1, lam, XLt, Xt, m, Yt, h2, t, output, out, stream=None):
    """Allocation-free FP64 solve on rotated inputs (see include/gwas.h).

    Returns (status, singular_pairs); raises GwasError on failures other than
    the singular-pairs warning.
    """
    for name, a in (("lam", lam), ("XLt", XLt), ("Xt", Xt), ("Yt", Yt), ("h2", h2), ("out", out)):
        if a is None and name == "XLt" and pm1 == 0:
            continue
        if not (hasattr(a, "data_ptr") and getattr(a, "is_cuda", False)):
            raise TypeError(f"{name}: gwas_solve_fp64_noalloc takes CUDA tensors only (device memory)")
    p = int(pm1) + 1
    _need(out, (8 * p if output == GWAS_OUT_FULL_B else 8) * int(t) * int(m), "out")
    sing = C.c_int64(0)
    dt = np.float64 if output == GWAS_OUT_FULL_B else np.float32
    rc = lib.gwas_solve_fp64_noalloc(n, pm1, _addr(lam, np.float64, (n,), "lam"),
                                     _addr(XLt, np.float64, (pm1, n), "XLt") if pm1 > 0 else None,
                                     _addr(Xt, np.float64, (m, n), "Xt"), m, _addr(Yt, np.float64, (t, n), "Yt"),
                                     _addr(h2, np.float64, (t,), "h2"), t, output, _addr(out, dt, None, "out"),
                                     stream, C.byref(sing))
    if rc not in (GWAS_OK, GWAS_ERR_SINGULAR_PAIRS):
        raise GwasError(rc, "gwas_solve_fp64_noalloc failed")
    return rc, sing.value


def gwas_sbr_info(ctx) -> dict:
    """How the mixed path obtains S_BR (see include/gwas.h): terms R (0: contracted per pair),
    the interpolation interval and the relative error bound."""
    r, lo, hi, b = C.c_int(), C.c_double(), C.c_double(), C.c_double()
    _check(lib.gwas_sbr_info(ctx, C.byref(r), C.byref(lo), C.byref(hi), C.byref(b)), ctx)
    return {"terms": r.value, "lo": lo.value, "hi": hi.value, "bound": b.value}


def gwas_cheb_plan(lam, reach, lo, hi, tol=1e-10):
    """(R, bound) of the S_BR interpolation plan for eigenvalues lam (float64) and the mask reach."""
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    reach = np.ascontiguousarray(reach, dtype=np.uint8)
    if reach.shape != lam.shape:
        raise ValueError("lam and reach differ in length")
    r, b = C.c_int(), C.c_double()
    rc = lib.gwas_cheb_plan(lam.size, lam.ctypes.data, reach.ctypes.data, float(lo), float(hi), float(tol),
                            C.byref(r), C.byref(b))
    if rc != GWAS_OK:
        raise GwasError(rc, "gwas_cheb_plan: invalid arguments")
    return r.value, b.value


def gwas_check_epilogue_math(x, device=0):
    """The epilogue's reciprocal and square root of x (float32 values) and CUDA's correctly rounded
    ones, as an array [count][4]: rcp, rcp_rn, sqrt, sqrt_rn."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty((x.size, 4), np.float32)
    rc = lib.gwas_check_epilogue_math(int(device), x.ctypes.data, int(x.size), out.ctypes.data)
    if rc != GWAS_OK:
        raise GwasError(rc, "gwas_check_epilogue_math failed")
    return out


def gwas_check_bounded_wait(device=0, limit_s=0.05):
    """(status, waited seconds) of the bounded-wait self-test (expected: GWAS_ERR_TIMEOUT)."""
    w = C.c_double()
    rc = lib.gwas_check_bounded_wait(int(device), float(limit_s), C.byref(w))
    return rc, w.value


def gwas_last_error(ctx=None) -> str:
    return lib.gwas_last_error(ctx).decode()


def gwas_destroy(ctx) -> None:
    _CTX.pop(_key(ctx), None)
    lib.gwas_destroy(ctx)


def gwas_eig_info(ctx) -> int:
    """Refinement steps of the context's eigendecomposition (-1: computed by the FP64 solver)."""
    st = C.c_int()
    _check(lib.gwas_eig_info(ctx, C.byref(st)), ctx)
    return st.value


def gwas_fp4_info(ctx) -> dict:
    """Whether the loaded genotypes have their e2m1 copy, and the launches of the fused kernel on
    e2m1 operands so far."""
    ready, launches = C.c_int(), C.c_int64()
    _check(lib.gwas_fp4_info(ctx, C.byref(ready), C.byref(launches)), ctx)
    return {"ready": bool(ready.value), "launches": launches.value}


def gwas_pool_info(device=0) -> dict:
    """Bytes the library's device memory pool holds from the device and bytes in live buffers."""
    r, u = C.c_uint64(), C.c_uint64()
    rc = lib.gwas_pool_info(int(device), C.byref(r), C.byref(u))
    if rc != GWAS_OK:
        raise GwasError(rc, "gwas_pool_info failed")
    return {"reserved": r.value, "used": u.value}


def gwas_pool_trim(device=0, keep_bytes=0) -> None:
    """Give the pool's unused device memory back until at most keep_bytes stay reserved."""
    rc = lib.gwas_pool_trim(int(device), int(keep_bytes))
    if rc != GWAS_OK:
        raise GwasError(rc, "gwas_pool_trim failed")


def _torch():
    try:
        import torch
        return torch
    except ImportError:  # pragma: no cover
        return None
