"""Thin ctypes binding of the C ABI in include/pr.h (argument marshalling only).

Every function keeps the C name.  Arrays are torch tensors on the context's
CUDA device; the binding checks their device, dtype, contiguity and size,
passes data_ptr() and the current CUDA stream, and raises PrError on a
non-zero status.  All computation happens in the CUDA library; if it cannot be
loaded the import fails loudly (there is no fallback).
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
LIB_PATH = os.path.join(PKG, "_lib", "libpr.so")
HEADER = os.path.join(ROOT, "include", "pr.h")

PR_F32, PR_F64 = 0, 1
PR_CORR_PROCRUSTES, PR_CORR_OMEGA1, PR_CORR_PLAIN = 0, 1, 2
STATUS = {0: "PR_OK", 1: "PR_EINVAL", 2: "PR_ENOMEM", 3: "PR_ECUDA", 4: "PR_ETIMEOUT",
          5: "PR_EUNSTABLE", 6: "PR_ENOTCONV"}


class PrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class pr_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nf", ctypes.c_int64 * 3), ("ratio", ctypes.c_int)]


class pr_options(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("grad_order", ctypes.c_int), ("interp", ctypes.c_int),
                ("tol", ctypes.c_double), ("block_depth", ctypes.c_int), ("max_iters", ctypes.c_int)]


_P = ctypes.c_void_p
# pr_set_allocator's callbacks: alloc(bytes, device, user) -> pointer, release(ptr, user)
_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p)
_RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_SIGNATURES = {
    "pr_set_allocator": (ctypes.c_int, [_ALLOC_FN, _RELEASE_FN, _P]),
    "pr_create": (ctypes.c_int, [ctypes.POINTER(pr_grid), _P, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int, ctypes.c_double, ctypes.POINTER(pr_options),
                                 ctypes.POINTER(_P)]),
    "pr_destroy": (None, [_P]),
    "pr_last_error": (ctypes.c_char_p, [_P]),
    "pr_fine_all_slices": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int, ctypes.c_int, _P]),
    "pr_check": (ctypes.c_int, [_P, _P]),
    "pr_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int)]),
    "pr_energy": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_double), _P]),
    "pr_fine_all_slices_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, ctypes.c_int, _P,
                                                  ctypes.c_double, ctypes.c_int, _P, _P, _P, _P,
                                                  _P, ctypes.c_char_p, ctypes.c_size_t]),
    "pr_coarse_sweep": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int, ctypes.c_int, _P]),
    "pr_iterate": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_double, _P, _P,
                                  _P, _P, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_int), _P]),
    "pr_iterate_phases": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "pr_procrustes_correct": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
    "pr_procrustes_apply": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_int), _P]),
    "pr_procrustes_reset": (ctypes.c_int, [_P]),
    "pr_adjoint": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "pr_batch_create": (ctypes.c_int, [ctypes.c_int, _P, _P, _P, _P, _P, ctypes.c_int, _P,
                                       ctypes.POINTER(_P)]),
    "pr_batch_launch": (ctypes.c_int, [_P, _P]),
    "pr_batch_info": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "pr_set_fused_columns": (ctypes.c_int, [_P, ctypes.c_int]),
    "pr_batch_destroy": (None, [_P]),
    "pr_batch_set_mode": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_int)]),
    "pr_debug_stall_waits": (ctypes.c_int, [_P, ctypes.c_int]),
    "pr_set_one_launch": (ctypes.c_int, [_P, ctypes.c_int]),
    "pr_set_resident": (ctypes.c_int, [_P, ctypes.c_int]),
    "pr_set_wide_rows": (ctypes.c_int, [_P, ctypes.c_int]),
    "pr_serial_sweep": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P, _P]),
    "pr_profile": (ctypes.c_int, [_P, ctypes.c_int]),
    "pr_profile_read": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_double)]),
    "pr_iterate_corrector_phases": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double),
                                                   ctypes.POINTER(ctypes.c_int),
                                                   ctypes.POINTER(ctypes.c_int)]),
    "pr_iterate_adjoint": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P,
                                          _P, _P]),
    "pr_snapshot_project": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int64,
                                           ctypes.c_int64, ctypes.c_int64, ctypes.c_int, _P,
                                           ctypes.c_int64, _P]),
    "pr_snapshot_deflate": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int64, _P,
                                           ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                           ctypes.c_int, _P, ctypes.c_int64, _P]),
}

_lib: Optional[ctypes.CDLL] = None


def declared_symbols() -> list[str]:
    """Entry points declared in include/pr.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(pr_\w+)\s*\(", text, flags=re.M)))


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libpr.so (built by paper_1905_00473_gb300.build) and bind signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libpr.so not built at {path}: run `python -m paper_1905_00473_gb300.build`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _stream_ptr(stream=None) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def _check(status: int, ctx_ptr) -> None:
    if status != 0:
        msg = load().pr_last_error(ctx_ptr)
        raise PrError(status, msg.decode() if msg else "")


# every callback pair ever installed: contexts keep calling the pair they were
# created with (until pr_destroy), so none may be collected
_allocator_refs = []


def pr_set_allocator(alloc=None, release=None) -> None:
    """Device memory of contexts created from now on: alloc(nbytes, device)
    returns a device address (int; 0 on failure) and release(address) gives
    it back; both None restores cudaMalloc.  Contexts keep the pair they were
    created with."""
    if alloc is None and release is None:
        _check(load().pr_set_allocator(_ALLOC_FN(), _RELEASE_FN(), None), None)   # NULL pointers
        return
    if alloc is None or release is None:
        raise ValueError("pr_set_allocator: give both functions or neither")
    ca = _ALLOC_FN(lambda nbytes, dev, user: alloc(int(nbytes), int(dev)) or None)
    cr = _RELEASE_FN(lambda ptr, user: release(int(ptr)))
    _allocator_refs.append((ca, cr))
    _check(load().pr_set_allocator(ca, cr, None), None)


def use_torch_allocator() -> None:
    """Contexts created from now on take their device memory from PyTorch's
    caching allocator (on the current stream of the device)."""
    import torch
    pr_set_allocator(lambda nbytes, dev: torch.cuda.caching_allocator_alloc(nbytes, device=dev),
                     lambda ptr: torch.cuda.caching_allocator_delete(ptr))


class Context:
    """Owns a pr_ctx; methods mirror the C entry points that take a context."""

    def __init__(self, handle: int, dim: int, n: int, N: int, dtype: int, ratio: int = 1):
        self.handle = ctypes.c_void_p(handle)
        self.dim, self.n, self.N, self.dtype, self.ratio = dim, n, N, dtype, ratio

    def __del__(self):
        try:
            if self.handle:
                load().pr_destroy(self.handle)
                self.handle = ctypes.c_void_p(None)
        except Exception:
            pass

    @property
    def torch_dtype(self):
        import torch
        return torch.float32 if self.dtype == PR_F32 else torch.float64

    def _arr(self, t, name: str, count=None, dtype=None):
        import torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        want = self.torch_dtype if dtype is None else dtype
        if t.dtype != want:
            raise TypeError(f"{name} must be {want}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        count = self.N * self.n ** self.dim if count is None else count
        if t.numel() != count:
            raise ValueError(f"{name} must hold {count} values")
        return ctypes.c_void_p(t.data_ptr())

    @property
    def n_coarse(self) -> int:
        return self.n // self.ratio

    @property
    def rows(self) -> int:
        """(d+1) n_c^d: length of an energy-component column."""
        return (self.dim + 1) * self.n_coarse ** self.dim


def pr_create(dim: int, n: int, ratio: int, c, dt_f: float, dt_c: float, N: int, T: float,
              dtype: int = PR_F32, block_depth: int = 0, grad_order: int = 4,
              tol: float = 1e-13) -> Context:
    import torch
    lib = load()
    if not isinstance(c, torch.Tensor) or not c.is_cuda or not c.is_contiguous():
        raise TypeError("c must be a contiguous CUDA tensor")
    want = torch.float32 if dtype == PR_F32 else torch.float64
    if c.dtype != want or c.numel() != n ** dim:
        raise ValueError(f"c must be {want} with n^dim values")
    g = pr_grid(dim, (ctypes.c_int64 * 3)(*([n] * dim + [0] * (3 - dim))), ratio)
    o = pr_options(dtype, grad_order, 0, tol, block_depth, 0)
    out = ctypes.c_void_p()
    st = lib.pr_create(ctypes.byref(g), ctypes.c_void_p(c.data_ptr()), dt_f, dt_c, N, T,
                       ctypes.byref(o), ctypes.byref(out))
    _check(st, None)
    return Context(out.value, dim, n, N, dtype, ratio)


def pr_fine_all_slices(ctx: Context, u_in, v_in, u_out, v_out, n_begin: int = 0,
                       n_end: Optional[int] = None, stream=None) -> None:
    n_end = ctx.N if n_end is None else n_end
    st = load().pr_fine_all_slices(ctx.handle, ctx._arr(u_in, "u_in"), ctx._arr(v_in, "v_in"),
                                   ctx._arr(u_out, "u_out"), ctx._arr(v_out, "v_out"),
                                   n_begin, n_end, ctypes.c_void_p(_stream_ptr(stream)))
    _check(st, ctx.handle)


def pr_check(ctx: Context, stream=None) -> None:
    _check(load().pr_check(ctx.handle, ctypes.c_void_p(_stream_ptr(stream))), ctx.handle)


def pr_info(ctx: Context) -> dict:
    mf, mc, bd = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    pts = ctypes.c_int64()
    _check(load().pr_info(ctx.handle, ctypes.byref(mf), ctypes.byref(mc), ctypes.byref(pts),
                          ctypes.byref(bd)), ctx.handle)
    return {"m_f": mf.value, "m_c": mc.value, "pts": pts.value, "block_depth": bd.value}


def pr_energy(ctx: Context, u, v, n_begin: int = 0, n_end: Optional[int] = None,
              stream=None) -> list[float]:
    n_end = ctx.N if n_end is None else n_end
    out = (ctypes.c_double * max(1, n_end - n_begin))()
    st = load().pr_energy(ctx.handle, ctx._arr(u, "u"), ctx._arr(v, "v"), n_begin, n_end, out,
                          ctypes.c_void_p(_stream_ptr(stream)))
    _check(st, ctx.handle)
    return list(out)[: n_end - n_begin]


def pr_profile(ctx: Context, on: bool) -> None:
    _check(load().pr_profile(ctx.handle, 1 if on else 0), ctx.handle)


def pr_profile_read(ctx: Context, kind: int) -> tuple[int, float]:
    """(launches, summed milliseconds) of kernel kind 0 (fused pass) or 1 (single level)."""
    cnt, ms = ctypes.c_int(), ctypes.c_double()
    _check(load().pr_profile_read(ctx.handle, kind, ctypes.byref(cnt), ctypes.byref(ms)),
           ctx.handle)
    return cnt.value, ms.value


def pr_fine_all_slices_noalloc(c, dt_f: float, m_f: int, u_in, v_in, u_out, v_out,
                               stream=None) -> None:
    """Context-free F over all slices with the library's fixed device scratch
    (no device allocation); FP32 tensors, shapes [N, n, ..., n] with c [n, ..., n].
    Shapes are checked first (ValueError), then dtype, device and layout
    (TypeError), all before anything is launched."""
    import torch
    for name, t in (("c", c), ("u_in", u_in), ("v_in", v_in), ("u_out", u_out), ("v_out", v_out)):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch.Tensor")
    dim = c.dim()
    if dim not in (1, 2, 3):
        raise ValueError("c must have 1, 2 or 3 axes")
    n = int(c.shape[0])
    if any(int(s) != n for s in c.shape):
        # the C entry point takes one n for every axis (n^dim points per slice)
        raise ValueError(f"c must have the same number of points on every axis, got {tuple(c.shape)}")
    if u_in.dim() != dim + 1 or tuple(u_in.shape[1:]) != tuple(c.shape):
        raise ValueError("u_in must be [N, *c.shape]")
    for t in (v_in, u_out, v_out):
        if t.shape != u_in.shape:
            raise ValueError("u_in, v_in, u_out, v_out must have the same shape")
    for name, t in (("c", c), ("u_in", u_in), ("v_in", v_in), ("u_out", u_out), ("v_out", v_out)):
        if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    msg = ctypes.create_string_buffer(512)
    st = load().pr_fine_all_slices_noalloc(
        dim, n, int(u_in.shape[0]), ctypes.c_void_p(c.data_ptr()), dt_f, m_f,
        ctypes.c_void_p(u_in.data_ptr()), ctypes.c_void_p(v_in.data_ptr()),
        ctypes.c_void_p(u_out.data_ptr()), ctypes.c_void_p(v_out.data_ptr()),
        ctypes.c_void_p(_stream_ptr(stream)), msg, len(msg))
    if st != 0:
        raise PrError(st, msg.value.decode())


def pr_coarse_sweep(ctx: Context, u, v, U_out, V_out, n_begin: int = 0,
                    n_end: Optional[int] = None, stream=None) -> None:
    n_end = ctx.N if n_end is None else n_end
    cc = ctx.N * ctx.n_coarse ** ctx.dim
    st = load().pr_coarse_sweep(ctx.handle, ctx._arr(u, "u"), ctx._arr(v, "v"),
                                ctx._arr(U_out, "U_out", cc), ctx._arr(V_out, "V_out", cc),
                                n_begin, n_end, ctypes.c_void_p(_stream_ptr(stream)))
    _check(st, ctx.handle)


def pr_serial_sweep(ctx: Context, corrector: int, Fu, Fv, Uu, Uv, u_slices, v_slices, stream=None) -> None:
    """Serial corrected sweep of Alg. 3: slices 1..N of u_slices/v_slices from
    slice 0, the fine values F u^k_{n-1} (Fu, Fv [N, ...]) and the coarse
    values C R u^k_{n-1} (Uu, Uv [N, coarse ...])."""
    pts = ctx.n ** ctx.dim
    cc = ctx.N * ctx.n_coarse ** ctx.dim
    st = load().pr_serial_sweep(ctx.handle, corrector, ctx._arr(Fu, "Fu", ctx.N * pts),
                                ctx._arr(Fv, "Fv", ctx.N * pts), ctx._arr(Uu, "Uu", cc), ctx._arr(Uv, "Uv", cc),
                                ctx._arr(u_slices, "u_slices", (ctx.N + 1) * pts),
                                ctx._arr(v_slices, "v_slices", (ctx.N + 1) * pts),
                                ctypes.c_void_p(_stream_ptr(stream)))
    _check(st, ctx.handle)


def pr_iterate(ctx: Context, u0, p0, K: int, corrector: int, u_slices, v_slices,
               u_ref=None, v_ref=None, tol_err: float = 0.0, stream=None) -> dict:
    """Runs Alg. 3 for up to K iterations (early stop at tol_err with a reference);
    returns {"k_done", "err", "residual", "rank"} histories."""
    pts = ctx.n ** ctx.dim
    err = (ctypes.c_double * max(1, K))()
    res = (ctypes.c_double * max(1, K))()
    rk = (ctypes.c_int * max(1, K))()
    kd = ctypes.c_int()
    ur = ctx._arr(u_ref, "u_ref", pts) if u_ref is not None else None
    vr = ctx._arr(v_ref, "v_ref", pts) if v_ref is not None else None
    st = load().pr_iterate(ctx.handle, ctx._arr(u0, "u0", pts), ctx._arr(p0, "p0", pts), K,
                           corrector, tol_err, ur, vr,
                           ctx._arr(u_slices, "u_slices", (ctx.N + 1) * pts),
                           ctx._arr(v_slices, "v_slices", (ctx.N + 1) * pts), err, res, rk,
                           ctypes.byref(kd), ctypes.c_void_p(_stream_ptr(stream)))
    _check(st, ctx.handle)
    k = kd.value
    return {"k_done": k, "err": list(err)[:k] if ur is not None else [],
            "residual": list(res)[:k], "rank": list(rk)[:k]}


def pr_iterate_phases(ctx: Context) -> dict:
    """Device milliseconds of the last pr_iterate's phases (Sec. 7.2.4 table columns)."""
    ms = (ctypes.c_double * 4)()
    _check(load().pr_iterate_phases(ctx.handle, ms), ctx.handle)
    return {"initial_coarse_ms": ms[0], "parallel_ms": ms[1], "corrector_ms": ms[2],
            "serial_update_ms": ms[3]}


def pr_procrustes_correct(ctx: Context, Fcols, Gcols, stream=None) -> None:
    """Fcols, Gcols: float64 CUDA tensors [ncols, rows] (one column per row of the tensor)."""
    import torch
    ncols = int(Fcols.shape[0])
    st = load().pr_procrustes_correct(
        ctx.handle, ctx._arr(Fcols, "Fcols", ncols * ctx.rows, torch.float64),
        ctx._arr(Gcols, "Gcols", ncols * ctx.rows, torch.float64), ncols,
        ctypes.c_void_p(_stream_ptr(stream)))
    _check(st, ctx.handle)


def pr_procrustes_apply(ctx: Context, g=None, out=None, stream=None) -> int:
    """out = Omega g; returns the rank s."""
    import torch
    rk = ctypes.c_int()
    gp = ctx._arr(g, "g", ctx.rows, torch.float64) if g is not None else None
    op = ctx._arr(out, "out", ctx.rows, torch.float64) if out is not None else None
    st = load().pr_procrustes_apply(ctx.handle, gp, op, ctypes.byref(rk),
                                    ctypes.c_void_p(_stream_ptr(stream)))
    _check(st, ctx.handle)
    return rk.value


def pr_procrustes_reset(ctx: Context) -> None:
    _check(load().pr_procrustes_reset(ctx.handle), ctx.handle)


def pr_adjoint(ctx: Context, u0, p0, gu_T, gv_T, gc, gu0, gp0, stream=None) -> None:
    """(dL/dc, dL/du0, dL/dp0) into gc, gu0, gp0 for the serial fine solve."""
    pts = ctx.n ** ctx.dim
    a = [ctx._arr(t, nm, pts) for t, nm in ((u0, "u0"), (p0, "p0"), (gu_T, "gu_T"), (gv_T, "gv_T"),
                                           (gc, "gc"), (gu0, "gu0"), (gp0, "gp0"))]
    st = load().pr_adjoint(ctx.handle, *a, ctypes.c_void_p(_stream_ptr(stream)))
    _check(st, ctx.handle)


class Batch:
    """A captured batch of fine sweeps over independent instances (pr_batch_*)."""

    def __init__(self, ctxs, u_in, v_in, u_out, v_out, autotune=True, stream=None):
        n = len(ctxs)
        P = ctypes.c_void_p * n
        self._keep = (list(ctxs), list(u_in), list(v_in), list(u_out), list(v_out))
        arrs = [P(*[ctx._arr(t, name) for ctx, t in zip(ctxs, ts)])
                for name, ts in (("u_in", u_in), ("v_in", v_in), ("u_out", u_out), ("v_out", v_out))]
        out = ctypes.c_void_p()
        st = load().pr_batch_create(n, P(*[c.handle for c in ctxs]), *arrs, 1 if autotune else 0,
                                    ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(out))
        _check(st, None)
        self.handle = out
        self.count = n

    def launch(self, stream=None):
        _check(load().pr_batch_launch(self.handle, ctypes.c_void_p(_stream_ptr(stream))), None)

    def set_mode(self, mode: int, stream=None) -> int:
        """0: per-instance launch chains, 1: one work-queue kernel, -1: time both and keep the
        faster.  Returns the mode in effect."""
        chosen = ctypes.c_int()
        _check(load().pr_batch_set_mode(self.handle, int(mode), ctypes.c_void_p(_stream_ptr(stream)),
                                        ctypes.byref(chosen)), None)
        return chosen.value

    def info(self, i):
        """(block depth, fused columns per thread (0 = the default), tuned ms) of instance i."""
        d, c, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(load().pr_batch_info(self.handle, i, ctypes.byref(d), ctypes.byref(c), ctypes.byref(ms)),
               None)
        return d.value, c.value, ms.value

    def __del__(self):
        try:
            if self.handle:
                load().pr_batch_destroy(self.handle)
                self.handle = ctypes.c_void_p(None)
        except Exception:
            pass


def pr_set_fused_columns(ctx: Context, columns: int) -> None:
    """Columns per thread of the fused 2D kernels: 2, 4 or 0 (by grid width)."""
    _check(load().pr_set_fused_columns(ctx.handle, int(columns)), ctx.handle)


def pr_debug_stall_waits(ctx: Context, enable: bool) -> None:
    _check(load().pr_debug_stall_waits(ctx.handle, 1 if enable else 0), ctx.handle)


def _f64_matrix(name: str, t, rows: int, cols: int):
    """(pointer, leading dimension) of a column-major FP64 CUDA matrix given as
    a torch tensor of shape (cols, rows) (each column contiguous)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    if t.dim() != 2 or t.shape[0] != cols or t.shape[1] != rows or t.stride(1) != 1:
        raise ValueError(f"{name} must have shape ({cols}, {rows}) with unit stride in rows")
    return ctypes.c_void_p(t.data_ptr()), max(int(t.stride(0)), rows, 1)


def pr_snapshot_project(ctx: Context, A, B, C, stream=None) -> None:
    """C = A^T B on the tensor cores (split-TF32).  Column-major matrices are
    passed as tensors of shape (columns, rows): A (M, K), B (N, K), C (N, M)."""
    M, K = int(A.shape[0]), int(A.shape[1])
    N = int(B.shape[0])
    pa, lda = _f64_matrix("A", A, K, M)
    pb, ldb = _f64_matrix("B", B, K, N)
    pc, ldc = _f64_matrix("C", C, M, N)
    _check(load().pr_snapshot_project(ctx.handle, pa, lda, pb, ldb, K, M, N, pc, ldc,
                                      ctypes.c_void_p(_stream_ptr(stream))), ctx.handle)


def pr_snapshot_deflate(ctx: Context, A, T, F, O, stream=None) -> None:
    """O = F - A T on the tensor cores (split-TF32).  Shapes (columns, rows):
    A (K, M), T (N, K), F and O (N, M)."""
    K, M = int(A.shape[0]), int(A.shape[1])
    N = int(F.shape[0])
    pa, lda = _f64_matrix("A", A, M, K)
    pt, ldt = _f64_matrix("T", T, K, N)
    pf, ldf = _f64_matrix("F", F, M, N)
    po, ldo = _f64_matrix("O", O, M, N)
    _check(load().pr_snapshot_deflate(ctx.handle, pa, lda, pt, ldt, pf, ldf, M, K, N, po, ldo,
                                      ctypes.c_void_p(_stream_ptr(stream))), ctx.handle)


def pr_iterate_corrector_phases(ctx: Context) -> dict:
    """Device time (ms) of the steps of creating the corrector in the last
    pr_iterate call, and how many SVDs went through the eigenproblem path."""
    ms = (ctypes.c_double * 5)()
    ne, na = ctypes.c_int(), ctypes.c_int()
    _check(load().pr_iterate_corrector_phases(ctx.handle, ms, ctypes.byref(ne), ctypes.byref(na)),
           ctx.handle)
    keys = ("project_deflate_ms", "qr_ms", "h_svd_ms", "rotate_ms", "residual_ms")
    out = {k: ms[i] for i, k in enumerate(keys)}
    out["eig_svds"], out["svds"] = ne.value, na.value
    return out


def pr_iterate_adjoint(ctx: Context, u0, p0, K: int, corrector: int, gu_T, gv_T, gc, gu0, gp0,
                       stream=None) -> None:
    """Reverse mode through K iterations of Alg. 3 with the correctors frozen:
    writes dL/dc, dL/du0, dL/dp0 for dL/du, dL/du_t at u^{K+1}_N."""
    pts = ctx.n ** ctx.dim
    st = load().pr_iterate_adjoint(ctx.handle, ctx._arr(u0, "u0", pts), ctx._arr(p0, "p0", pts), K,
                                   corrector, ctx._arr(gu_T, "gu_T", pts), ctx._arr(gv_T, "gv_T", pts),
                                   ctx._arr(gc, "gc", pts), ctx._arr(gu0, "gu0", pts),
                                   ctx._arr(gp0, "gp0", pts), ctypes.c_void_p(_stream_ptr(stream)))
    _check(st, ctx.handle)


def pr_set_one_launch(ctx: Context, on: bool) -> None:
    """Whole sweep in one persistent launch, or one launch per pass (the default)."""
    _check(load().pr_set_one_launch(ctx.handle, 1 if on else 0), ctx.handle)


def pr_set_wide_rows(ctx: Context, mode: int) -> None:
    """2048-point rows at depth 8: 1 = two-CTA cluster rows, 2 = x-strips."""
    _check(load().pr_set_wide_rows(ctx.handle, int(mode)), ctx.handle)


def pr_set_resident(ctx: Context, on: bool) -> None:
    """Small 2D slices held in cluster shared memory for all kicks, or the
    per-pass launches (default: on at n = 128, off at n = 256)."""
    _check(load().pr_set_resident(ctx.handle, 1 if on else 0), ctx.handle)
