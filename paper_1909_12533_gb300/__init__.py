"""Python binding of the SP2 C ABI (include/sp2.h).

Argument marshalling only: every step of the expansion runs inside
``libsp2.so`` (CUDA kernels for sm_103a plus the host driver).  The library must
be built (``python -m paper_1909_12533_gb300.build``); there is no fallback.

Low level: ``sp2_default_params``, ``sp2_create``, ``sp2_run``, ``sp2_get_D``,
``sp2_copy_D``, ``sp2_backward``, ``sp2_get_stats``, ``sp2_destroy``,
``sp2_strerror`` mirror the C entry points.  ``SP2`` wraps one context and
``SP2Function`` is the ``torch.autograd.Function`` (L = trace(D W)).
"""
from __future__ import annotations

import ctypes
from ctypes import POINTER, byref, c_double, c_int32, c_int64, c_size_t, c_void_p
from pathlib import Path

import numpy as np

TILE = 32
MAX_ITER = 128

SP2_OK = 0
ERRORS = {
    -1: "SP2_ERR_INVALID_ARG", -2: "SP2_ERR_BOUNDS", -3: "SP2_ERR_PATTERN", -4: "SP2_ERR_NONFINITE",
    -5: "SP2_ERR_OOM", -6: "SP2_ERR_CUDA", -7: "SP2_ERR_NOT_CONVERGED", -8: "SP2_ERR_TIMEOUT",
    -9: "SP2_ERR_STATE", -10: "SP2_ERR_CAPACITY", -11: "SP2_ERR_TOO_LARGE", -12: "SP2_ERR_RANGE",
}
NOT_CONVERGED = -7
MODES = {"sp2": 0, "sp2acc": 1, "trace": 2}
STOPS = {"parameterless": 0, "idempotency": 1}
TRUNCS = {"frobenius": 0, "frobinf": 1, "mixed": 2}
PRECISIONS = {"fp64": 0, "split16": 1}
STORAGES = {"symmetric": 0, "general": 1}


class sp2_bsr(ctypes.Structure):
    _fields_ = [("n", c_int64), ("b", c_int32), ("nnzb", c_int64), ("brow", c_void_p), ("bcol", c_void_p),
                ("val", c_void_p), ("on_device", c_int32)]


class sp2_allocator(ctypes.Structure):
    _fields_ = [("alloc", c_void_p), ("free", c_void_p), ("user", c_void_p)]


class sp2_params(ctypes.Structure):
    _fields_ = [("mode", c_int32), ("stop", c_int32), ("idem_tol", c_double), ("trunc", c_int32),
                ("frobinf_part", c_int64), ("gamma", c_double), ("delta_acc", c_double), ("n_max_cap", c_int32),
                ("precision", c_int32), ("slices", c_int32), ("mixed_from", c_int32), ("mixed_until", c_int32),
                ("ckpt_every", c_int32), ("record_masks", c_int32), ("fp64_tail", c_double),
                ("acc_flush_min", c_int32), ("wait_limit_ms", c_int32), ("selftest", c_int32),
                ("storage", c_int32), ("split_supply", c_int32)]


class sp2_stats(ctypes.Structure):
    _fields_ = [("status", c_int32), ("converged", c_int32), ("n", c_int32), ("n_min", c_int32), ("n_max", c_int32),
                ("squares", c_int32), ("lmin", c_double), ("lmax", c_double), ("homo_est", c_double),
                ("lumo_est", c_double), ("have_estimates", c_int32), ("nnzb_final", c_int64),
                ("tile_triplets", c_int64), ("alg_flops", c_double), ("run_ms", c_double), ("square_ms", c_double),
                ("p", c_int32 * MAX_ITER), ("alpha", c_double * MAX_ITER), ("tau", c_double * MAX_ITER),
                ("e", c_double * MAX_ITER), ("t", c_double * MAX_ITER), ("nnzb_hist", c_int64 * MAX_ITER),
                ("prec_hist", c_int32 * MAX_ITER), ("kernel_launches", c_int64),
                ("backward_ms", c_double), ("tc_hw_flops", c_double)]


# Entry points declared in include/sp2.h: (name, restype, argtypes)
_SIGS = [
    ("sp2_default_params", c_int32, [POINTER(sp2_params)]),
    ("sp2_create", c_int32, [POINTER(sp2_bsr), c_int64, c_double, c_double, c_double, POINTER(sp2_params),
                             POINTER(sp2_allocator), c_void_p, POINTER(c_void_p)]),
    ("sp2_create_dense", c_int32, [c_void_p, c_int64, c_int64, c_int32, c_int64, c_double, c_double, c_double,
                                   POINTER(sp2_params), POINTER(sp2_allocator), c_void_p, POINTER(c_void_p)]),
    ("sp2_run", c_int32, [c_void_p, POINTER(sp2_stats)]),
    ("sp2_estimate_bounds", c_int32, [c_void_p, c_double, POINTER(c_double), POINTER(c_double)]),
    ("sp2_get_D", c_int32, [c_void_p, POINTER(sp2_bsr)]),
    ("sp2_copy_D", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int32, POINTER(c_int64)]),
    ("sp2_copy_D_dense", c_int32, [c_void_p, c_void_p, c_int64, c_int32]),
    ("sp2_backward", c_int32, [c_void_p, POINTER(sp2_bsr), POINTER(sp2_bsr)]),
    ("sp2_truncate", c_int32, [POINTER(sp2_bsr), c_double, c_int32, c_int64, c_void_p, c_void_p]),
    ("sp2_truncate_noalloc", c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_double, c_int32, c_int64,
                                       c_void_p, c_void_p]),
    ("sp2_get_stats", c_int32, [c_void_p, POINTER(sp2_stats)]),
    ("sp2_destroy", None, [c_void_p]),
    ("sp2_strerror", ctypes.c_char_p, [c_int32]),
    ("sp2_release_memory", c_int32, []),
]

_LIB = None


def lib_path() -> Path:
    return Path(__file__).with_name("libsp2.so")


def load() -> ctypes.CDLL:
    """Load libsp2.so (raises if it has not been built; there is no fallback)."""
    global _LIB
    if _LIB is None:
        p = lib_path()
        if not p.exists():
            raise RuntimeError(f"{p} is missing: build it with `python -m paper_1909_12533_gb300.build`")
        lib = ctypes.CDLL(str(p))
        for name, res, args in _SIGS:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


class SP2Error(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({sp2_strerror(code)})")


def sp2_strerror(code: int) -> str:
    return load().sp2_strerror(code).decode()


def sp2_release_memory() -> None:
    """Return the device memory the library's pools keep for reuse."""
    rc = load().sp2_release_memory()
    if rc != SP2_OK:
        raise SP2Error(rc, "sp2_release_memory")


def sp2_default_params(**overrides) -> sp2_params:
    p = sp2_params()
    rc = load().sp2_default_params(byref(p))
    if rc != SP2_OK:
        raise SP2Error(rc, "sp2_default_params")
    enums = {"mode": MODES, "stop": STOPS, "trunc": TRUNCS, "precision": PRECISIONS, "storage": STORAGES}
    for k, v in overrides.items():
        if k in enums and isinstance(v, str):
            v = enums[k][v]
        setattr(p, k, v)
    return p


# ------------------------------------------------------------------ marshalling
def _ptr(a):
    """(pointer, on_device) of a numpy array or torch tensor (kept alive by caller)."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data, 0
    return int(a.data_ptr()), 1 if a.is_cuda else 0


def make_bsr(n: int, brow, bcol, val) -> tuple[sp2_bsr, tuple]:
    """Build an sp2_bsr over numpy arrays or torch tensors (int32, int32, float64,
    contiguous).  Returns the struct and the objects that must stay alive."""
    if isinstance(brow, np.ndarray):
        brow = np.ascontiguousarray(brow, dtype=np.int32)
        bcol = np.ascontiguousarray(bcol, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float64)
    else:
        import torch
        brow = brow.to(torch.int32).contiguous()
        bcol = bcol.to(torch.int32).contiguous()
        val = val.to(torch.float64).contiguous()
    pb, d1 = _ptr(brow)
    pc, d2 = _ptr(bcol)
    pv, d3 = _ptr(val)
    if not (d1 == d2 == d3):
        raise ValueError("brow, bcol and val must all be host or all be device buffers")
    s = sp2_bsr(n=int(n), b=TILE, nnzb=int(brow.shape[0]), brow=pb, bcol=pc, val=pv, on_device=d1)
    return s, (brow, bcol, val)


def _stream_handle(stream):
    if stream is not None:
        return c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return c_void_p(int(torch.cuda.current_stream().cuda_stream))
    except Exception:  # pragma: no cover - torch missing
        pass
    return c_void_p(0)


def _is_dense(F) -> bool:
    """A 2-D numpy array or torch tensor (dense F), as opposed to a tile set."""
    shape = getattr(F, "shape", None)
    return shape is not None and len(shape) == 2 and not hasattr(F, "brow")


def sp2_create(F, nocc: int, homo_ub: float, lumo_lb: float, tau: float, params: sp2_params | None = None,
               stream=None, allocator: sp2_allocator | None = None) -> c_void_p:
    """F: a tile set (object with n, brow, bcol, val: numpy -> host copy, CUDA
    tensors -> device copy), or a dense symmetric 2-D float64 numpy array / torch
    tensor (sp2_create_dense).  ``allocator``: an sp2_allocator whose alloc/free
    are ctypes callbacks (the caller keeps them alive), None = library pool."""
    ctx = c_void_p()
    prm = params if params is not None else sp2_default_params()
    al = byref(allocator) if allocator is not None else None
    if _is_dense(F):
        if isinstance(F, np.ndarray):
            Fd = np.ascontiguousarray(F, dtype=np.float64)
        else:
            import torch
            Fd = F.to(torch.float64).contiguous()
        ptr, on_dev = _ptr(Fd)
        n = int(Fd.shape[0])
        if Fd.shape[1] != n:
            raise ValueError("dense F must be square")
        rc = load().sp2_create_dense(c_void_p(ptr), n, n, on_dev, int(nocc), float(homo_ub), float(lumo_lb),
                                     float(tau), byref(prm), al, _stream_handle(stream), byref(ctx))
        del Fd
    else:
        bsr, keep = make_bsr(F.n, F.brow, F.bcol, F.val)
        rc = load().sp2_create(byref(bsr), int(nocc), float(homo_ub), float(lumo_lb), float(tau), byref(prm), al,
                               _stream_handle(stream), byref(ctx))
        del keep
    if rc != SP2_OK:
        raise SP2Error(rc, "sp2_create")
    return ctx


def sp2_run(ctx) -> tuple[int, sp2_stats]:
    st = sp2_stats()
    rc = load().sp2_run(ctx, byref(st))
    if rc not in (SP2_OK, NOT_CONVERGED):
        raise SP2Error(rc, "sp2_run")
    return rc, st


def sp2_estimate_bounds(ctx, margin: float = 0.1) -> tuple[float, float]:
    """(homo_ub, lumo_lb) for a second run from the Step 3 estimates of the
    last run of ctx, each moved away from the gap by margin * estimated gap."""
    h = c_double()
    l = c_double()
    rc = load().sp2_estimate_bounds(ctx, float(margin), byref(h), byref(l))
    if rc != SP2_OK:
        raise SP2Error(rc, "sp2_estimate_bounds")
    return h.value, l.value


def sp2_get_D(ctx) -> sp2_bsr:
    v = sp2_bsr()
    rc = load().sp2_get_D(ctx, byref(v))
    if rc != SP2_OK:
        raise SP2Error(rc, "sp2_get_D")
    return v


def sp2_copy_D(ctx, out=None):
    """Host copy of D: (brow, bcol, val).  Without ``out``, new numpy arrays;
    with ``out`` = (brow, bcol, val) host buffers (numpy arrays or CPU torch
    tensors, e.g. pinned, with room for at least nnzb tiles) the tiles are copied
    into them and views of length nnzb are returned."""
    n = c_int64()
    rc = load().sp2_copy_D(ctx, None, None, None, 0, 0, byref(n))
    if rc not in (SP2_OK, -10):
        raise SP2Error(rc, "sp2_copy_D")
    if out is None:
        brow = np.empty(n.value, np.int32)
        bcol = np.empty(n.value, np.int32)
        val = np.empty((n.value, TILE, TILE), np.float64)
    else:
        brow, bcol, val = out
        if brow.shape[0] < n.value or bcol.shape[0] < n.value or val.shape[0] < n.value:
            raise ValueError("output buffers hold fewer tiles than D")
        for x, kind in ((brow, "int32"), (bcol, "int32"), (val, "float64")):
            if str(x.dtype).split(".")[-1] != kind or not (x.flags["C_CONTIGUOUS"] if isinstance(x, np.ndarray)
                                                          else x.is_contiguous()):
                raise ValueError("output buffers must be contiguous int32, int32, float64")
    ptrs = [_ptr(x) for x in (brow, bcol, val)]
    if any(d for _, d in ptrs):
        raise ValueError("sp2_copy_D writes host buffers")
    rc = load().sp2_copy_D(ctx, ptrs[0][0], ptrs[1][0], ptrs[2][0], n.value, 0, byref(n))
    if rc != SP2_OK:
        raise SP2Error(rc, "sp2_copy_D")
    return brow[: n.value], bcol[: n.value], val[: n.value]


def sp2_copy_D_dense(ctx, out=None, device: bool = False):
    """D as a dense symmetric matrix.  ``out``: a contiguous float64 n x n numpy
    array / CPU tensor (host) or CUDA tensor (device); without it a new numpy
    array (device=False) or CUDA tensor (device=True) is returned."""
    v = sp2_get_D(ctx)
    n = int(v.n)
    if out is None:
        if device:
            import torch
            out = torch.empty((n, n), dtype=torch.float64, device="cuda")
        else:
            out = np.empty((n, n), np.float64)
    ptr, on_dev = _ptr(out)
    if tuple(out.shape) != (n, n):
        raise ValueError(f"out must be {n} x {n}")
    rc = load().sp2_copy_D_dense(ctx, c_void_p(ptr), n, on_dev)
    if rc != SP2_OK:
        raise SP2Error(rc, "sp2_copy_D_dense")
    return out


def sp2_backward(ctx, W) -> sp2_bsr:
    bsr, keep = make_bsr(W.n, W.brow, W.bcol, W.val)
    out = sp2_bsr()
    rc = load().sp2_backward(ctx, byref(bsr), byref(out))
    del keep
    if rc != SP2_OK:
        raise SP2Error(rc, "sp2_backward")
    return out


def sp2_truncate(X, tau: float, mode="frobenius", frobinf_part: int = 4096, stream=None):
    """Keep flags (1 = kept) of X's tiles after the truncation of Eq. (8).
    Host inputs give a numpy array, device inputs a torch CUDA tensor."""
    bsr, keep_alive = make_bsr(X.n, X.brow, X.bcol, X.val)
    m = TRUNCS[mode] if isinstance(mode, str) else int(mode)
    if bsr.on_device:
        import torch
        keep = torch.empty(bsr.nnzb, dtype=torch.int32, device="cuda")
        kp = keep.data_ptr()
    else:
        keep = np.empty(bsr.nnzb, np.int32)
        kp = keep.ctypes.data
    rc = load().sp2_truncate(byref(bsr), float(tau), m, int(frobinf_part), c_void_p(kp), _stream_handle(stream))
    del keep_alive
    if rc != SP2_OK:
        raise SP2Error(rc, "sp2_truncate")
    return keep


def sp2_get_stats(ctx) -> sp2_stats:
    st = sp2_stats()
    rc = load().sp2_get_stats(ctx, byref(st))
    if rc != SP2_OK:
        raise SP2Error(rc, "sp2_get_stats")
    return st


def sp2_destroy(ctx) -> None:
    if ctx:
        load().sp2_destroy(ctx)


def stats_dict(st: sp2_stats) -> dict:
    n = st.n
    sq = st.squares
    d = {k: getattr(st, k) for k, *_ in sp2_stats._fields_ if k not in
         ("p", "alpha", "tau", "e", "t", "nnzb_hist", "prec_hist")}
    nm = st.n_max
    d["p"] = [st.p[i] for i in range(nm + 1)]
    d["alpha"] = [st.alpha[i] for i in range(nm + 1)]
    d["tau"] = [st.tau[i] for i in range(nm + 1)]
    d["e"] = [st.e[i] for i in range(sq)]
    d["t"] = [st.t[i] for i in range(sq)]
    d["nnzb_hist"] = [st.nnzb_hist[i] for i in range(max(n + 1, 0))]
    d["prec_hist"] = [st.prec_hist[i] for i in range(sq)]
    return d


def device_view_to_torch(v: sp2_bsr):
    """Copy a borrowed device view into fresh torch CUDA tensors (brow, bcol, val)."""
    import torch
    n = v.nnzb
    brow = torch.empty(n, dtype=torch.int32, device="cuda")
    bcol = torch.empty(n, dtype=torch.int32, device="cuda")
    val = torch.empty((n, TILE, TILE), dtype=torch.float64, device="cuda")
    cudart = _cudart()
    for dst, src, nbytes in ((brow, v.brow, n * 4), (bcol, v.bcol, n * 4), (val, v.val, n * TILE * TILE * 8)):
        if nbytes:
            rc = cudart.cudaMemcpyAsync(c_void_p(dst.data_ptr()), c_void_p(src), c_size_t(nbytes), 3,
                                        c_void_p(torch.cuda.current_stream().cuda_stream))
            if rc != 0:
                raise RuntimeError(f"cudaMemcpyAsync failed ({rc})")
    return brow, bcol, val


_CUDART = None


def _cudart():
    global _CUDART
    if _CUDART is None:
        import glob
        import torch  # noqa: F401  (loads the runtime torch was built with)
        cands = ["libcudart.so.13", "libcudart.so.12", "libcudart.so"]
        for c in cands:
            try:
                _CUDART = ctypes.CDLL(c)
                break
            except OSError:
                continue
        if _CUDART is None:
            for g in glob.glob("/usr/local/cuda/lib64/libcudart.so*"):
                _CUDART = ctypes.CDLL(g)
                break
        _CUDART.cudaMemcpyAsync.argtypes = [c_void_p, c_void_p, c_size_t, c_int32, c_void_p]
        _CUDART.cudaMemcpyAsync.restype = c_int32
    return _CUDART


# ------------------------------------------------------------------ convenience
class SP2:
    """One SP2 context: create on construction, ``run()``, ``D_host()``,
    ``D_device()``, ``backward(W)``, ``close()``."""

    def __init__(self, F, nocc, homo_ub, lumo_lb, tau, stream=None, allocator=None, **params):
        self.prm = sp2_default_params(**params)
        self.F = F
        self.allocator = allocator      # kept alive with the context
        self.ctx = sp2_create(F, nocc, homo_ub, lumo_lb, tau, self.prm, stream, allocator)
        self.code = None
        self.stats = None

    def run(self) -> dict:
        self.code, st = sp2_run(self.ctx)
        self.stats = stats_dict(st)
        return self.stats

    def D_host(self, out=None):
        return sp2_copy_D(self.ctx, out)

    def D_device(self):
        return device_view_to_torch(sp2_get_D(self.ctx))

    def D_dense(self, out=None, device: bool = False):
        return sp2_copy_D_dense(self.ctx, out, device)

    def backward(self, W):
        return device_view_to_torch(sp2_backward(self.ctx, W))

    def close(self):
        if self.ctx:
            sp2_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run(F, nocc, homo_ub, lumo_lb, tau, stream=None, **params):
    """One SP2 expansion: D and the run statistics.

    F is a tile set (n, brow, bcol, val) or a dense symmetric matrix (numpy
    array or torch tensor).  Returns (D, stats): for a dense F, D is dense
    (numpy on the host, a CUDA tensor when F is a CUDA tensor); for a tile set,
    D is (brow, bcol, val) on the host.  Raises SP2Error on failure; a run that
    hits n_max without the stop test firing returns with stats["converged"] = 0."""
    ctx = SP2(F, nocc, homo_ub, lumo_lb, tau, stream=stream, **params)
    try:
        st = ctx.run()
        if _is_dense(F):
            D = ctx.D_dense(device=not isinstance(F, np.ndarray) and bool(getattr(F, "is_cuda", False)))
        else:
            D = ctx.D_host()
    finally:
        ctx.close()
    return D, st


def run_two_pass(F, nocc, tau1, tau, margin: float = 0.1, stream=None, first=None, **params):
    """Section 6's protocol when no eigenvalue bounds are known: run 1 is the
    trace-correcting expansion (mode "trace") with the threshold tau1, its Step 3
    estimates widened by ``margin`` (sp2_estimate_bounds) are the homo/lumo
    bounds of run 2, the SP2ACC expansion with tau (and **params).  ``first``:
    extra parameters of run 1 only.  Returns (D, stats of run 2, stats of run 1,
    (homo_ub, lumo_lb)) with D as ``run`` returns it."""
    p1 = dict(params)
    p1.pop("gamma", None)
    p1.update(first or {})
    p1["mode"] = "trace"
    ctx = SP2(F, nocc, float("nan"), float("nan"), tau1, stream=stream, **p1)
    try:
        st1 = ctx.run()
        bounds = sp2_estimate_bounds(ctx.ctx, margin)
    finally:
        ctx.close()
    D, st2 = run(F, nocc, bounds[0], bounds[1], tau, stream=stream, **params)
    return D, st2, st1, bounds


def header_functions() -> list[str]:
    """Names of the functions declared in include/sp2.h (for export checks)."""
    import re
    h = (Path(__file__).resolve().parent.parent / "include" / "sp2.h").read_text()
    h = re.sub(r"/\*.*?\*/", " ", h, flags=re.S)  # drop comments
    return sorted(set(re.findall(r"^\s*(?:int|void|const\s+char\s*\*)\s*(sp2_[A-Za-z0-9_]+)\s*\(", h, re.M)))


# ------------------------------------------------------------------ autograd
def _autograd_function():
    import torch

    class _Tiles:
        def __init__(self, n, brow, bcol, val):
            self.n, self.brow, self.bcol, self.val = n, brow, bcol, val

    class SP2Function(torch.autograd.Function):
        """D = SP2ACC(F) on the tile pattern of F (stored upper tiles, CUDA tensors).

        forward(F_val, F_brow, F_bcol, n, nocc, homo_ub, lumo_lb, tau, params)
        returns (D_val, D_brow, D_bcol); only D_val carries a gradient.
        params: sp2_params fields by name, plus allow_not_converged (default
        False: a run that reaches n_max without the stop test raises SP2Error).
        backward: for L with dL/dD_val = gD, W = gD on D's pattern with
        off-diagonal tiles halved (each stands for two blocks of the symmetric
        D), so L = trace(D W); sp2_backward gives dF_ij = dL/dF_ij, and a stored
        off-diagonal F tile (F_IJ and F_JI) receives 2 dF_IJ."""

        @staticmethod
        def forward(ctx, F_val, F_brow, F_bcol, n, nocc, homo_ub, lumo_lb, tau, params=None):
            F = _Tiles(int(n), F_brow, F_bcol, F_val.detach())
            prm = dict(params or {})
            allow = bool(prm.pop("allow_not_converged", False))
            prm["record_masks"] = 1
            obj = SP2(F, nocc, homo_ub, lumo_lb, tau, **prm)
            obj.run()
            if obj.code == NOT_CONVERGED and not allow:
                obj.close()
                raise SP2Error(obj.code, "sp2_run (pass allow_not_converged=True in params to accept the last "
                                         "iterate)")
            if obj.code not in (SP2_OK, NOT_CONVERGED):
                raise SP2Error(obj.code, "sp2_run")
            d_brow, d_bcol, d_val = obj.D_device()
            ctx.obj = obj
            ctx.n = int(n)
            ctx.f_off = (F_brow != F_bcol)
            ctx.save_for_backward(d_brow, d_bcol)
            ctx.mark_non_differentiable(d_brow, d_bcol)
            return d_val, d_brow, d_bcol

        @staticmethod
        def backward(ctx, g_val, _g_brow, _g_bcol):
            d_brow, d_bcol = ctx.saved_tensors
            w = g_val.detach().to(torch.float64).clone()
            off = d_brow != d_bcol
            w[off] *= 0.5
            W = _Tiles(ctx.n, d_brow, d_bcol, w.contiguous())
            # the context stays open until this autograd node is freed, so a
            # second backward (retain_graph=True) runs the same recorded sweep
            _, _, dF = ctx.obj.backward(W)
            dF = dF.clone()
            dF[ctx.f_off] *= 2.0
            return dF, None, None, None, None, None, None, None, None

    return SP2Function


_SP2_FUNCTION = None


def __getattr__(name):
    # built on first use (imports torch), then the same class every time
    global _SP2_FUNCTION
    if name == "SP2Function":
        if _SP2_FUNCTION is None:
            _SP2_FUNCTION = _autograd_function()
        return _SP2_FUNCTION
    raise AttributeError(name)
