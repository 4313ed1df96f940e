"""Python binding of the LocalPower C ABI (include/localpower.h).

Argument marshalling only: every step of the method runs in the CUDA library.
Host data are NumPy arrays (pointer space LP_HOST); device data are CUDA
torch tensors (LP_DEVICE, via ``data_ptr()``), torch being used only as a
holder of device memory and streams.  The functions keep the C names.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

LP_OK, LP_ERR_INVALID, LP_ERR_STATE, LP_ERR_OOM, LP_ERR_CUDA, LP_ERR_NUMERIC, LP_ERR_TIMEOUT, LP_ERR_UNSUPPORTED = range(8)
STATUS_NAMES = ["LP_OK", "LP_ERR_INVALID", "LP_ERR_STATE", "LP_ERR_OOM", "LP_ERR_CUDA", "LP_ERR_NUMERIC",
                "LP_ERR_TIMEOUT", "LP_ERR_UNSUPPORTED"]
LP_F32, LP_BF16, LP_FP8_E4M3, LP_F32_BF16X2 = 0, 1, 2, 3
LP_AGG_IDENTITY, LP_AGG_SIGN, LP_AGG_OPT = 0, 1, 2
LP_HOST, LP_DEVICE = 0, 1
LP_FLAG_RITZ, LP_FLAG_TIMING, LP_FLAG_SIMT, LP_FLAG_TC_RESIDENT, LP_FLAG_NO_GRAPH, LP_FLAG_TRACE = 1, 2, 4, 8, 16, 32
LP_FLAG_KXK_FP64 = 64
LP_MAX_K = 32

AGG = {"identity": LP_AGG_IDENTITY, "sign": LP_AGG_SIGN, "opt": LP_AGG_OPT}
DTYPE = {"f32": LP_F32, "bf16": LP_BF16, "e4m3": LP_FP8_E4M3, "f32_bf16x2": LP_F32_BF16X2}
PATHS = {0: "simt", 1: "tc_resident", 2: "tc_streaming", 3: "tc_pair"}

# Every symbol the header declares, in declaration order.
EXPORTS = ["lp_create", "lp_load_partitions", "lp_solve", "lp_solve_seeded", "lp_result", "lp_destroy", "lp_last_error",
           "lp_set_tuning", "lp_autotune", "lp_trace", "lp_eta", "lp_server_create", "lp_server_submit", "lp_server_progress",
           "lp_server_result", "lp_server_query", "lp_server_error", "lp_server_destroy", "lp_batch_create",
           "lp_batch_add", "lp_batch_autotune", "lp_batch_solve", "lp_batch_result", "lp_batch_size",
           "lp_batch_groups", "lp_batch_error", "lp_batch_destroy", "lp_power_step", "lp_orth", "lp_align_aggregate", "lp_power_step_static"]


class lp_stats(C.Structure):
    _fields_ = [("rounds", C.c_int32), ("local_steps", C.c_int32), ("step_launches", C.c_int32), ("k", C.c_int32),
                ("n", C.c_int64), ("d", C.c_int64), ("m", C.c_int32), ("path", C.c_int32),
                ("a_bytes", C.c_double), ("ms_solve", C.c_double), ("ms_step_kernels", C.c_double),
                ("kernel_launches", C.c_int32), ("reserved", C.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class lp_tuning(C.Structure):
    _fields_ = [("ring_units", C.c_int32), ("lag_units", C.c_int32), ("prefetch_units", C.c_int32),
                ("cache_hints", C.c_int32), ("slice_cols", C.c_int32), ("kernel", C.c_int32),
                ("test_stall_cycles", C.c_int32)]


class lp_request(C.Structure):
    _fields_ = [("m", C.c_int), ("rows", C.POINTER(C.c_int64)), ("d", C.c_int64), ("row_pitch", C.c_int64),
                ("dtype", C.c_int), ("parts", C.POINTER(C.c_void_p)), ("row_scales", C.POINTER(C.c_void_p)),
                ("space", C.c_int), ("k", C.c_int), ("p_schedule", C.POINTER(C.c_int)), ("T", C.c_int),
                ("agg", C.c_int), ("y0", C.POINTER(C.c_double)), ("refine_rounds", C.c_int), ("flags", C.c_uint)]


class lp_server_info(C.Structure):
    _fields_ = [("queued", C.c_int64), ("active", C.c_int64), ("completed", C.c_int64),
                ("hbm_in_use", C.c_uint64), ("hbm_peak", C.c_uint64), ("hbm_budget", C.c_uint64)]


class LPError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {message}")


_lib: C.CDLL | None = None


def lib_path() -> str:
    from . import build
    return build.LIB_PATH


def load(path: str | None = None, build_if_missing: bool = True) -> C.CDLL:
    """Load the shared library (building it first if it is absent).  Raises if
    it cannot be built or loaded: there is no fallback path."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        from . import build
        path = build.build() if build_if_missing else build.LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"LocalPower CUDA library not found at {path}")
    L = C.CDLL(path)
    P, I, I64, U = C.c_void_p, C.c_int, C.c_int64, C.c_uint
    L.lp_create.argtypes = [C.POINTER(P), I, C.c_size_t, P]
    L.lp_load_partitions.argtypes = [P, I, C.POINTER(I64), I64, I, C.POINTER(P), C.POINTER(P), I]
    L.lp_solve.argtypes = [P, I, C.POINTER(I), I, I, P, I, U]
    L.lp_solve_seeded.argtypes = [P, I, C.POINTER(I), I, I, C.c_uint64, I, U]
    L.lp_result.argtypes = [P, P, P, C.POINTER(lp_stats)]
    L.lp_destroy.argtypes = [P]
    L.lp_destroy.restype = None
    L.lp_last_error.argtypes = [P]
    L.lp_last_error.restype = C.c_char_p
    L.lp_power_step.argtypes = [P, I, P, I, P, I]
    L.lp_orth.argtypes = [P, I, I64, I, P, P, I, C.c_uint]
    L.lp_align_aggregate.argtypes = [P, I, I64, I, I, I, P, P, P, P, P, I, C.c_uint]
    L.lp_power_step_static.argtypes = [P, I, C.POINTER(I64), I64, I, P, P, P]
    L.lp_set_tuning.argtypes = [P, C.POINTER(lp_tuning)]
    L.lp_trace.argtypes = [P, P, P]
    L.lp_eta.argtypes = [P, P, P]
    L.lp_autotune.argtypes = [P, I, C.POINTER(lp_tuning), C.POINTER(I), C.POINTER(C.c_double)]
    L.lp_server_create.argtypes = [C.POINTER(P), I, C.c_size_t, I]
    L.lp_server_submit.argtypes = [P, C.POINTER(lp_request), C.POINTER(I64)]
    L.lp_server_progress.argtypes = [P, C.POINTER(I64), I, C.POINTER(I)]
    L.lp_server_result.argtypes = [P, I64, P, P, C.POINTER(lp_stats)]
    L.lp_server_query.argtypes = [P, C.POINTER(lp_server_info)]
    L.lp_server_error.argtypes = [P]
    L.lp_server_error.restype = C.c_char_p
    L.lp_server_destroy.argtypes = [P]
    L.lp_server_destroy.restype = None
    L.lp_batch_create.argtypes = [C.POINTER(P), I, C.c_size_t]
    L.lp_batch_add.argtypes = [P, C.POINTER(lp_request), C.POINTER(I)]
    L.lp_batch_autotune.argtypes = [P]
    L.lp_batch_solve.argtypes = [P]
    L.lp_batch_result.argtypes = [P, I, P, P, C.POINTER(lp_stats)]
    L.lp_batch_size.argtypes = [P]
    L.lp_batch_groups.argtypes = [P]
    L.lp_batch_error.argtypes = [P]
    L.lp_batch_error.restype = C.c_char_p
    L.lp_batch_destroy.argtypes = [P]
    L.lp_batch_destroy.restype = None
    for name in EXPORTS:
        if name not in ("lp_destroy", "lp_last_error", "lp_server_error", "lp_server_destroy", "lp_batch_error",
                        "lp_batch_destroy"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(ctx, status: int):
    if status != LP_OK:
        msg = load().lp_last_error(ctx).decode(errors="replace")
        raise LPError(status, msg)


# --------------------------------------------------------------------------- marshalling

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype=None):
    """(pointer, space, keepalive) for a NumPy array or a CUDA torch tensor."""
    if _is_torch(x):
        if not x.is_cuda:
            x = x.numpy()
        else:
            if not x.is_contiguous():
                raise ValueError("device tensors must be contiguous")
            return C.c_void_p(x.data_ptr()), LP_DEVICE, x
    a = np.ascontiguousarray(x, dtype=dtype)
    return C.c_void_p(a.ctypes.data), LP_HOST, a


def lp_create(device: int = 0, hbm_budget_bytes: int = 0, stream=None):
    """Open a context; returns an opaque handle (c_void_p)."""
    L = load()
    ctx = C.c_void_p()
    s = C.c_void_p(stream.cuda_stream) if stream is not None and hasattr(stream, "cuda_stream") else C.c_void_p(stream)
    _check(None, L.lp_create(C.byref(ctx), device, hbm_budget_bytes, s))
    return ctx


def lp_destroy(ctx) -> None:
    load().lp_destroy(ctx)


KERNELS = {"default": 0, "stream": 1, "pair": 2}


def lp_set_tuning(ctx, ring_units: int = 0, lag_units: int = 0, prefetch_units: int = 0, cache_hints: int = 0,
                  reset: bool = False, slice_cols: int = 0, kernel: str = "default",
                  test_stall_cycles: int = 0) -> None:
    """Tuning of the tensor-core step (zeros keep the defaults; reset=True passes NULL);
    kernel is "default", "stream" or "pair" (LP_KERNEL_*)."""
    L = load()
    if reset:
        _check(ctx, L.lp_set_tuning(ctx, None))
        return
    t = lp_tuning(ring_units, lag_units, prefetch_units, cache_hints, slice_cols, KERNELS[kernel], test_stall_cycles)
    _check(ctx, L.lp_set_tuning(ctx, C.byref(t)))


def lp_autotune(ctx, k: int) -> dict:
    """Time the step-kernel candidates for rank k and keep the fastest; returns the choice."""
    L = load()
    t = lp_tuning()
    path = C.c_int(0)
    ms = C.c_double(0.0)
    _check(ctx, L.lp_autotune(ctx, int(k), C.byref(t), C.byref(path), C.byref(ms)))
    return {"path": PATHS.get(path.value, path.value), "path_code": path.value, "ms_per_step": ms.value,
            "ring_units": t.ring_units, "lag_units": t.lag_units, "prefetch_units": t.prefetch_units,
            "cache_hints": t.cache_hints, "slice_cols": t.slice_cols,
            "kernel": {v: k for k, v in KERNELS.items()}.get(t.kernel, t.kernel)}


def lp_eta(ctx, m: int):
    """(eta of Def. 2, [||M_i - M||_2 for each i] + [||M||_2]) for the loaded partitions."""
    eta = np.zeros(1, dtype=np.float64)
    norms = np.empty(m + 1, dtype=np.float64)
    _check(ctx, load().lp_eta(ctx, eta.ctypes.data, norms.ctypes.data))
    return float(eta[0]), norms


def lp_trace(ctx, rounds: int, d: int, k: int):
    """(Z_t for every round as rounds x d x k, rho_t per round) of the last LP_FLAG_TRACE solve."""
    Z = np.empty((rounds, d, k), dtype=np.float64)
    rho = np.empty(rounds, dtype=np.float64)
    _check(ctx, load().lp_trace(ctx, Z.ctypes.data, rho.ctypes.data))
    return Z, rho


def lp_last_error(ctx=None) -> str:
    return load().lp_last_error(ctx).decode(errors="replace")


def lp_load_partitions(ctx, parts, dtype: str = "f32", row_scales=None) -> None:
    """parts: list of s_i x d arrays (float32, or uint16 BF16 bits, or uint8 E4M3
    codes) all on the host or all on the device; row_scales: list of float32
    arrays (E4M3 only)."""
    L = load()
    m = len(parts)
    np_dt = {"f32": np.float32, "bf16": np.uint16, "e4m3": np.uint8, "f32_bf16x2": np.float32}[dtype]
    ptrs, keep, spaces = [], [], set()
    for p in parts:
        q, sp, k = _ptr(p, np_dt)
        ptrs.append(q.value)
        keep.append(k)
        spaces.add(sp)
    if len(spaces) != 1:
        raise ValueError("partitions must all be host or all device")
    space = spaces.pop()
    rows = (C.c_int64 * m)(*[int(p.shape[0]) for p in parts])
    d = int(parts[0].shape[1])
    arr = (C.c_void_p * m)(*ptrs)
    sarr = None
    if row_scales is not None:
        sp_list = []
        for s in row_scales:
            q, sp, k = _ptr(s, np.float32)
            if sp != space:
                raise ValueError("row scales must live where the partitions do")
            sp_list.append(q.value)
            keep.append(k)
        sarr = (C.c_void_p * m)(*sp_list)
    _check(ctx, L.lp_load_partitions(ctx, m, rows, d, DTYPE[dtype], arr, sarr, space))


def lp_solve(ctx, k: int, p_schedule, agg: str, y0: np.ndarray, refine_rounds: int = 0, flags: int = 0) -> None:
    L = load()
    sched = np.ascontiguousarray(np.asarray(p_schedule, dtype=np.int32))
    T = int(sched.shape[0])
    y0c = np.ascontiguousarray(y0, dtype=np.float64)
    _check(ctx, L.lp_solve(ctx, int(k), sched.ctypes.data_as(C.POINTER(C.c_int)) if T else None, T, AGG[agg],
                           C.c_void_p(y0c.ctypes.data), int(refine_rounds), int(flags)))


def lp_solve_seeded(ctx, k: int, p_schedule, agg: str, seed: int, refine_rounds: int = 0, flags: int = 0) -> None:
    """lp_solve with Y_0 drawn by the library from `seed` (SplitMix64 + Box-Muller)."""
    L = load()
    sched = np.ascontiguousarray(np.asarray(p_schedule, dtype=np.int32))
    T = int(sched.shape[0])
    _check(ctx, L.lp_solve_seeded(ctx, int(k), sched.ctypes.data_as(C.POINTER(C.c_int)) if T else None, T, AGG[agg],
                                  C.c_uint64(int(seed)), int(refine_rounds), int(flags)))


def lp_result(ctx, d: int, k: int):
    """(Z d x k FP64, sigma k FP64, stats dict)."""
    L = load()
    Z = np.empty((d, k), dtype=np.float64)
    sig = np.empty(k, dtype=np.float64)
    st = lp_stats()
    status = L.lp_result(ctx, C.c_void_p(Z.ctypes.data), C.c_void_p(sig.ctypes.data), C.byref(st))
    _check(ctx, status)
    return Z, sig, st.as_dict()


def lp_power_step(ctx, k: int, z, z_shared: bool, m: int, d: int, out=None):
    """Y_i = M_i Z_i for every loaded partition; returns (m, d, k) FP64 (NumPy,
    or the given device tensor ``out``)."""
    L = load()
    zp, zsp, keep = _ptr(z, np.float64)
    if out is None:
        if zsp == LP_DEVICE:
            import torch
            out = torch.empty((m, d, k), dtype=torch.float64, device=z.device)
        else:
            out = np.empty((m, d, k), dtype=np.float64)
    yp, ysp, keep2 = _ptr(out, np.float64)
    if ysp != zsp:
        raise ValueError("z and out must share a pointer space")
    _check(ctx, L.lp_power_step(ctx, int(k), zp, 1 if z_shared else 0, yp, zsp))
    return out


def lp_orth(ctx, Y, kxk_fp64: bool = False):
    """Z_b = orth(Y_b) for a (batch, d, k) FP64 array (host) or tensor (device);
    kxk_fp64: the Gram and Cholesky in FP64 (LP_FLAG_KXK_FP64)."""
    L = load()
    b, d, k = Y.shape
    yp, sp, keep = _ptr(Y, np.float64)
    if sp == LP_DEVICE:
        import torch
        Z = torch.empty_like(Y)
    else:
        Z = np.empty((b, d, k), dtype=np.float64)
    zp, _, keep2 = _ptr(Z, np.float64)
    _check(ctx, L.lp_orth(ctx, int(b), int(d), int(k), yp, zp, sp, LP_FLAG_KXK_FP64 if kxk_fp64 else 0))
    return Z


def lp_align_aggregate(ctx, agg: str, base: int, w, Ys, Zs, kxk_fp64: bool = False):
    """(Y d x k, D (m, k, k)) for host FP64 inputs Ys, Zs of shape (m, d, k);
    kxk_fp64: the Procrustes SVD in FP64 (LP_FLAG_KXK_FP64)."""
    L = load()
    m, d, k = Ys.shape
    Ys = np.ascontiguousarray(Ys, dtype=np.float64)
    Zs = np.ascontiguousarray(Zs, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    Y = np.empty((d, k), dtype=np.float64)
    D = np.empty((m, k, k), dtype=np.float64)
    _check(ctx, L.lp_align_aggregate(ctx, int(m), int(d), int(k), AGG[agg], int(base), C.c_void_p(w.ctypes.data),
                                     C.c_void_p(Ys.ctypes.data), C.c_void_p(Zs.ctypes.data),
                                     C.c_void_p(Y.ctypes.data), C.c_void_p(D.ctypes.data), LP_HOST,
                                     LP_FLAG_KXK_FP64 if kxk_fp64 else 0))
    return Y, D


def lp_power_step_static(A, rows, k: int, z, y, stream=None) -> None:
    """The allocation-free power step: A (CUDA float32 tensor, partitions back to
    back), rows (the s_i), z (CUDA float64 d x k), y (CUDA float64 (m, d, k),
    written).  Asynchronous on ``stream`` (a torch stream or None)."""
    L = load()
    for t in (A, z, y):
        if not (_is_torch(t) and t.is_cuda and t.is_contiguous()):
            raise ValueError("A, z and y must be contiguous CUDA tensors")
    m = len(rows)
    r = (C.c_int64 * m)(*[int(x) for x in rows])
    s = C.c_void_p(stream.cuda_stream) if stream is not None else C.c_void_p(None)
    status = L.lp_power_step_static(C.c_void_p(A.data_ptr()), m, r, int(A.shape[1]), int(k),
                                    C.c_void_p(z.data_ptr()), C.c_void_p(y.data_ptr()), s)
    _check(None, status)


# --------------------------------------------------------------------------- convenience

class LocalPower:
    """A context with loaded partitions: ``LocalPower(parts).solve(k, schedule, agg, y0)``."""

    def __init__(self, parts, dtype: str = "f32", row_scales=None, device: int = 0, hbm_budget_bytes: int = 0,
                 stream=None):
        self.ctx = lp_create(device, hbm_budget_bytes, stream)
        try:
            lp_load_partitions(self.ctx, parts, dtype, row_scales)
        except Exception:
            lp_destroy(self.ctx)
            self.ctx = None
            raise
        self.m = len(parts)
        self.d = int(parts[0].shape[1])
        self.sizes = [int(p.shape[0]) for p in parts]

    def solve(self, k: int, schedule, agg: str, y0, refine_rounds: int = 0, ritz: bool = False, timing: bool = False,
              kxk_fp64: bool = False):
        flags = ((LP_FLAG_RITZ if ritz else 0) | (LP_FLAG_TIMING if timing else 0)
                 | (LP_FLAG_KXK_FP64 if kxk_fp64 else 0))
        lp_solve(self.ctx, k, schedule, agg, y0, refine_rounds, flags)
        return lp_result(self.ctx, self.d, k)

    def submit(self, k: int, schedule, agg: str, y0, refine_rounds: int = 0, ritz: bool = False, timing: bool = False,
               kxk_fp64: bool = False):
        flags = ((LP_FLAG_RITZ if ritz else 0) | (LP_FLAG_TIMING if timing else 0)
                 | (LP_FLAG_KXK_FP64 if kxk_fp64 else 0))
        lp_solve(self.ctx, k, schedule, agg, y0, refine_rounds, flags)

    def result(self, k: int):
        return lp_result(self.ctx, self.d, k)

    def power_step(self, k: int, z, shared: bool = True):
        return lp_power_step(self.ctx, k, z, shared, self.m, self.d)

    def eta(self):
        return lp_eta(self.ctx, self.m)

    def close(self) -> None:
        if self.ctx is not None:
            lp_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------- request server

class Server:
    """lp_server_*: continuous batching of independent solves.  Keeps each
    request's buffers alive until its result is fetched."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, max_active: int = 16):
        L = load()
        self.h = C.c_void_p()
        st = L.lp_server_create(C.byref(self.h), device, hbm_budget_bytes, max_active)
        if st != LP_OK:
            raise LPError(st, "lp_server_create failed")
        self._keep = {}
        self._shape = {}

    def _check(self, st):
        if st != LP_OK:
            raise LPError(st, load().lp_server_error(self.h).decode(errors="replace"))

    def submit(self, parts, k: int, p_schedule, agg: str, y0, dtype: str = "f32", row_scales=None,
               refine_rounds: int = 0, flags: int = LP_FLAG_RITZ, row_pitch: int = 0, d: int | None = None) -> int:
        """parts: host arrays or CUDA tensors (s_i x pitch); d defaults to the parts' width."""
        req, keep, dd = _make_request(parts, k, p_schedule, agg, y0, dtype, row_scales, refine_rounds, flags,
                                      row_pitch, d)
        rid = C.c_int64(0)
        self._check(load().lp_server_submit(self.h, C.byref(req), C.byref(rid)))
        self._keep[rid.value] = keep
        self._shape[rid.value] = (dd, int(k))
        return rid.value

    def progress(self, cap: int = 256) -> list[int]:
        ids = (C.c_int64 * cap)()
        n = C.c_int(0)
        self._check(load().lp_server_progress(self.h, ids, cap, C.byref(n)))
        return [ids[i] for i in range(n.value)]

    def result(self, rid: int):
        d, k = self._shape.get(rid, (1, 1))   # unknown ids: the library reports LP_ERR_STATE
        Z = np.empty((d, k), dtype=np.float64)
        sig = np.empty(k, dtype=np.float64)
        st = lp_stats()
        code = load().lp_server_result(self.h, rid, Z.ctypes.data, sig.ctypes.data, C.byref(st))
        self._keep.pop(rid, None)
        self._shape.pop(rid, None)
        self._check(code)
        return Z, sig, st.as_dict()

    def query(self) -> dict:
        info = lp_server_info()
        self._check(load().lp_server_query(self.h, C.byref(info)))
        return {f: getattr(info, f) for f, _ in info._fields_}

    def close(self):
        if self.h:
            load().lp_server_destroy(self.h)
            self.h = C.c_void_p()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _make_request(parts, k, p_schedule, agg, y0, dtype, row_scales, refine_rounds, flags, row_pitch, d):
    """An lp_request for the server or the batch runner, and the objects that must outlive it."""
    np_dt = {"f32": np.float32, "bf16": np.uint16, "e4m3": np.uint8, "f32_bf16x2": np.float32}[dtype]
    m = len(parts)
    keep, ptrs, spaces = [], [], set()
    for p in parts:
        q, sp, kk = _ptr(p, np_dt)
        ptrs.append(q.value)
        keep.append(kk)
        spaces.add(sp)
    if len(spaces) != 1:
        raise ValueError("partitions must all be host or all device")
    dd = int(d if d is not None else parts[0].shape[1])
    rows = (C.c_int64 * m)(*[int(p.shape[0]) for p in parts])
    parr = (C.c_void_p * m)(*ptrs)
    sarr = None
    if row_scales is not None:
        sl = []
        for sc in row_scales:
            q, _, kk = _ptr(sc, np.float32)
            sl.append(q.value)
            keep.append(kk)
        sarr = (C.c_void_p * m)(*sl)
    sched = np.ascontiguousarray(np.asarray(p_schedule, dtype=np.int32))
    y0c = np.ascontiguousarray(y0, dtype=np.float64)
    req = lp_request(m, rows, dd, int(row_pitch), DTYPE[dtype], parr, sarr, spaces.pop(), int(k),
                     sched.ctypes.data_as(C.POINTER(C.c_int)), len(sched), AGG[agg],
                     y0c.ctypes.data_as(C.POINTER(C.c_double)), int(refine_rounds), int(flags))
    keep += [rows, parr, sarr, sched, y0c]
    return req, keep, dd


class Batch:
    """lp_batch_*: independent instances solved by one graph launch."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.h = C.c_void_p()
        st = load().lp_batch_create(C.byref(self.h), device, hbm_budget_bytes)
        if st != LP_OK:
            raise LPError(st, "lp_batch_create failed")
        self._shape = []

    def _check(self, st):
        if st != LP_OK:
            raise LPError(st, load().lp_batch_error(self.h).decode(errors="replace"))

    def add(self, parts, k: int, p_schedule, agg: str, y0, dtype: str = "f32", row_scales=None,
            refine_rounds: int = 0, flags: int = LP_FLAG_RITZ, row_pitch: int = 0, d: int | None = None) -> int:
        req, keep, dd = _make_request(parts, k, p_schedule, agg, y0, dtype, row_scales, refine_rounds, flags,
                                      row_pitch, d)
        idx = C.c_int(0)
        self._check(load().lp_batch_add(self.h, C.byref(req), C.byref(idx)))
        self._shape.append((dd, int(k)))
        return idx.value

    def autotune(self):
        self._check(load().lp_batch_autotune(self.h))

    def solve(self):
        self._check(load().lp_batch_solve(self.h))

    def result(self, i: int):
        d, k = self._shape[i]
        Z = np.empty((d, k), dtype=np.float64)
        sig = np.empty(k, dtype=np.float64)
        st = lp_stats()
        self._check(load().lp_batch_result(self.h, i, Z.ctypes.data, sig.ctypes.data, C.byref(st)))
        return Z, sig, st.as_dict()

    def __len__(self):
        return int(load().lp_batch_size(self.h))

    def groups(self) -> int:
        """Groups the instances form (instances sharing d, dtype, k, schedule,
        aggregator and flags; 0 until the next solve or autotune)."""
        return int(load().lp_batch_groups(self.h))

    def close(self):
        if self.h:
            load().lp_batch_destroy(self.h)
            self.h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
