"""Python binding of libgofmm (include/gofmm.h): argument marshalling only.

Every function has the name of the C entry point it calls, without the
``gofmm_`` prefix.  Device buffers are torch tensors (PyTorch supplies device
memory and streams); host buffers are numpy arrays.  Nothing here computes:
if the native library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Callable, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libgofmm.so")

OK = 0
ERR_ARG, ERR_CALLBACK, ERR_NONFINITE, ERR_NOMEM = -1, -2, -3, -4
ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_IO = -5, -6, -7, -8
GEN_CALLBACK, GEN_GAUSSIAN, GEN_IMQ = 0, 1, 2
DIST_GRAM_L2, DIST_ANGLE, DIST_LEXICOGRAPHIC, DIST_RANDOM = 0, 1, 2, 3
FAR_SYMMETRIC, FAR_PAPER = 0, 1
CACHE_BLOCKS, CACHE_NONE = 0, 1
DTYPE_F64, DTYPE_F32 = 0, 1
PREC_FP64, PREC_FP32, PREC_TF32, PREC_BF16, PREC_BF16X3 = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": PREC_FP64, "fp32": PREC_FP32, "tf32": PREC_TF32, "bf16": PREC_BF16,
              "bf16x3": PREC_BF16X3}
SCHED_FUSED, SCHED_STAGED, SCHED_PAIR, SCHED_HYBRID = 0, 1, 2, 3
ORDER_CRITICAL, ORDER_LOCAL, ORDER_SCHEDULE, ORDER_READY, ORDER_LEVELS = 0, 1, 2, 3, 4

BLOCK_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(C.c_int64), C.c_int64,
                       C.POINTER(C.c_int64), C.c_int64, C.POINTER(C.c_double))


class EntriesC(C.Structure):
    _fields_ = [("kind", C.c_int), ("dim", C.c_int), ("n", C.c_int64),
                ("points", C.POINTER(C.c_double)), ("bandwidth", C.c_double),
                ("diag_shift", C.c_double), ("fn", BLOCK_FN), ("ctx", C.c_void_p)]


class ParamsC(C.Structure):
    _fields_ = [("leaf_size", C.c_int64), ("max_rank", C.c_int64), ("tau", C.c_double),
                ("budget", C.c_double), ("kappa", C.c_int), ("distance", C.c_int),
                ("far_mode", C.c_int), ("cache_mode", C.c_int), ("n_centroid", C.c_int),
                ("n_sample", C.c_int), ("ann_max_iter", C.c_int), ("num_threads", C.c_int),
                ("ann_target_recall", C.c_double), ("knn_exact_max", C.c_int64),
                ("seed", C.c_uint64), ("device", C.c_int), ("sample_device", C.c_int)]


class TuneC(C.Structure):
    _fields_ = [("piece", C.c_int), ("schedule", C.c_int), ("order", C.c_int), ("from_cache", C.c_int),
                ("n_candidates", C.c_int), ("cand_piece", C.c_int * 16), ("cand_schedule", C.c_int * 16),
                ("cand_order", C.c_int * 16), ("cand_ms", C.c_float * 16), ("key", C.c_char * 32)]


class StatsC(C.Structure):
    _fields_ = [("n", C.c_int64), ("depth", C.c_int64), ("n_leaves", C.c_int64),
                ("min_rank", C.c_int64), ("max_rank", C.c_int64), ("mean_rank", C.c_double),
                ("near_pairs", C.c_int64), ("far_pairs", C.c_int64), ("max_near", C.c_int64),
                ("flops_n2s", C.c_double), ("flops_s2s", C.c_double), ("flops_s2n", C.c_double),
                ("flops_l2l", C.c_double), ("near_entries", C.c_int64), ("far_entries", C.c_int64),
                ("interp_entries", C.c_int64), ("skel_total", C.c_int64),
                ("ann_iterations", C.c_int), ("ann_recall", C.c_double),
                ("compress_seconds", C.c_double), ("interp_t_entries", C.c_int64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"native library not built: {LIB_PATH} "
                          "(run python paper_1707_00164_b300/build.py)")
    lib = C.CDLL(LIB_PATH)
    H = C.c_void_p
    sig = {
        "gofmm_default_params": (None, [C.POINTER(ParamsC)]),
        "gofmm_compress": (C.c_int, [C.POINTER(EntriesC), C.POINTER(ParamsC), C.POINTER(H)]),
        "gofmm_prepare": (C.c_int, [H, C.c_int64, C.c_int]),
        "gofmm_evaluate": (C.c_int, [H, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int64,
                                     C.c_int, C.c_int, C.c_void_p]),
        "gofmm_evaluate_host": (C.c_int, [H, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                          C.c_int64, C.c_int, C.c_int, C.c_void_p]),
        "gofmm_evaluate_host_async": (C.c_int, [H, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                                C.c_int64, C.c_int, C.c_int, C.c_void_p]),
        "gofmm_evaluate_static": (C.c_int, [H, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                            C.c_int64, C.c_int, C.c_int, C.c_void_p]),
        "gofmm_synchronize": (C.c_int, [H, C.c_void_p]),
        "gofmm_trim": (C.c_int, [H]),
        "gofmm_debug_stall_next": (C.c_int, [H, C.c_int]),
        "gofmm_engine_create": (C.c_int, [C.c_int, C.c_int, C.c_int64, C.POINTER(H)]),
        "gofmm_engine_submit": (C.c_int, [H, H, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int64,
                                          C.POINTER(C.c_int64)]),
        "gofmm_engine_step": (C.c_int, [H, C.c_void_p, C.POINTER(C.c_int64)]),
        "gofmm_engine_poll": (C.c_int, [H, C.c_int64, C.POINTER(C.c_int)]),
        "gofmm_engine_workspace": (C.c_int, [H, H, C.c_int64, C.POINTER(C.c_int64)]),
        "gofmm_engine_drain": (C.c_int, [H, C.c_void_p]),
        "gofmm_engine_stats": (C.c_int, [H, C.POINTER(C.c_int64), C.c_int]),
        "gofmm_engine_free": (C.c_int, [H]),
        "gofmm_batch_create": (C.c_int, [C.POINTER(H), C.POINTER(C.c_int64), C.c_int, C.c_int, C.POINTER(H)]),
        "gofmm_batch_evaluate": (C.c_int, [H, C.POINTER(C.c_void_p), C.POINTER(C.c_int64), C.POINTER(C.c_void_p),
                                           C.POINTER(C.c_int64), C.c_void_p]),
        "gofmm_batch_info": (C.c_int, [H, C.POINTER(C.c_int64), C.c_int]),
        "gofmm_batch_free": (C.c_int, [H]),
        "gofmm_free": (C.c_int, [H]),
        "gofmm_export": (C.c_int, [H, C.c_char_p]),
        "gofmm_import": (C.c_int, [C.c_char_p, C.POINTER(EntriesC), C.c_int, C.c_int, C.POINTER(H)]),
        "gofmm_stats": (C.c_int, [H, C.POINTER(StatsC)]),
        "gofmm_set_timing": (C.c_int, [H, C.c_int]),
        "gofmm_stage_times": (C.c_int, [H, C.POINTER(C.c_float), C.c_int]),
        "gofmm_view": (C.c_int64, [H, C.c_int, C.c_void_p]),
        "gofmm_set_tc_config": (C.c_int, [H, C.c_int, C.c_int, C.c_int, C.c_int]),
        "gofmm_get_tc_config": (C.c_int, [H, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                          C.POINTER(C.c_int)]),
        "gofmm_autotune": (C.c_int, [H, C.c_int64, C.c_int, C.c_char_p, C.c_void_p, C.POINTER(TuneC)]),
        "gofmm_autotune_batch": (C.c_int, [C.POINTER(H), C.POINTER(C.c_int64), C.c_int, C.c_int, C.c_char_p,
                                           C.c_void_p, C.POINTER(TuneC)]),
        "gofmm_autotune_key": (C.c_int, [C.POINTER(H), C.POINTER(C.c_int64), C.c_int, C.c_int, C.c_char_p]),
        "gofmm_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


LIB = _load()


class GofmmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libgofmm error {code}: {msg}")
        self.code = code


def last_error() -> str:
    return LIB.gofmm_last_error().decode()


def _check(rc: int):
    if rc != OK:
        raise GofmmError(rc, last_error())


class Entries:
    """gofmm_entries: a generator (points kept alive here) or a callback
    ``fn(I, J) -> ndarray`` returning the nI x nJ block K(I, J)."""

    def __init__(self, kind: int, n: int, points: Optional[np.ndarray] = None,
                 bandwidth: float = 1.0, shift: float = 0.0, fn: Optional[Callable] = None):
        self.kind, self.n = kind, int(n)
        self.points = None if points is None else np.ascontiguousarray(points, dtype=np.float64)
        self.bandwidth, self.shift, self.fn = float(bandwidth), float(shift), fn
        self._cb = None

    @staticmethod
    def gaussian(points, h, shift):
        return Entries(GEN_GAUSSIAN, len(points), points, h, shift)

    @staticmethod
    def imq(points, l, shift):
        return Entries(GEN_IMQ, len(points), points, l, shift)

    @staticmethod
    def callback(n, fn):
        return Entries(GEN_CALLBACK, n, fn=fn)

    def c(self) -> EntriesC:
        e = EntriesC()
        e.kind, e.n = self.kind, self.n
        e.bandwidth, e.diag_shift = self.bandwidth, self.shift
        if self.points is not None:
            e.dim = self.points.shape[1]
            e.points = self.points.ctypes.data_as(C.POINTER(C.c_double))
        if self.fn is not None:
            user = self.fn

            def tramp(ctx, I, nI, J, nJ, out):
                try:
                    Ia = np.ctypeslib.as_array(I, shape=(nI,)).copy()
                    Ja = np.ctypeslib.as_array(J, shape=(nJ,)).copy()
                    blk = np.asarray(user(Ia, Ja), dtype=np.float64)
                    np.ctypeslib.as_array(out, shape=(nI, nJ))[...] = blk
                    return 0
                except Exception:  # reported to the library as a failing callback
                    return 1

            self._cb = BLOCK_FN(tramp)
            e.fn = self._cb
        return e


def default_params(**over) -> ParamsC:
    p = ParamsC()
    LIB.gofmm_default_params(C.byref(p))
    for k, v in over.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


class Handle:
    def __init__(self, ptr: C.c_void_p):
        self.ptr = ptr

    def __del__(self):
        if getattr(self, "ptr", None):
            LIB.gofmm_free(self.ptr)
            self.ptr = None


def compress(entries: Entries, params: Optional[ParamsC] = None) -> Handle:
    e = entries.c()
    out = C.c_void_p()
    _check(LIB.gofmm_compress(C.byref(e), C.byref(params) if params is not None else None,
                              C.byref(out)))
    return Handle(out)


def prepare(h: Handle, r_max: int, precision: int):
    _check(LIB.gofmm_prepare(h.ptr, int(r_max), int(precision)))


def _dtype_code(t) -> int:
    name = str(t.dtype)
    if name in ("torch.float64", "float64"):
        return DTYPE_F64
    if name in ("torch.float32", "float32"):
        return DTYPE_F32
    raise TypeError(f"unsupported dtype {t.dtype}")


def evaluate(h: Handle, W, U, precision: int, stream=None):
    """U = K~ W for torch CUDA tensors (N x r, unit column stride) on
    `stream` (a torch.cuda.Stream; default: the current stream)."""
    import torch
    if W.dim() != 2 or U.dim() != 2 or W.stride(1) != 1 or U.stride(1) != 1:
        raise ValueError("W and U must be 2-D with unit column stride")
    if not (W.is_cuda and U.is_cuda):
        raise ValueError("W and U must be CUDA tensors (use evaluate_host for host buffers)")
    if W.shape != U.shape or W.dtype != U.dtype:
        raise ValueError("W and U must have the same shape and dtype")
    s = stream if stream is not None else torch.cuda.current_stream(W.device)
    _check(LIB.gofmm_evaluate(h.ptr, C.c_void_p(W.data_ptr()), W.stride(0), C.c_void_p(U.data_ptr()),
                              U.stride(0), W.shape[1], _dtype_code(W), int(precision),
                              C.c_void_p(s.cuda_stream)))


def evaluate_static(h: Handle, W, U, precision: int, stream=None):
    """gofmm_evaluate_static: as evaluate, for FP64/FP32, with the scratch in
    the library's fixed device array (no allocation; handle prepared
    beforehand)."""
    import torch
    if W.dim() != 2 or U.dim() != 2 or W.stride(1) != 1 or U.stride(1) != 1:
        raise ValueError("W and U must be 2-D with unit column stride")
    if W.shape != U.shape or W.dtype != U.dtype:
        raise ValueError("W and U must have the same shape and dtype")
    s = stream if stream is not None else torch.cuda.current_stream(W.device)
    _check(LIB.gofmm_evaluate_static(h.ptr, C.c_void_p(W.data_ptr()), W.stride(0),
                                     C.c_void_p(U.data_ptr()), U.stride(0), W.shape[1],
                                     _dtype_code(W), int(precision), C.c_void_p(s.cuda_stream)))


def _host_args(W: np.ndarray, U: np.ndarray):
    if W.ndim != 2 or W.shape != U.shape or W.dtype != U.dtype:
        raise ValueError("W and U must be 2-D arrays of one shape and dtype")
    if W.strides[1] != W.itemsize or U.strides[1] != U.itemsize:
        raise ValueError("W and U need unit column stride")
    return (C.c_void_p(W.ctypes.data), W.strides[0] // W.itemsize, C.c_void_p(U.ctypes.data),
            U.strides[0] // U.itemsize, W.shape[1], _dtype_code(W))


def evaluate_host(h: Handle, W: np.ndarray, U: np.ndarray, precision: int, stream=None):
    """As evaluate, with host numpy arrays (C-contiguous rows); blocks until
    U holds the result."""
    sp = None if stream is None else C.c_void_p(stream.cuda_stream)
    _check(LIB.gofmm_evaluate_host(h.ptr, *_host_args(W, U), int(precision), sp))


def evaluate_host_async(h: Handle, W: np.ndarray, U: np.ndarray, precision: int, stream=None):
    """As evaluate_host, but returns once the work is enqueued: U is final
    (and W may change) after synchronize(h, stream).  W and U must stay
    alive until then; pinned memory lets the copies overlap other calls."""
    sp = None if stream is None else C.c_void_p(stream.cuda_stream)
    _check(LIB.gofmm_evaluate_host_async(h.ptr, *_host_args(W, U), int(precision), sp))


def debug_stall_next(h: Handle, precision: int):
    """gofmm_debug_stall_next: the next evaluation waits on a count nothing
    reaches (tests the bounded-wait error path)."""
    _check(LIB.gofmm_debug_stall_next(h.ptr, int(precision)))


def trim(h: Handle):
    """gofmm_trim: drop device stores only the CUDA-core precisions use."""
    _check(LIB.gofmm_trim(h.ptr))


def synchronize(h: Handle, stream=None):
    """Wait for the stream; raise on errors the kernels recorded (bounded
    waits that gave up: ERR_TIMEOUT)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(LIB.gofmm_synchronize(h.ptr, C.c_void_p(s.cuda_stream)))


def free(h: Handle):
    if h.ptr:
        rc = LIB.gofmm_free(h.ptr)
        if rc == OK:  # refused (requests in flight): the handle stays valid
            h.ptr = None
        _check(rc)


def export(h: Handle, path: str):
    _check(LIB.gofmm_export(h.ptr, path.encode()))


def import_(path: str, entries: Entries, cache_mode: int = CACHE_BLOCKS, device: int = 0) -> Handle:
    e = entries.c()
    out = C.c_void_p()
    _check(LIB.gofmm_import(path.encode(), C.byref(e), int(cache_mode), int(device), C.byref(out)))
    return Handle(out)


def stats(h: Handle) -> dict:
    s = StatsC()
    _check(LIB.gofmm_stats(h.ptr, C.byref(s)))
    return {name: getattr(s, name) for name, _ in StatsC._fields_}


def set_tc_config(h: Handle, precision: int, piece: int = 256, schedule: int = SCHED_FUSED,
                  order: int = ORDER_CRITICAL):
    _check(LIB.gofmm_set_tc_config(h.ptr, int(precision), int(piece), int(schedule), int(order)))


def get_tc_config(h: Handle, precision: int) -> dict:
    p, s, o = C.c_int(), C.c_int(), C.c_int()
    _check(LIB.gofmm_get_tc_config(h.ptr, int(precision), C.byref(p), C.byref(s), C.byref(o)))
    return dict(piece=p.value, schedule=s.value, order=o.value)


def _tune_dict(t: TuneC) -> dict:
    n = t.n_candidates
    return dict(piece=t.piece, schedule=t.schedule, order=t.order, from_cache=bool(t.from_cache),
                key=t.key.decode(),
                candidates=[dict(piece=t.cand_piece[k], schedule=t.cand_schedule[k], order=t.cand_order[k],
                                 ms=t.cand_ms[k]) for k in range(n)])


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return C.c_void_p(None)
    return C.c_void_p(stream.cuda_stream)


def autotune(h: Handle, r: int, precision: int, cache_path: Optional[str] = None, stream=None) -> dict:
    t = TuneC()
    path = cache_path.encode() if cache_path else None
    _check(LIB.gofmm_autotune(h.ptr, int(r), int(precision), path, _stream_ptr(stream), C.byref(t)))
    return _tune_dict(t)


def _handle_array(handles):
    return (C.c_void_p * len(handles))(*[h.ptr.value if isinstance(h.ptr, C.c_void_p) else h.ptr
                                         for h in handles])


def autotune_batch(handles, rs, precision: int, cache_path: Optional[str] = None, stream=None) -> dict:
    t = TuneC()
    r = (C.c_int64 * len(handles))(*[int(x) for x in rs])
    path = cache_path.encode() if cache_path else None
    _check(LIB.gofmm_autotune_batch(_handle_array(handles), r, len(handles), int(precision), path,
                                    _stream_ptr(stream), C.byref(t)))
    return _tune_dict(t)


def autotune_key(handles, rs, precision: int) -> str:
    buf = C.create_string_buffer(32)
    r = (C.c_int64 * len(handles))(*[int(x) for x in rs])
    _check(LIB.gofmm_autotune_key(_handle_array(handles), r, len(handles), int(precision), buf))
    return buf.value.decode()


def set_timing(h: Handle, enable: bool):
    _check(LIB.gofmm_set_timing(h.ptr, int(enable)))


def stage_times(h: Handle) -> dict:
    ms = (C.c_float * 7)()
    _check(LIB.gofmm_stage_times(h.ptr, ms, 7))
    return dict(gather=ms[0], upward=ms[1], s2s=ms[2], s2n=ms[3], leaf=ms[4], total=ms[5],
                launches=int(ms[6]))


def view(h: Handle, what: int) -> np.ndarray:
    n = LIB.gofmm_view(h.ptr, what, None)
    if n < 0:
        raise GofmmError(int(n), last_error())
    out = np.empty(n, dtype=np.float64 if what == 5 else np.int64)
    LIB.gofmm_view(h.ptr, what, C.c_void_p(out.ctypes.data))
    return out


def structure(h: Handle) -> dict:
    """Tree order, near/far lists, skeletons and interpolation matrices as
    Python objects (heap numbering: root 0, children 2h+1, 2h+2)."""
    st = stats(h)
    L = st["depth"]
    nn = (2 << L) - 1
    nl = 1 << L

    def csr(arr, count):
        off = arr[:count + 1]
        vals = arr[count + 1:]
        return [vals[off[i]:off[i + 1]] for i in range(count)]

    perm = view(h, 0)
    leaf_off = view(h, 1)
    near = csr(view(h, 2), nl)
    far = csr(view(h, 3), nn)
    skel = csr(view(h, 4), nn)
    pvals = view(h, 5)
    P, pos = {}, 0
    first_leaf = nl - 1
    for node in range(1, nn):
        s = skel[node].size
        nc = (leaf_off[node - first_leaf + 1] - leaf_off[node - first_leaf]) if node >= first_leaf \
            else skel[2 * node + 1].size + skel[2 * node + 2].size
        P[node] = pvals[pos:pos + s * nc].reshape(s, nc)
        pos += s * nc
    return dict(depth=L, perm=perm, leaf_off=leaf_off, near=near, far=far, skel=skel, P=P)


class Engine:
    """gofmm_engine: many evaluations in flight, one grouped launch per step."""

    QUEUED, RUNNING, DONE = 0, 1, 2

    def __init__(self, precision: int, pool_bytes: int, device: int = 0):
        self.ptr = C.c_void_p()
        _check(LIB.gofmm_engine_create(int(device), int(precision), int(pool_bytes), C.byref(self.ptr)))
        self._keep = {}

    def submit(self, h: Handle, W, U) -> int:
        """Queue U = K~ W (torch CUDA float32 tensors, N x r); both must stay
        alive until the request is done."""
        if W.stride(1) != 1 or U.stride(1) != 1 or W.shape != U.shape:
            raise ValueError("W and U: same shape, unit column stride")
        rid = C.c_int64()
        _check(LIB.gofmm_engine_submit(self.ptr, h.ptr, C.c_void_p(W.data_ptr()), W.stride(0),
                                       C.c_void_p(U.data_ptr()), U.stride(0), W.shape[1], C.byref(rid)))
        self._keep[rid.value] = (h, W, U)
        return rid.value

    def workspace(self, h: Handle, r: int) -> int:
        """Pool bytes one request of h with r right-hand sides takes."""
        b = C.c_int64()
        _check(LIB.gofmm_engine_workspace(self.ptr, h.ptr, int(r), C.byref(b)))
        return b.value

    def step(self, stream=None) -> int:
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        n = C.c_int64()
        _check(LIB.gofmm_engine_step(self.ptr, C.c_void_p(s.cuda_stream), C.byref(n)))
        return n.value

    def poll(self, rid: int) -> int:
        st = C.c_int()
        _check(LIB.gofmm_engine_poll(self.ptr, int(rid), C.byref(st)))
        if st.value == self.DONE:
            self._keep.pop(rid, None)
        return st.value

    def drain(self, stream=None):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(LIB.gofmm_engine_drain(self.ptr, C.c_void_p(s.cuda_stream)))
        self._keep.clear()

    def stats(self) -> dict:
        out = (C.c_int64 * 7)()
        _check(LIB.gofmm_engine_stats(self.ptr, out, 7))
        return dict(steps=out[0], launches=out[1], max_active=out[2], completed=out[3], queued=out[4],
                    running=out[5], finishing=out[6])

    def free(self):
        if self.ptr:
            rc = LIB.gofmm_engine_free(self.ptr)
            self.ptr = None
            _check(rc)

    def __del__(self):
        if getattr(self, "ptr", None):
            LIB.gofmm_engine_free(self.ptr)
            self.ptr = None


class Batch:
    """gofmm_batch: a fixed list of evaluations run as one merged step sequence."""

    def __init__(self, handles, rs, precision: int):
        n = len(handles)
        hs = (C.c_void_p * n)(*[h.ptr.value if isinstance(h.ptr, C.c_void_p) else h.ptr for h in handles])
        r = (C.c_int64 * n)(*[int(x) for x in rs])
        self.ptr = C.c_void_p()
        _check(LIB.gofmm_batch_create(hs, r, n, int(precision), C.byref(self.ptr)))
        self.handles = list(handles)
        self.n = n

    def evaluate(self, Ws, Us, stream=None):
        import torch
        n = self.n
        W = (C.c_void_p * n)(*[w.data_ptr() for w in Ws])
        U = (C.c_void_p * n)(*[u.data_ptr() for u in Us])
        lw = (C.c_int64 * n)(*[w.stride(0) for w in Ws])
        lu = (C.c_int64 * n)(*[u.stride(0) for u in Us])
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(LIB.gofmm_batch_evaluate(self.ptr, W, lw, U, lu, C.c_void_p(s.cuda_stream)))

    def info(self) -> dict:
        out = (C.c_int64 * 2)()
        _check(LIB.gofmm_batch_info(self.ptr, out, 2))
        return dict(launches=out[0], error=out[1])

    def free(self):
        if self.ptr:
            rc = LIB.gofmm_batch_free(self.ptr)
            self.ptr = None
            _check(rc)

    def __del__(self):
        if getattr(self, "ptr", None):
            LIB.gofmm_batch_free(self.ptr)
            self.ptr = None
