"""Python binding of libbmm.so: argument marshalling only.

Every step of every product runs in the CUDA kernels behind the C ABI
(include/bmm.h). There is no CPU fallback: if the library is missing, the
import of any compute call raises.

Matrices are contiguous torch tensors of dtype int64 on the current CUDA
device holding the packed uint64 words (row-major, bit j of row i is bit
j % 64 of word i*(cols/64) + j/64).
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbmm.so")

OK, ERR_INVALID, ERR_ALIGN, ERR_NOMEM, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED = range(7)
PATH_AUTO, PATH_TC_FP8, PATH_TC_I8, PATH_POPC, PATH_TC_FP8_PAIR, PATH_TC_FP4_PAIR = 0, 1, 2, 3, 4, 5
TENSOR_PATHS = (PATH_TC_FP8, PATH_TC_FP8_PAIR, PATH_TC_FP4_PAIR)
WINOGRAD, SELF_INVERSE, CHAINING = 0, 1, 2
GF2, BOOL = 0, 1

EXPORTED = [
    "bmm_opts_default", "bmm_gf2", "bmm_bool", "bmm_gf2_ex", "bmm_bool_ex", "bmm_workspace_size",
    "bmm_gf2_batched", "bmm_bool_batched", "bmm_batched", "bmm_batched_plan_create",
    "bmm_batched_plan_run", "bmm_batched_plan_destroy", "bmm_transpose", "bmm_base_product",
    "bmm_basis_change", "bmm_stream_status", "bmm_status_string", "bmm_last_cuda_error",
    "bmm_device_supported", "bmm_plan", "bmm_product_noalloc", "bmm_selftest_wait_timeout",
    "bmm_trace_enable", "bmm_trace_read", "bmm_launch_count", "bmm_autotune",
    "bmm_autotune_clear", "bmm_batched_plan_path", "bmm_batched_plan_create_ex",
    "bmm_host_opts_default", "bmm_host_plan", "bmm_gf2_host", "bmm_bool_host",
    "bmm_host_release", "bmm_batched_plan_create_paths", "bmm_batched_plan_choice",
    "bmm_batched_plan_stats", "bmm_batched_model",
]
TUNE_MODEL = 1
PHASE_BASE, PHASE_XOR, PHASE_TRANSPOSE = 0, 1, 2


class BmmError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        name = _lib_handle().bmm_status_string(status).decode() if _LIB else str(status)
        extra = ""
        if status == ERR_CUDA and _LIB:
            extra = f" (cudaError {_LIB.bmm_last_cuda_error()})"
        super().__init__(f"{what}: {name}{extra}")


class Opts(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("strassen_depth", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("serial_depth", ctypes.c_int32),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_uint64),
                ("kernel_level", ctypes.c_int32)]


class TuneResult(ctypes.Structure):
    _fields_ = [("best", Opts), ("est_ms", ctypes.c_double), ("measured", ctypes.c_int32),
                ("candidates", ctypes.c_int32)]


class HostOpts(ctypes.Structure):
    _fields_ = [("device", Opts), ("device_bytes", ctypes.c_uint64),
                ("host_depth", ctypes.c_int32), ("threads", ctypes.c_int32)]


class HostPlanInfo(ctypes.Structure):
    _fields_ = [("host_depth", ctypes.c_int32), ("sub_m", ctypes.c_int64),
                ("sub_k", ctypes.c_int64), ("sub_n", ctypes.c_int64), ("count", ctypes.c_int64),
                ("device_bytes", ctypes.c_uint64), ("staging_bytes", ctypes.c_uint64),
                ("upload_bytes", ctypes.c_uint64), ("download_bytes", ctypes.c_uint64)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("strassen_depth", ctypes.c_int32),
                ("serial_depth", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("leaves", ctypes.c_int64), ("workspace_bytes", ctypes.c_uint64),
                ("kernel_level", ctypes.c_int32), ("kp", ctypes.c_int64),
                ("pass_bytes", ctypes.c_uint64)]


class BatchedChoice(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("tile_m", ctypes.c_int32), ("tile_n", ctypes.c_int32),
                ("tail_n", ctypes.c_int32), ("k_step", ctypes.c_int32),
                ("k_steps", ctypes.c_int64), ("strassen_depth", ctypes.c_int32),
                ("est_us", ctypes.c_double)]


class BatchedStats(ctypes.Structure):
    _fields_ = [("problems", ctypes.c_int32), ("tensor_problems", ctypes.c_int32),
                ("popc_problems", ctypes.c_int32), ("tensor_path", ctypes.c_int32),
                ("tensor_tiles", ctypes.c_int64), ("tensor_tiles_n128", ctypes.c_int64),
                ("popc_tiles", ctypes.c_int64), ("macs_needed", ctypes.c_double),
                ("macs_issued", ctypes.c_double), ("est_ms", ctypes.c_double),
                ("model_measured", ctypes.c_int32), ("strassen_problems", ctypes.c_int32)]


class BatchedModel(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("measured", ctypes.c_int32),
                ("tensor_units", ctypes.c_int32), ("tensor_stage_ns", ctypes.c_double),
                ("tensor_stage_n128_ns", ctypes.c_double), ("tensor_tile_ns", ctypes.c_double),
                ("popc_units", ctypes.c_int32), ("popc_stage_ns", ctypes.c_double),
                ("popc_tile_ns", ctypes.c_double)]


_LIB = None


def _lib_handle():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        L.bmm_opts_default.argtypes = [ctypes.POINTER(Opts)]
        L.bmm_opts_default.restype = None
        for f in (L.bmm_gf2, L.bmm_bool):
            f.argtypes = [vp, vp, vp, i64, i64, i64, vp]
            f.restype = i32
        for f in (L.bmm_gf2_ex, L.bmm_bool_ex):
            f.argtypes = [vp, vp, vp, i64, i64, i64, ctypes.POINTER(Opts), vp]
            f.restype = i32
        L.bmm_workspace_size.argtypes = [i32, i64, i64, i64, ctypes.POINTER(Opts),
                                         ctypes.POINTER(ctypes.c_uint64)]
        L.bmm_workspace_size.restype = i32
        for f in (L.bmm_gf2_batched, L.bmm_bool_batched):
            f.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp]
            f.restype = i32
        L.bmm_batched.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp]
        L.bmm_batched.restype = i32
        L.bmm_batched_plan_create.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp,
                                              ctypes.POINTER(ctypes.c_void_p)]
        L.bmm_batched_plan_create.restype = i32
        L.bmm_batched_plan_create_ex.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, i32,
                                                 ctypes.POINTER(ctypes.c_void_p)]
        L.bmm_batched_plan_create_ex.restype = i32
        L.bmm_batched_plan_run.argtypes = [vp, vp]
        L.bmm_batched_plan_run.restype = i32
        L.bmm_batched_plan_destroy.argtypes = [vp]
        L.bmm_batched_plan_destroy.restype = i32
        L.bmm_batched_plan_path.argtypes = [vp, ctypes.POINTER(i32)]
        L.bmm_batched_plan_path.restype = i32
        L.bmm_batched_plan_create_paths.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp,
                                                    ctypes.POINTER(ctypes.c_void_p)]
        L.bmm_batched_plan_create_paths.restype = i32
        L.bmm_batched_plan_choice.argtypes = [vp, i32, ctypes.POINTER(BatchedChoice)]
        L.bmm_batched_plan_choice.restype = i32
        L.bmm_batched_plan_stats.argtypes = [vp, ctypes.POINTER(BatchedStats)]
        L.bmm_batched_plan_stats.restype = i32
        L.bmm_batched_model.argtypes = [i32, ctypes.POINTER(BatchedModel)]
        L.bmm_batched_model.restype = i32
        L.bmm_transpose.argtypes = [vp, vp, i64, i64, vp]
        L.bmm_transpose.restype = i32
        L.bmm_base_product.argtypes = [i32, i32, vp, vp, vp, i64, i64, i64, vp]
        L.bmm_base_product.restype = i32
        L.bmm_basis_change.argtypes = [i32, i32, vp, i64, i64, i32, vp]
        L.bmm_basis_change.restype = i32
        L.bmm_stream_status.argtypes = [vp]
        L.bmm_stream_status.restype = i32
        L.bmm_status_string.argtypes = [i32]
        L.bmm_status_string.restype = ctypes.c_char_p
        L.bmm_last_cuda_error.restype = i32
        L.bmm_device_supported.restype = i32
        L.bmm_plan.argtypes = [i32, i64, i64, i64, ctypes.POINTER(Opts),
                               ctypes.POINTER(PlanInfo)]
        L.bmm_plan.restype = i32
        L.bmm_product_noalloc.argtypes = [i32, vp, vp, vp, i64, i64, i64, vp]
        L.bmm_product_noalloc.restype = i32
        L.bmm_selftest_wait_timeout.argtypes = [i64, vp]
        L.bmm_selftest_wait_timeout.restype = i32
        L.bmm_trace_enable.argtypes = [i32]
        L.bmm_trace_enable.restype = None
        L.bmm_trace_read.argtypes = [i32, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double)]
        L.bmm_trace_read.restype = i32
        L.bmm_launch_count.restype = i64
        L.bmm_autotune.argtypes = [i32, i64, i64, i64, ctypes.c_uint32, vp,
                                   ctypes.POINTER(TuneResult)]
        L.bmm_autotune.restype = i32
        L.bmm_autotune_clear.argtypes = []
        L.bmm_autotune_clear.restype = None
        L.bmm_host_opts_default.argtypes = [ctypes.POINTER(HostOpts)]
        L.bmm_host_opts_default.restype = None
        L.bmm_host_plan.argtypes = [i32, i64, i64, i64, ctypes.POINTER(HostOpts),
                                    ctypes.POINTER(HostPlanInfo)]
        L.bmm_host_plan.restype = i32
        for f in (L.bmm_gf2_host, L.bmm_bool_host):
            f.argtypes = [vp, vp, vp, i64, i64, i64, ctypes.POINTER(HostOpts), vp]
            f.restype = i32
        L.bmm_host_release.argtypes = []
        L.bmm_host_release.restype = None
        _LIB = L
    return _LIB


def lib():
    """The loaded ctypes handle of libbmm.so."""
    return _lib_handle()


def _stream(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> int:
    if t is None:
        return 0
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data  # numpy array in host memory


def _check(status: int, what: str):
    if status != OK:
        raise BmmError(status, what)


def opts(path: int | None = None, depth: int | None = None, variant: int | None = None,
         serial: int | None = None, workspace=None, workspace_bytes: int = 0,
         kernel_level: int | None = None) -> Opts:
    o = Opts()
    _lib_handle().bmm_opts_default(ctypes.byref(o))
    if path is not None:
        o.path = path
    if depth is not None:
        o.strassen_depth = depth
    if variant is not None:
        o.variant = variant
    if serial is not None:
        o.serial_depth = serial
    if kernel_level is not None:
        o.kernel_level = kernel_level
    if workspace is not None:
        o.workspace = _ptr(workspace)
        o.workspace_bytes = workspace_bytes
    return o


def empty(rows: int, cols: int, device="cuda"):
    """An uninitialised packed rows x cols bit matrix on the device."""
    import torch

    return torch.empty(rows * cols // 64, dtype=torch.int64, device=device)


def gf2(A, B, C, m: int, k: int, n: int, stream=None, **kw) -> None:
    """C = A B over GF(2)."""
    L = _lib_handle()
    if kw:
        o = opts(**kw)
        _check(L.bmm_gf2_ex(_ptr(A), _ptr(B), _ptr(C), m, k, n, ctypes.byref(o), _stream(stream)),
               "bmm_gf2_ex")
    else:
        _check(L.bmm_gf2(_ptr(A), _ptr(B), _ptr(C), m, k, n, _stream(stream)), "bmm_gf2")


def boolean(A, B, C, m: int, k: int, n: int, stream=None, **kw) -> None:
    """C = A B over the Boolean algebra."""
    L = _lib_handle()
    if kw:
        o = opts(**kw)
        _check(L.bmm_bool_ex(_ptr(A), _ptr(B), _ptr(C), m, k, n, ctypes.byref(o),
                             _stream(stream)), "bmm_bool_ex")
    else:
        _check(L.bmm_bool(_ptr(A), _ptr(B), _ptr(C), m, k, n, _stream(stream)), "bmm_bool")


def product(op: int, A, B, C, m: int, k: int, n: int, stream=None, **kw) -> None:
    (gf2 if op == GF2 else boolean)(A, B, C, m, k, n, stream=stream, **kw)


def product_noalloc(op: int, A, B, C, m: int, k: int, n: int, stream=None) -> None:
    """Cubic product that allocates nothing (fixed device scratch; see bmm.h)."""
    _check(_lib_handle().bmm_product_noalloc(op, _ptr(A), _ptr(B), _ptr(C), m, k, n,
                                             _stream(stream)), "bmm_product_noalloc")


def workspace_size(op: int, m: int, k: int, n: int, **kw) -> int:
    o = opts(**kw)
    out = ctypes.c_uint64(0)
    _check(_lib_handle().bmm_workspace_size(op, m, k, n, ctypes.byref(o), ctypes.byref(out)),
           "bmm_workspace_size")
    return int(out.value)


def autotune(op: int, m: int, k: int, n: int, model: bool = False, stream=None) -> dict:
    """Time the candidate (path, Strassen depth) pairs for this shape, record the
    fastest for the planner's automatic choice and return it."""
    r = TuneResult()
    _check(_lib_handle().bmm_autotune(op, m, k, n, TUNE_MODEL if model else 0, _stream(stream),
                                      ctypes.byref(r)), "bmm_autotune")
    return {"path": r.best.path, "strassen_depth": r.best.strassen_depth, "est_ms": r.est_ms,
            "measured": bool(r.measured), "candidates": r.candidates}


def autotune_clear() -> None:
    """Forget every recorded tuning choice."""
    _lib_handle().bmm_autotune_clear()


def plan(op: int, m: int, k: int, n: int, **kw) -> dict:
    """The planner's resolution of the options for these sizes."""
    o = opts(**kw)
    info = PlanInfo()
    _check(_lib_handle().bmm_plan(op, m, k, n, ctypes.byref(o), ctypes.byref(info)), "bmm_plan")
    return {f: int(getattr(info, f)) for f, _ in PlanInfo._fields_}


def host_opts(device_bytes: int = 0, host_depth: int = -1, threads: int = 0,
              **kw) -> HostOpts:
    """Options of a host-memory product (bmm_host_opts); kw as opts() for the
    device products."""
    o = HostOpts()
    _lib_handle().bmm_host_opts_default(ctypes.byref(o))
    o.device = opts(**kw)
    o.device_bytes = device_bytes
    o.host_depth = host_depth
    o.threads = threads
    return o


def host_plan(op: int, m: int, k: int, n: int, **kw) -> dict:
    """What a host-memory product with these sizes does (host levels, device
    products, memory and traffic)."""
    o = host_opts(**kw)
    info = HostPlanInfo()
    _check(_lib_handle().bmm_host_plan(op, m, k, n, ctypes.byref(o), ctypes.byref(info)),
           "bmm_host_plan")
    return {f: int(getattr(info, f)) for f, _ in HostPlanInfo._fields_}


def product_host(op: int, A, B, C, m: int, k: int, n: int, stream=None, **kw) -> None:
    """C = A B with A, B, C in host memory (numpy arrays or CPU tensors, packed
    row-major words; pinned memory overlaps the copies). Blocks until C is
    complete."""
    o = host_opts(**kw)
    f = _lib_handle().bmm_gf2_host if op == GF2 else _lib_handle().bmm_bool_host
    _check(f(_ptr(A), _ptr(B), _ptr(C), m, k, n, ctypes.byref(o), _stream(stream)),
           "bmm_gf2_host" if op == GF2 else "bmm_bool_host")


def host_release() -> None:
    """Free the buffers host-memory products keep between calls."""
    _lib_handle().bmm_host_release()


def transpose(X, Xt, rows: int, cols: int, stream=None) -> None:
    _check(_lib_handle().bmm_transpose(_ptr(X), _ptr(Xt), rows, cols, _stream(stream)),
           "bmm_transpose")


def base_product(op: int, path: int, A, Bt, C, m: int, k: int, n: int, stream=None) -> None:
    """C = A Bt^T (the base case in NT form) on one path."""
    _check(_lib_handle().bmm_base_product(op, path, _ptr(A), _ptr(Bt), _ptr(C), m, k, n,
                                          _stream(stream)), "bmm_base_product")


def basis_change(variant: int, inverse: bool, X, rows: int, cols: int, depth: int,
                 stream=None) -> None:
    _check(_lib_handle().bmm_basis_change(variant, int(inverse), _ptr(X), rows, cols, depth,
                                          _stream(stream)), "bmm_basis_change")


def _batch_arrays(ops, As, Bs, Cs, ms, ks, ns):
    count = len(As)
    P = ctypes.c_void_p * count
    I = ctypes.c_int64 * count
    O = ctypes.c_int32 * count
    return (count, O(*ops), P(*map(_ptr, As)), P(*map(_ptr, Bs)), P(*map(_ptr, Cs)), I(*ms),
            I(*ks), I(*ns))


def batched(ops, As, Bs, Cs, ms, ks, ns, stream=None) -> None:
    """C_i = A_i B_i for every i in one persistent launch; ops[i] 0 = GF(2),
    1 = Boolean (or one int for the whole batch). Returns when done."""
    if isinstance(ops, int):
        ops = [ops] * len(As)
    arr = _batch_arrays(ops, As, Bs, Cs, ms, ks, ns)
    _check(_lib_handle().bmm_batched(*arr, _stream(stream)), "bmm_batched")


def _struct_dict(x) -> dict:
    return {f: getattr(x, f) for f, _ in x._fields_}


class BatchedPlan:
    """A reusable batch plan (see bmm_batched_plan_create); run() only launches.
    path: a bmm_path for every problem (default: the automatic choice per
    problem); paths: one bmm_path per problem instead (AUTO entries left to
    the model)."""

    def __init__(self, ops, As, Bs, Cs, ms, ks, ns, path: int = PATH_AUTO, paths=None):
        if isinstance(ops, int):
            ops = [ops] * len(As)
        self._arr = _batch_arrays(ops, As, Bs, Cs, ms, ks, ns)
        h = ctypes.c_void_p(0)
        if paths is None:
            _check(_lib_handle().bmm_batched_plan_create_ex(*self._arr, path, ctypes.byref(h)),
                   "bmm_batched_plan_create_ex")
        else:
            self._paths = (ctypes.c_int32 * len(paths))(*paths)
            _check(_lib_handle().bmm_batched_plan_create_paths(*self._arr, self._paths,
                                                               ctypes.byref(h)),
                   "bmm_batched_plan_create_paths")
        self._h = h

    def choice(self, i: int) -> dict:
        """What the plan decided for problem i (path, tile form, k steps)."""
        c = BatchedChoice()
        _check(_lib_handle().bmm_batched_plan_choice(self._h, i, ctypes.byref(c)),
               "bmm_batched_plan_choice")
        return _struct_dict(c)

    def stats(self) -> dict:
        """Problems per path, tiles per form, MACs needed and issued, model time."""
        st = BatchedStats()
        _check(_lib_handle().bmm_batched_plan_stats(self._h, ctypes.byref(st)),
               "bmm_batched_plan_stats")
        return _struct_dict(st)

    def run(self, stream=None) -> None:
        _check(_lib_handle().bmm_batched_plan_run(self._h, _stream(stream)),
               "bmm_batched_plan_run")

    def path(self) -> int:
        """The base-case path the plan runs."""
        p = ctypes.c_int32(0)
        _check(_lib_handle().bmm_batched_plan_path(self._h, ctypes.byref(p)),
               "bmm_batched_plan_path")
        return p.value

    def destroy(self) -> None:
        if self._h:
            _check(_lib_handle().bmm_batched_plan_destroy(self._h), "bmm_batched_plan_destroy")
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def batched_model(path: int = PATH_AUTO) -> dict:
    """The batched schedule's cost model on the current device (measured on
    first use)."""
    m = BatchedModel()
    _check(_lib_handle().bmm_batched_model(path, ctypes.byref(m)), "bmm_batched_model")
    return _struct_dict(m)


def stream_status(stream=None) -> None:
    """Synchronise the stream and raise if a device-side wait timed out."""
    _check(_lib_handle().bmm_stream_status(_stream(stream)), "bmm_stream_status")


def device_supported() -> bool:
    return bool(_lib_handle().bmm_device_supported())


def trace_enable(on: bool) -> None:
    """Record a CUDA event pair around every library kernel launch (or stop)."""
    _lib_handle().bmm_trace_enable(int(on))


def trace_read(phase: int) -> tuple[int, float]:
    """(launches, summed device milliseconds) recorded for one phase."""
    n = ctypes.c_int64(0)
    ms = ctypes.c_double(0.0)
    _check(_lib_handle().bmm_trace_read(phase, ctypes.byref(n), ctypes.byref(ms)),
           "bmm_trace_read")
    return int(n.value), float(ms.value)


def launch_count() -> int:
    return int(_lib_handle().bmm_launch_count())
