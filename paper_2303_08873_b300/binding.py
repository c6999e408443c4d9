"""ctypes binding of ``libadaptive_region.so`` (argument marshalling only).

Function names match the C ABI (``include/ar.h``, ``include/ar_loops.h``).
Pointer arguments accept ``torch.Tensor`` (``data_ptr()``), numpy arrays, plain
integers or ``None``; stream arguments accept ``torch.cuda.Stream``, a raw
``cudaStream_t`` integer or ``None`` (default stream).  Negative status codes
raise :class:`ArError`.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# AR_CHECKED=1 selects the bounds-check flavour of the library (build.py --checked)
CHECKED = os.environ.get("AR_CHECKED", "0") == "1"
LIB_PATH = os.path.join(HERE, "libadaptive_region_checked.so" if CHECKED else "libadaptive_region.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python paper_2303_08873_b300/build.py"
        f"{' --checked' if CHECKED else ''}` "
        "(there is no non-CUDA fallback)")
lib = ctypes.CDLL(LIB_PATH)

AR_OK, AR_ERR_ARG, AR_ERR_STATE, AR_ERR_CUDA, AR_ERR_NOMODEL, AR_ERR_IO, AR_ERR_TIMEOUT, AR_ERR_OOM = (
    0, -1, -2, -3, -4, -5, -6, -7)
STATUS_NAMES = {0: "AR_OK", -1: "AR_ERR_ARG", -2: "AR_ERR_STATE", -3: "AR_ERR_CUDA", -4: "AR_ERR_NOMODEL",
                -5: "AR_ERR_IO", -6: "AR_ERR_TIMEOUT", -7: "AR_ERR_OOM"}
AR_MAX_FEATURES = 8
AR_MAX_VARIANTS = 64
AR_LOOP_DAXPY, AR_LOOP_JACOBI7, AR_LOOP_SPMV, AR_LOOP_NBODY, AR_LOOP_HEAT7 = 0, 1, 2, 3, 4
MODEL_KINDS = {0: "dtree", 1: "mlp", 2: "exhaustive", 3: "fixed", 4: "rfc"}


class ArError(RuntimeError):
    def __init__(self, code: int, msg: str = ""):
        self.code = code
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}" if msg else STATUS_NAMES.get(code, str(code)))


# ------------------------------------------------------------------ types
_vp = ctypes.c_void_p
_i = ctypes.c_int
_i64 = ctypes.c_int64
_d = ctypes.c_double
_f = ctypes.c_float
_sz = ctypes.c_size_t
_cs = ctypes.c_char_p
_pi = ctypes.POINTER(ctypes.c_int)
_pi64 = ctypes.POINTER(ctypes.c_int64)
_pd = ctypes.POINTER(ctypes.c_double)
_pf = ctypes.POINTER(ctypes.c_float)

LAUNCH_FN = ctypes.CFUNCTYPE(_i, _vp, _i, _d, _vp, _vp)
FAKE_TIME_FN = ctypes.CFUNCTYPE(_d, _pf, _i, _i, _vp)


class ArDaxpyArgs(ctypes.Structure):
    _fields_ = [("n", _i64), ("a", _d), ("x", _vp), ("y", _vp)]


class ArJacobi7Args(ctypes.Structure):
    _fields_ = [("N", _i), ("sweeps", _i), ("u0", _vp), ("out", _vp), ("work", _vp), ("status", _vp)]


class ArHeat7Args(ctypes.Structure):
    _fields_ = [("N", _i), ("steps", _i), ("alpha", _d), ("u0", _vp), ("out", _vp), ("work", _vp),
                ("status", _vp)]


class ArSpmvArgs(ctypes.Structure):
    _fields_ = [("rows", _i64), ("nnz", _i64), ("rowptr", _vp), ("col", _vp), ("val", _vp), ("x", _vp),
                ("y", _vp), ("workspace", _vp), ("workspace_bytes", _sz)]


class ArNbodyArgs(ctypes.Structure):
    _fields_ = [("N", _i64), ("pos4", _vp), ("acc4", _vp), ("eps", _f)]


class ArDaxpySplitArgs(ctypes.Structure):
    _fields_ = [("n", _i64), ("a", _d), ("x", _vp), ("y", _vp), ("x_dev", _vp), ("y_dev", _vp),
                ("gpu_variant", _i)]


class ArSpmvSplitArgs(ctypes.Structure):
    _fields_ = [("rows", _i64), ("nnz", _i64), ("cols", _i64), ("rowptr", _vp), ("col", _vp), ("val", _vp),
                ("x", _vp), ("y", _vp), ("rowptr_dev", _vp), ("col_dev", _vp), ("val_dev", _vp), ("x_dev", _vp),
                ("y_dev", _vp), ("workspace", _vp), ("workspace_bytes", _sz), ("gpu_variant", _i)]


class ArExecCall(ctypes.Structure):
    _fields_ = [("loop", ctypes.c_int32), ("sweeps", ctypes.c_int32), ("n", _i64), ("nnz", _i64), ("a", _d),
                ("eps", _f), ("reserved", ctypes.c_int32), ("in0", _vp), ("in1", _vp), ("in2", _vp), ("in3", _vp),
                ("out0", _vp), ("out1", _vp), ("out1_bytes", ctypes.c_uint64)]


class ArHostCopy(ctypes.Structure):
    _fields_ = [("host", _vp), ("device", _vp), ("bytes", _sz)]


class ArExecModels(ctypes.Structure):
    _fields_ = [("F", ctypes.c_int32 * 4), ("V", ctypes.c_int32 * 4), ("H", ctypes.c_int32),
                ("theta", _vp * 4), ("mu", _vp * 4), ("sd", _vp * 4)]


AR_EXEC_MAX_CALLS = 256
AR_EXEC_MAX_PHASES = 64


_SIGS = {
    # ar.h
    "ar_region_create": (_i, [_cs, _i, _cs, _i, ctypes.POINTER(_vp)]),
    "ar_region_destroy": (None, [_vp]),
    "ar_variant_register": (_i, [_vp, _cs, _d, LAUNCH_FN, _vp, _pi]),
    "ar_variant_register_range": (_i, [_vp, _d, _d, _d, LAUNCH_FN, _vp, _pi]),
    "ar_region_info": (_i, [_vp, _pi, _pi, _pi, _pi, _pi]),
    "ar_variant_info": (_i, [_vp, _i, _pd, _cs, _i, _pi]),
    "ar_begin": (_i, [_vp, _vp]),
    "ar_set_feature": (_i, [_vp, _f]),
    "ar_get_policy": (_i, [_vp, _pi]),
    "ar_end": (_i, [_vp, _vp]),
    "ar_invoke": (_i, [_vp, _pf, _i, _vp, _vp, _pi, _pd]),
    "ar_invoke_host": (_i, [_vp, _pf, _i, _vp, _vp, ctypes.POINTER(ArHostCopy), _i, ctypes.POINTER(ArHostCopy), _i,
                            _pi, _pd]),
    "ar_select": (_i, [_vp, _pf, _i, _pi, _pf]),
    "ar_profile": (_i, [_vp, _pf, _i, _vp, _vp, _i, _pf, _pi]),
    "ar_train": (_i, [_vp]),
    "ar_flush_records": (_i, [_vp]),
    "ar_add_record": (_i, [_vp, _pf, _i, _i, _f]),
    "ar_record_counts": (_i, [_vp, _pi64, _pi64]),
    "ar_get_records": (_i, [_vp, _i64, _i64, _pf, _pi, _pf]),
    "ar_tree_export": (_i, [_vp, _i, _pi, _pd, _pi, _pi, _pi, _pi]),
    "ar_forest_size": (_i, [_vp, _pi]),
    "ar_forest_tree_export": (_i, [_vp, _i, _i, _pi, _pd, _pi, _pi, _pi, _pi]),
    "ar_mlp_export": (_i, [_vp, _pf, _pf, _pf, _pi, _pi, _pi]),
    "ar_region_save": (_i, [_vp, _cs]),
    "ar_region_load": (_i, [_vp, _cs]),
    "ar_last_error": (_i, [_vp, _cs, _i]),
    "ar_set_fake_timer": (_i, [_vp, FAKE_TIME_FN, _vp]),
    "ar_set_l2_flush": (_i, [_vp, _vp, _sz]),
    # ar_loops.h
    "ar_loop_num_variants": (_i, [_i]),
    "ar_loop_default_variant": (_i, [_i]),
    "ar_loop_variant_name": (_i, [_i, _i, _cs, _i]),
    "ar_region_add_builtin": (_i, [_vp, _i, _pi]),
    "ar_region_add_builtin_first": (_i, [_vp, _i, _i, _pi]),
    "ar_daxpy": (_i, [_i, _i64, _d, _vp, _vp, _vp]),
    "ar_jacobi7": (_i, [_i, _i, _i, _vp, _vp, _vp, _vp, _vp]),
    "ar_heat7": (_i, [_i, _i, _i, _d, _vp, _vp, _vp, _vp, _vp]),
    "ar_spmv_workspace_bytes": (_i, [_i, _i64, _i64, ctypes.POINTER(_sz)]),
    "ar_spmv": (_i, [_i, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "ar_spmv_merge_path_noalloc": (_i, [_i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "ar_csr_features_workspace_bytes": (_i, [_i64, ctypes.POINTER(_sz)]),
    "ar_spmv_gather_floor": (_i, [_i64, _vp, _vp, _vp, _vp, _vp]),
    "ar_csr_features": (_i, [_i64, _vp, _vp, _vp, _sz, _vp]),
    "ar_nbody": (_i, [_i, _i64, _vp, _vp, _f, _vp]),
    "ar_nbody_geometry": (_i, [_i, _i64, _pi64, _pi, _pi, _pi, _pi]),
    "ar_nbody_batched_workspace_bytes": (_i, [_i, ctypes.POINTER(_sz)]),
    "ar_nbody_batched": (_i, [_i, _vp, _vp, _vp, _f, _vp, _sz, _vp]),
    "ar_daxpy_split": (_i, [_d, ctypes.POINTER(ArDaxpySplitArgs), _vp]),
    "ar_spmv_split": (_i, [_d, ctypes.POINTER(ArSpmvSplitArgs), _vp]),
    "ar_region_add_split": (_i, [_vp, _i, _d, _d, _d, _pi]),
    "ar_split_threads": (_i, []),
    "ar_exec_workspace_bytes": (_i, [_i, ctypes.POINTER(_sz)]),
    "ar_exec_num_variants": (_i, [_i]),
    "ar_wait_selftest": (_i, [_i, ctypes.c_uint, _vp, _vp]),
    "ar_exec_batch": (_i, [_vp, _i, ctypes.POINTER(ArExecModels), _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "ar_exec_fallback_workspace_bytes": (_i, [_i64, ctypes.POINTER(_sz)]),
    "ar_exec_fallback": (_i, [_vp, _i, _pf, _pf, _f, ctypes.POINTER(_vp), _i, ctypes.POINTER(ArExecModels), _i, _vp,
                              _sz, _vp, ctypes.POINTER(ctypes.c_int32), _pi]),
    "ar_mlp_num_params": (_i, [_i, _i, _i]),
    "ar_mlp_forward": (_i, [_vp, _vp, _vp, _i, _i, _i, _i64, _vp, _vp, _vp, _vp, _vp]),
    "ar_mlp_grad": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _vp, _vp, _vp, _vp, _vp]),
    "ar_mlp_adam": (_i, [_vp, _vp, _vp, _vp, _i64, _i, _f, _vp]),
    "ar_mlp_train": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _i, _i, _i, _vp, _vp, _vp, _i, _i, _f, _vp, _vp]),
    "ar_measure_fma_rates": (_i, [_pd, _pd]),
    "ar_measure_fp32x2_rate": (_i, [_pd]),
    "ar_check_status": (_i, [_pi, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32), _i]),
}

for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args

EXPORTED = tuple(_SIGS)


# ------------------------------------------------------------------ helpers
def ptr(x):
    """Device/host address of a tensor, array or int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def stream_handle(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def check(rc: int, region=None) -> int:
    if rc is not None and rc < 0:
        msg = ""
        if region is not None:
            buf = ctypes.create_string_buffer(512)
            lib.ar_last_error(region, buf, 512)
            msg = buf.value.decode(errors="replace")
        raise ArError(rc, msg)
    return rc


def _floats(features):
    f = np.ascontiguousarray(np.asarray(features, dtype=np.float32).ravel())
    return f, f.ctypes.data_as(_pf), f.size


# ------------------------------------------------------------------ loops
def loop_num_variants(loop: int) -> int:
    return check(lib.ar_loop_num_variants(loop))


def loop_default_variant(loop: int) -> int:
    return check(lib.ar_loop_default_variant(loop))


def loop_variant_name(loop: int, variant: int) -> str:
    buf = ctypes.create_string_buffer(64)
    check(lib.ar_loop_variant_name(loop, variant, buf, 64))
    return buf.value.decode()


def ar_daxpy(variant, n, a, x, y, stream=None):
    return check(lib.ar_daxpy(variant, n, a, ptr(x), ptr(y), stream_handle(stream)))


def ar_jacobi7(variant, N, sweeps, u0, out, work, status=None, stream=None):
    return check(lib.ar_jacobi7(variant, N, sweeps, ptr(u0), ptr(out), ptr(work), ptr(status),
                                stream_handle(stream)))


def ar_spmv_gather_floor(nnz, col, val, x, sink8, stream=None):
    return check(lib.ar_spmv_gather_floor(nnz, ptr(col), ptr(val), ptr(x), ptr(sink8), stream_handle(stream)))


def ar_heat7(variant, N, steps, alpha, u0, out, work, status=None, stream=None):
    return check(lib.ar_heat7(variant, N, steps, alpha, ptr(u0), ptr(out), ptr(work), ptr(status),
                              stream_handle(stream)))


def ar_spmv_workspace_bytes(variant, rows, nnz):
    b = ctypes.c_size_t()
    check(lib.ar_spmv_workspace_bytes(variant, rows, nnz, ctypes.byref(b)))
    return b.value


def ar_spmv(variant, rows, nnz, rowptr, col, val, x, y, workspace=None, workspace_bytes=0, stream=None):
    return check(lib.ar_spmv(variant, rows, nnz, ptr(rowptr), ptr(col), ptr(val), ptr(x), ptr(y), ptr(workspace),
                             workspace_bytes, stream_handle(stream)))


def ar_spmv_merge_path_noalloc(rows, nnz, rowptr, col, val, x, y, stream=None):
    return check(lib.ar_spmv_merge_path_noalloc(rows, nnz, ptr(rowptr), ptr(col), ptr(val), ptr(x), ptr(y),
                                                stream_handle(stream)))


def ar_csr_features_workspace_bytes(rows):
    b = ctypes.c_size_t()
    check(lib.ar_csr_features_workspace_bytes(rows, ctypes.byref(b)))
    return b.value


def ar_csr_features(rows, rowptr, out5, workspace, workspace_bytes, stream=None):
    return check(lib.ar_csr_features(rows, ptr(rowptr), ptr(out5), ptr(workspace), workspace_bytes,
                                     stream_handle(stream)))


def ar_nbody(variant, N, pos4, acc4, eps=1e-2, stream=None):
    return check(lib.ar_nbody(variant, N, ptr(pos4), ptr(acc4), eps, stream_handle(stream)))


def ar_nbody_geometry(variant, N):
    """dict(grid, cluster, bodies_per_thread, resident_per_sm, sms, waves)."""
    g, c, b, r, m = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check(lib.ar_nbody_geometry(variant, N, ctypes.byref(g), ctypes.byref(c), ctypes.byref(b), ctypes.byref(r),
                                ctypes.byref(m)))
    return {"grid": g.value, "cluster": c.value, "bodies_per_thread": b.value, "resident_per_sm": r.value,
            "sms": m.value, "waves": g.value * c.value / (r.value * m.value)}


def ar_nbody_batched_workspace_bytes(count):
    b = ctypes.c_size_t()
    check(lib.ar_nbody_batched_workspace_bytes(count, ctypes.byref(b)))
    return b.value


def ar_nbody_batched(count, offs, pos4, acc4, eps, workspace, workspace_bytes, stream=None):
    return check(lib.ar_nbody_batched(count, ptr(offs), ptr(pos4), ptr(acc4), eps, ptr(workspace), workspace_bytes,
                                      stream_handle(stream)))


def ar_daxpy_split(gpu_fraction, args, stream=None):
    return check(lib.ar_daxpy_split(gpu_fraction, ctypes.byref(args), stream_handle(stream)))


def ar_spmv_split(gpu_fraction, args, stream=None):
    return check(lib.ar_spmv_split(gpu_fraction, ctypes.byref(args), stream_handle(stream)))


def ar_split_threads():
    return check(lib.ar_split_threads())


def ar_exec_num_variants(loop):
    return check(lib.ar_exec_num_variants(loop))


def ar_exec_workspace_bytes(max_calls):
    b = ctypes.c_size_t()
    check(lib.ar_exec_workspace_bytes(max_calls, ctypes.byref(b)))
    return b.value


def ar_exec_batch(calls, ncalls, models, force_variant, variant, conf, features, t_start, t_end, status, workspace,
                  workspace_bytes, stream=None):
    """calls: device buffer holding `ncalls` ArExecCall records; models: an
    ArExecModels (host) or None."""
    mp = ctypes.byref(models) if models is not None else None
    return check(lib.ar_exec_batch(ptr(calls), ncalls, mp, ptr(force_variant), ptr(variant), ptr(conf), ptr(features),
                                   ptr(t_start), ptr(t_end), ptr(status), ptr(workspace), workspace_bytes,
                                   stream_handle(stream)))


def ar_exec_fallback_workspace_bytes(max_daxpy_n):
    b = ctypes.c_size_t()
    check(lib.ar_exec_fallback_workspace_bytes(max_daxpy_n, ctypes.byref(b)))
    return b.value


def ar_exec_fallback(calls, features, conf, tau, regions, reps, models, retrain, workspace, workspace_bytes,
                     stream=None):
    """calls: list of ArExecCall (host); features: (n, 8) float32 and conf:
    (n,) float32 host arrays (the batch's outputs); regions: four Region
    objects or None.  Returns (best variant per call, -1 if not profiled;
    number of calls profiled)."""
    n = len(calls)
    arr = (ArExecCall * max(n, 1))(*calls)
    f = np.ascontiguousarray(np.asarray(features, dtype=np.float32).reshape(n, 8) if n else np.zeros((1, 8), np.float32))
    c = np.ascontiguousarray(np.asarray(conf, dtype=np.float32).reshape(n) if n else np.zeros(1, np.float32))
    regs = (_vp * 4)(*[r.h if r is not None else None for r in regions])
    best = np.full(max(n, 1), -1, dtype=np.int32)
    cnt = ctypes.c_int()
    mp = ctypes.byref(models) if models is not None else None
    check(lib.ar_exec_fallback(ctypes.addressof(arr), n, f.ctypes.data_as(_pf), c.ctypes.data_as(_pf), tau, regs, reps,
                               mp, int(retrain), ptr(workspace), workspace_bytes, stream_handle(stream),
                               best.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(cnt)))
    return best[:n], cnt.value


def exec_table_bytes(calls) -> bytes:
    """Pack a list of ArExecCall into the byte image of the device call table."""
    arr = (ArExecCall * len(calls))(*calls)
    return bytes(arr)


def ar_mlp_num_params(F, H, V):
    return check(lib.ar_mlp_num_params(F, H, V))


def ar_mlp_forward(theta, mu, sd, F, H, V, B, feats, probs=None, variant=None, conf=None, stream=None):
    return check(lib.ar_mlp_forward(ptr(theta), ptr(mu), ptr(sd), F, H, V, B, ptr(feats), ptr(probs),
                                    ptr(variant), ptr(conf), stream_handle(stream)))


def ar_mlp_grad(theta, mu, sd, F, H, V, B, feats, labels, grad, loss=None, stream=None):
    return check(lib.ar_mlp_grad(ptr(theta), ptr(mu), ptr(sd), F, H, V, B, ptr(feats), ptr(labels), ptr(grad),
                                 ptr(loss), stream_handle(stream)))


def ar_mlp_adam(theta, grad, m, v, n, t, lr, stream=None):
    return check(lib.ar_mlp_adam(ptr(theta), ptr(grad), ptr(m), ptr(v), n, t, lr, stream_handle(stream)))


def ar_mlp_train(theta, adam_m, adam_v, mu, sd, F, H, V, n, feats, labels, perm, epochs, batch, lr, loss=None,
                 stream=None):
    return check(lib.ar_mlp_train(ptr(theta), ptr(adam_m), ptr(adam_v), ptr(mu), ptr(sd), F, H, V, n, ptr(feats),
                                  ptr(labels), ptr(perm), epochs, batch, lr, ptr(loss), stream_handle(stream)))


def ar_measure_fma_rates():
    a, b = ctypes.c_double(), ctypes.c_double()
    check(lib.ar_measure_fma_rates(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def ar_check_status(clear: bool = True):
    """(enabled, first failing check as (source id << 16 | line), failures)
    of the bounds-check build; (False, 0, 0) in the normal build."""
    en, first, cnt = ctypes.c_int(), ctypes.c_uint32(), ctypes.c_uint32()
    check(lib.ar_check_status(ctypes.byref(en), ctypes.byref(first), ctypes.byref(cnt), int(clear)))
    return bool(en.value), first.value, cnt.value


def ar_measure_fp32x2_rate():
    """float32 lane FMAs per second issued as packed pairs (FFMA2)."""
    a = ctypes.c_double()
    check(lib.ar_measure_fp32x2_rate(ctypes.byref(a)))
    return a.value


# ------------------------------------------------------------------ regions
class Region:
    """Owning wrapper of an ``ar_region*`` (one call per C function)."""

    def __init__(self, id: str, num_features: int, model_spec: str = "", min_train_data: int = 0):
        h = _vp()
        check(lib.ar_region_create(id.encode(), num_features, model_spec.encode(), min_train_data, ctypes.byref(h)))
        self.h = h
        self.nf = num_features
        self._keep = []  # ctypes callbacks and argument blocks that must stay alive

    def close(self):
        if getattr(self, "h", None):
            lib.ar_region_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def _ck(self, rc):
        return check(rc, self.h)

    # registration
    def add_builtin(self, loop: int) -> int:
        n = ctypes.c_int()
        self._ck(lib.ar_region_add_builtin(self.h, loop, ctypes.byref(n)))
        return n.value

    def add_builtin_first(self, loop: int, count: int) -> int:
        n = ctypes.c_int()
        self._ck(lib.ar_region_add_builtin_first(self.h, loop, count, ctypes.byref(n)))
        return n.value

    def add_split(self, loop: int, begin: float = 0.0, end: float = 1.0, step: float = 0.1) -> int:
        """GPU fractions [begin:end:step] of a host-data split loop (ar_region_add_split)."""
        n = ctypes.c_int()
        self._ck(lib.ar_region_add_split(self.h, loop, begin, end, step, ctypes.byref(n)))
        return n.value

    def add_exec_variants(self, loop: int) -> int:
        """The variants the mixed-stream executor runs for `loop`."""
        return self.add_builtin_first(loop, ar_exec_num_variants(loop))

    def register(self, name: str, value: float, launcher) -> int:
        cb = launcher if isinstance(launcher, LAUNCH_FN) else LAUNCH_FN(launcher)
        self._keep.append(cb)
        idx = ctypes.c_int()
        self._ck(lib.ar_variant_register(self.h, name.encode(), value, cb, None, ctypes.byref(idx)))
        return idx.value

    def register_range(self, begin: float, end: float, step: float, launcher) -> int:
        cb = launcher if isinstance(launcher, LAUNCH_FN) else LAUNCH_FN(launcher)
        self._keep.append(cb)
        n = ctypes.c_int()
        self._ck(lib.ar_variant_register_range(self.h, begin, end, step, cb, None, ctypes.byref(n)))
        return n.value

    def info(self) -> dict:
        v, f, m, t, k = (ctypes.c_int() for _ in range(5))
        self._ck(lib.ar_region_info(self.h, *(ctypes.byref(x) for x in (v, f, m, t, k))))
        return {"num_variants": v.value, "num_features": f.value, "min_train_data": m.value,
                "trained": bool(t.value), "model": MODEL_KINDS.get(k.value, k.value)}

    def variant(self, idx: int) -> dict:
        val, usable = ctypes.c_double(), ctypes.c_int()
        name = ctypes.create_string_buffer(128)
        self._ck(lib.ar_variant_info(self.h, idx, ctypes.byref(val), name, 128, ctypes.byref(usable)))
        return {"value": val.value, "name": name.value.decode(), "usable": bool(usable.value)}

    # Apollo-shaped calls
    def begin(self, stream=None):
        return self._ck(lib.ar_begin(self.h, stream_handle(stream)))

    def set_feature(self, value: float):
        return self._ck(lib.ar_set_feature(self.h, value))

    def get_policy(self) -> int:
        v = ctypes.c_int()
        self._ck(lib.ar_get_policy(self.h, ctypes.byref(v)))
        return v.value

    def end(self, stream=None):
        return self._ck(lib.ar_end(self.h, stream_handle(stream)))

    # convenience calls
    def invoke(self, features, args=None, stream=None):
        f, fp, n = _floats(features)
        v, val = ctypes.c_int(), ctypes.c_double()
        a = ctypes.cast(ctypes.pointer(args), _vp) if args is not None else None
        self._ck(lib.ar_invoke(self.h, fp, n, a, stream_handle(stream), ctypes.byref(v), ctypes.byref(val)))
        return v.value, val.value

    def invoke_host(self, features, args, copies_in, copies_out, stream=None):
        """ar_invoke_host: copies_in / copies_out are lists of (host, device,
        bytes) with host and device given as tensors, arrays or addresses."""
        f, fp, n = _floats(features)
        cin = (ArHostCopy * max(1, len(copies_in)))(*[ArHostCopy(ptr(h), ptr(d), b) for h, d, b in copies_in])
        cout = (ArHostCopy * max(1, len(copies_out)))(*[ArHostCopy(ptr(h), ptr(d), b) for h, d, b in copies_out])
        v, val = ctypes.c_int(), ctypes.c_double()
        a = ctypes.cast(ctypes.pointer(args), _vp) if args is not None else None
        self._ck(lib.ar_invoke_host(self.h, fp, n, a, stream_handle(stream), cin, len(copies_in), cout,
                                    len(copies_out), ctypes.byref(v), ctypes.byref(val)))
        return v.value, val.value

    def select(self, features):
        f, fp, n = _floats(features)
        v, c = ctypes.c_int(), ctypes.c_float()
        self._ck(lib.ar_select(self.h, fp, n, ctypes.byref(v), ctypes.byref(c)))
        return v.value, c.value

    def profile(self, features, args=None, stream=None, reps: int = 0):
        f, fp, n = _floats(features)
        V = self.info()["num_variants"]
        ms = (ctypes.c_float * V)()
        best = ctypes.c_int()
        a = ctypes.cast(ctypes.pointer(args), _vp) if args is not None else None
        self._ck(lib.ar_profile(self.h, fp, n, a, stream_handle(stream), reps, ms, ctypes.byref(best)))
        return list(ms), best.value

    def train(self):
        return self._ck(lib.ar_train(self.h))

    def flush_records(self):
        return self._ck(lib.ar_flush_records(self.h))

    def add_record(self, features, variant: int, ms: float):
        f, fp, n = _floats(features)
        return self._ck(lib.ar_add_record(self.h, fp, n, variant, ms))

    def counts(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._ck(lib.ar_record_counts(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def records(self, first: int = 0):
        """Resolved records [first, end) as a list of (features tuple, variant, ms)."""
        n, _ = self.counts()
        n -= first
        if n <= 0:
            return []
        F = np.zeros((n, AR_MAX_FEATURES), dtype=np.float32)
        V = np.zeros(n, dtype=np.int32)
        M = np.zeros(n, dtype=np.float32)
        self._ck(lib.ar_get_records(self.h, first, n, F.ctypes.data_as(_pf), V.ctypes.data_as(_pi),
                                    M.ctypes.data_as(_pf)))
        return [(tuple(float(x) for x in F[i, :self.nf]), int(V[i]), float(M[i])) for i in range(n)]

    def tree(self):
        """Decision tree as a list of (feature, threshold, left, right, label)."""
        cnt = ctypes.c_int()
        self._ck(lib.ar_tree_export(self.h, 0, None, None, None, None, None, ctypes.byref(cnt)))
        n = cnt.value
        fe = (ctypes.c_int * n)()
        th = (ctypes.c_double * n)()
        le = (ctypes.c_int * n)()
        ri = (ctypes.c_int * n)()
        la = (ctypes.c_int * n)()
        self._ck(lib.ar_tree_export(self.h, n, fe, th, le, ri, la, ctypes.byref(cnt)))
        return [(fe[i], th[i] if fe[i] >= 0 else 0.0, le[i], ri[i], la[i]) for i in range(n)]

    def forest(self):
        """Random forest as a list of trees in the layout of tree()."""
        nt = ctypes.c_int()
        self._ck(lib.ar_forest_size(self.h, ctypes.byref(nt)))
        out = []
        for t in range(nt.value):
            cnt = ctypes.c_int()
            self._ck(lib.ar_forest_tree_export(self.h, t, 0, None, None, None, None, None, ctypes.byref(cnt)))
            n = cnt.value
            fe, th = (ctypes.c_int * n)(), (ctypes.c_double * n)()
            le, ri, la = (ctypes.c_int * n)(), (ctypes.c_int * n)(), (ctypes.c_int * n)()
            self._ck(lib.ar_forest_tree_export(self.h, t, n, fe, th, le, ri, la, ctypes.byref(cnt)))
            out.append([(fe[i], th[i] if fe[i] >= 0 else 0.0, le[i], ri[i], la[i]) for i in range(n)])
        return out

    def mlp(self):
        F, H, V = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._ck(lib.ar_mlp_export(self.h, None, None, None, ctypes.byref(F), ctypes.byref(H), ctypes.byref(V)))
        P = ar_mlp_num_params(F.value, H.value, V.value)
        th = np.zeros(P, dtype=np.float32)
        mu = np.zeros(F.value, dtype=np.float32)
        sd = np.zeros(F.value, dtype=np.float32)
        self._ck(lib.ar_mlp_export(self.h, th.ctypes.data_as(_pf), mu.ctypes.data_as(_pf), sd.ctypes.data_as(_pf),
                                   None, None, None))
        return {"F": F.value, "H": H.value, "V": V.value, "theta": th, "mu": mu, "sd": sd}

    def save(self, path: str):
        return self._ck(lib.ar_region_save(self.h, str(path).encode()))

    def load(self, path: str):
        return self._ck(lib.ar_region_load(self.h, str(path).encode()))

    def last_error(self) -> str:
        buf = ctypes.create_string_buffer(512)
        lib.ar_last_error(self.h, buf, 512)
        return buf.value.decode(errors="replace")

    def set_fake_timer(self, fn):
        """fn(features tuple, variant) -> ms; None restores CUDA-event timing."""
        if fn is None:
            return self._ck(lib.ar_set_fake_timer(self.h, FAKE_TIME_FN(), None))
        nf = self.nf

        def _cb(fp, n, v, user):
            return float(fn(tuple(fp[i] for i in range(n)), v))

        cb = FAKE_TIME_FN(_cb)
        self._keep.append(cb)
        return self._ck(lib.ar_set_fake_timer(self.h, cb, None)) if nf >= 0 else None

    def set_l2_flush(self, buf, nbytes: int):
        return self._ck(lib.ar_set_l2_flush(self.h, ptr(buf), nbytes))


__all__ = ["ArExecCall", "ArExecModels", "ar_exec_workspace_bytes", "ar_exec_batch", "exec_table_bytes",
           "ar_exec_fallback", "ar_exec_fallback_workspace_bytes", "ar_exec_num_variants",
           "ArDaxpySplitArgs", "ArSpmvSplitArgs", "ar_daxpy_split", "ar_spmv_split", "ar_split_threads", "ArHostCopy", "ar_check_status", "CHECKED",
           "AR_EXEC_MAX_CALLS", "AR_EXEC_MAX_PHASES", "ArError", "Region", "ArDaxpyArgs", "ArJacobi7Args", "ArHeat7Args", "ArSpmvArgs", "ArNbodyArgs", "ar_spmv",
           "ar_spmv_workspace_bytes", "ar_spmv_merge_path_noalloc", "ar_spmv_gather_floor", "ar_csr_features", "ar_csr_features_workspace_bytes", "ar_nbody",
           "ar_nbody_batched", "ar_nbody_batched_workspace_bytes", "ar_nbody_geometry", "LAUNCH_FN", "FAKE_TIME_FN", "lib", "ptr",
           "stream_handle", "check", "loop_num_variants", "loop_default_variant", "loop_variant_name", "ar_daxpy",
           "ar_jacobi7", "ar_heat7", "ar_mlp_num_params", "ar_mlp_forward", "ar_mlp_grad", "ar_mlp_adam", "ar_mlp_train",
           "ar_measure_fma_rates", "ar_measure_fp32x2_rate", "EXPORTED", "AR_LOOP_DAXPY", "AR_LOOP_JACOBI7", "AR_LOOP_SPMV",
           "AR_LOOP_NBODY", "AR_LOOP_HEAT7", "AR_OK", "AR_ERR_ARG", "AR_ERR_STATE", "AR_ERR_CUDA", "AR_ERR_NOMODEL", "AR_ERR_IO",
           "AR_ERR_TIMEOUT", "AR_ERR_OOM", "AR_MAX_FEATURES", "AR_MAX_VARIANTS"]
