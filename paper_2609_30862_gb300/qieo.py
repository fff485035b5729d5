"""Thin ctypes binding of the C ABI in include/qieo.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does nothing but
convert arguments and raise QieoError on a non-zero status. All computation runs in the
CUDA library; if the library is missing this module raises instead of computing anything
on the host.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

QIEO_OK = 0
QIEO_ERR_INVALID = 1
QIEO_ERR_OOM = 2
QIEO_ERR_CUDA = 3
QIEO_ERR_TIMEOUT = 4
QIEO_ERR_BUSY = 5

QIEO_RULE_R1 = 0
QIEO_RULE_R2 = 1

QIEO_FLAG_NO_GRAPH = 0x1
QIEO_FLAG_SYNC_RUN = 0x2
QIEO_FLAG_FORCE_WIDE = 0x4
QIEO_FLAG_TIME_KERNELS = 0x8
QIEO_FLAG_COOPERATIVE = 0x10
QIEO_FLAG_REGISTER_PREFETCH = 0x20
QIEO_FLAG_UNFUSED = 0x40
QIEO_FLAG_CONVERGE = 0x80
QIEO_CONVERGE_WINDOW = 20
QIEO_FLAG_STATE_I8 = 0x100
QIEO_FLAG_PER_GENERATION = 0x200
QIEO_FLAG_TIME_GENERATIONS = 0x400
QIEO_FLAG_STREAMED = 0x800
QIEO_FLAG_SIXTEEN = 0x1000
QIEO_FLAG_NO_FIXED_WORDS = 0x2000
QIEO_FLAG_SPARSE_ALWAYS = 0x4000

# Every symbol include/qieo.h declares.
EXPORTS = (
    "qieo_default_params", "qieo_create_instance", "qieo_destroy_instance", "qieo_reset",
    "qieo_run", "qieo_set_wait_timeout", "qieo_synchronize", "qieo_get_best",
    "qieo_get_state", "qieo_get_fitness",
    "qieo_get_alleles", "qieo_get_allele_row", "qieo_get_elite_history", "qieo_get_threshold_table",
    "qieo_get_launch_shape", "qieo_set_launch_shape", "qieo_get_kernel_time",
    "qieo_get_phase_times", "qieo_get_generation_times", "qieo_measure_integer_ceiling",
    "qieo_get_drawn_vectors",
    "qieo_create_row_block", "qieo_rows_observe", "qieo_rows_rotate",
    "qieo_get_convergence", "qieo_checkpoint_size",
    "qieo_checkpoint_save", "qieo_checkpoint_load", "qieo_philox",
    "qieo_generation_noalloc", "qieo_create_batch", "qieo_batch_run", "qieo_destroy_batch",
    "qieo_run_batch", "qieo_autotune", "qieo_server_create", "qieo_server_submit", "qieo_server_poll",
    "qieo_server_get_stats", "qieo_server_cancel", "qieo_server_destroy", "qieo_last_error",
)

QIEO_SOLVE_QUEUED = 0
QIEO_SOLVE_RUNNING = 1
QIEO_SOLVE_DONE = 2
QIEO_SOLVE_CANCELLED = 3
QIEO_SOLVE_FAILED = 4

QIEO_NOALLOC_MAX_NP = 65536


class QieoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("qieo status %d: %s" % (status, msg))
        self.status = status


class qieo_problem(C.Structure):
    _fields_ = [("ng", C.c_int32), ("weights", C.c_void_p), ("values", C.c_void_p),
                ("capacity", C.c_int64)]


class qieo_params(C.Structure):
    _fields_ = [("np", C.c_int32), ("dtheta_den", C.c_int32), ("penalty_lambda", C.c_int64),
                ("seed", C.c_uint32), ("instance_id", C.c_uint32), ("rotate_rule", C.c_int32),
                ("elite_on_host", C.c_int32), ("flags", C.c_int32), ("stream", C.c_void_p)]


class qieo_launch_shape(C.Structure):
    _fields_ = [("lanes_per_row", C.c_int32), ("warps_per_row", C.c_int32),
                ("grid_ctas", C.c_int32), ("narrow", C.c_int32), ("tiles", C.c_int32),
                ("rows_per_cta", C.c_int32), ("persistent", C.c_int32), ("resident", C.c_int32),
                ("fixed_words", C.c_int32)]


class qieo_server_config(C.Structure):
    _fields_ = [("memory_bytes", C.c_int64), ("max_active", C.c_int32), ("gens_per_step", C.c_int32)]


class qieo_integer_ceiling(C.Structure):
    _fields_ = [("drawn_genes_per_s", C.c_double), ("philox_genes_per_s", C.c_double),
                ("genes_per_launch", C.c_int64), ("grid_ctas", C.c_int32), ("reps", C.c_int32)]


class qieo_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("steps", C.c_int64), ("kernel_launches", C.c_int64), ("queued", C.c_int32),
                ("active", C.c_int32), ("max_active", C.c_int32), ("reserved", C.c_int32)]


class qieo_solve_result(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("fitness", C.c_int64),
                ("generation", C.c_int32), ("chromosome", C.c_int32), ("submit_s", C.c_double),
                ("admit_s", C.c_double), ("done_s", C.c_double), ("generations_run", C.c_int32),
                ("converged", C.c_int32)]


_LIB: C.CDLL | None = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load libqieo.so (building it in-tree with nvcc if it is missing or stale)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if build_if_missing and _build.stale():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("QIEO CUDA library not built: %s is missing" % _build.LIB)
    L = C.CDLL(_build.LIB)
    P, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    sig = {
        "qieo_default_params": ([P], None),
        "qieo_create_instance": ([P, P, P], C.c_int),
        "qieo_destroy_instance": ([P], C.c_int),
        "qieo_reset": ([P], C.c_int),
        "qieo_run": ([P, i32], C.c_int),
        "qieo_set_wait_timeout": ([P, i64], C.c_int),
        "qieo_synchronize": ([P], C.c_int),
        "qieo_get_best": ([P, P, P, P, P], C.c_int),
        "qieo_get_state": ([P, P, P], C.c_int),
        "qieo_get_fitness": ([P, P], C.c_int),
        "qieo_get_alleles": ([P, P], C.c_int),
        "qieo_get_allele_row": ([P, i32, P], C.c_int),
        "qieo_get_elite_history": ([P, i32, i32, P, P], C.c_int),
        "qieo_get_threshold_table": ([P, P], C.c_int),
        "qieo_get_launch_shape": ([P, P], C.c_int),
        "qieo_set_launch_shape": ([P, P], C.c_int),
        "qieo_get_kernel_time": ([P, P, P], C.c_int),
        "qieo_get_phase_times": ([P, P, P], C.c_int),
        "qieo_get_generation_times": ([P, i32, P, P], C.c_int),
        "qieo_get_drawn_vectors": ([P, i32, i32, P], C.c_int),
        "qieo_measure_integer_ceiling": ([i32, P], C.c_int),
        "qieo_create_row_block": ([P, P, i32, P], C.c_int),
        "qieo_rows_observe": ([P, i32, P, P], C.c_int),
        "qieo_rows_rotate": ([P, P], C.c_int),
        "qieo_get_convergence": ([P, P, P], C.c_int),
        "qieo_checkpoint_size": ([P, P], C.c_int),
        "qieo_checkpoint_save": ([P, P, C.c_size_t], C.c_int),
        "qieo_checkpoint_load": ([P, P, C.c_size_t], C.c_int),
        "qieo_philox": ([P, P, i32], C.c_int),
        "qieo_generation_noalloc": ([P, P, i32, P, P, P, P], C.c_int),
        "qieo_create_batch": ([P, i32, P], C.c_int),
        "qieo_batch_run": ([P, i32], C.c_int),
        "qieo_destroy_batch": ([P], C.c_int),
        "qieo_run_batch": ([P, i32, i32], C.c_int),
        "qieo_autotune": ([P, i32, P], C.c_int),
        "qieo_server_create": ([P, P], C.c_int),
        "qieo_server_submit": ([P, P, P, i32, P], C.c_int),
        "qieo_server_poll": ([P, i64, i32, P, P], C.c_int),
        "qieo_server_get_stats": ([P, P], C.c_int),
        "qieo_server_cancel": ([P, i64], C.c_int),
        "qieo_server_destroy": ([P], C.c_int),
        "qieo_last_error": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _LIB = L
    return L


def _check(status: int) -> None:
    if status != QIEO_OK:
        raise QieoError(status, load().qieo_last_error().decode("utf8", "replace"))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def qieo_default_params() -> qieo_params:
    p = qieo_params()
    load().qieo_default_params(C.byref(p))
    return p


def qieo_create_instance(weights, values, capacity: int, params: qieo_params):
    """Returns an opaque handle (c_void_p). weights/values: int32 host arrays."""
    w = np.ascontiguousarray(weights, dtype=np.int32)
    v = np.ascontiguousarray(values, dtype=np.int32)
    if w.shape != v.shape or w.ndim != 1:
        raise ValueError("weights and values must be 1-D arrays of equal length")
    pr = qieo_problem(int(w.shape[0]), w.ctypes.data, v.ctypes.data, int(capacity))
    h = C.c_void_p()
    _check(load().qieo_create_instance(C.byref(pr), C.byref(params), C.byref(h)))
    return h


def qieo_create_row_block(weights, values, capacity: int, params: qieo_params, row0: int):
    """Returns an opaque handle of a row block (rows row0 .. row0 + params.np - 1)."""
    w = np.ascontiguousarray(weights, dtype=np.int32)
    v = np.ascontiguousarray(values, dtype=np.int32)
    if w.shape != v.shape or w.ndim != 1:
        raise ValueError("weights and values must be 1-D arrays of equal length")
    pr = qieo_problem(int(w.shape[0]), w.ctypes.data, v.ctypes.data, int(capacity))
    h = C.c_void_p()
    _check(load().qieo_create_row_block(C.byref(pr), C.byref(params), int(row0), C.byref(h)))
    return h


def qieo_rows_observe(h, t: int):
    f, c = C.c_int64(), C.c_int32()
    _check(load().qieo_rows_observe(h, int(t), C.byref(f), C.byref(c)))
    return int(f.value), int(c.value)


def qieo_rows_rotate(h, elite_bits) -> None:
    e = np.ascontiguousarray(elite_bits, dtype=np.uint8)
    _check(load().qieo_rows_rotate(h, _ptr(e)))


def qieo_destroy_instance(h) -> None:
    _check(load().qieo_destroy_instance(h))


def qieo_reset(h) -> None:
    _check(load().qieo_reset(h))


def qieo_run(h, generations: int) -> None:
    _check(load().qieo_run(h, int(generations)))


def qieo_set_wait_timeout(h, ns: int) -> None:
    _check(load().qieo_set_wait_timeout(h, int(ns)))


def qieo_synchronize(h) -> None:
    _check(load().qieo_synchronize(h))


def qieo_get_best(h, ng: int):
    bits = np.zeros(ng, dtype=np.uint8)
    f, g, c = C.c_int64(), C.c_int32(), C.c_int32()
    _check(load().qieo_get_best(h, _ptr(bits), C.byref(f), C.byref(g), C.byref(c)))
    return bits, int(f.value), int(g.value), int(c.value)


def qieo_get_state(h, np_: int, ng: int):
    k = np.zeros((np_, ng), dtype=np.int16)
    t = C.c_int32()
    _check(load().qieo_get_state(h, _ptr(k), C.byref(t)))
    return k, int(t.value)


def qieo_get_fitness(h, np_: int) -> np.ndarray:
    f = np.zeros(np_, dtype=np.int64)
    _check(load().qieo_get_fitness(h, _ptr(f)))
    return f


def qieo_get_alleles(h, np_: int, ng: int) -> np.ndarray:
    x = np.zeros((np_, ng), dtype=np.uint8)
    _check(load().qieo_get_alleles(h, _ptr(x)))
    return x


def qieo_get_allele_row(h, c: int, ng: int) -> np.ndarray:
    x = np.zeros(ng, dtype=np.uint8)
    _check(load().qieo_get_allele_row(h, int(c), _ptr(x)))
    return x


def qieo_get_elite_history(h, first: int, n: int):
    e = np.zeros(n, dtype=np.int32)
    f = np.zeros(n, dtype=np.int64)
    _check(load().qieo_get_elite_history(h, int(first), int(n), _ptr(e), _ptr(f)))
    return e, f


def qieo_get_threshold_table(h, D: int) -> np.ndarray:
    T = np.zeros(2 * (D // 4) + 1, dtype=np.uint64)
    _check(load().qieo_get_threshold_table(h, _ptr(T)))
    return T


def qieo_get_launch_shape(h) -> qieo_launch_shape:
    s = qieo_launch_shape()
    _check(load().qieo_get_launch_shape(h, C.byref(s)))
    return s


def qieo_set_launch_shape(h, lanes_per_row: int, warps_per_row: int, grid_ctas: int = 0) -> None:
    s = qieo_launch_shape(int(lanes_per_row), int(warps_per_row), int(grid_ctas), 0, 0, 0, 0)
    _check(load().qieo_set_launch_shape(h, C.byref(s)))


def qieo_get_phase_times(h):
    """({CIP, QIP, Evaluation, DetermineElite} ms, generations covered)."""
    ms = (C.c_double * 4)()
    n = C.c_int64()
    _check(load().qieo_get_phase_times(h, ms, C.byref(n)))
    return {"cip": ms[0], "qip": ms[1], "evaluation": ms[2], "determine_elite": ms[3]}, int(n.value)


def qieo_get_convergence(h):
    """(stopped, stable generations) of an instance created with QIEO_FLAG_CONVERGE."""
    a, b = C.c_int32(), C.c_int32()
    _check(load().qieo_get_convergence(h, C.byref(a), C.byref(b)))
    return bool(a.value), int(b.value)


def qieo_checkpoint_save(h) -> bytes:
    """The instance's checkpoint as bytes."""
    n = C.c_size_t()
    _check(load().qieo_checkpoint_size(h, C.byref(n)))
    buf = C.create_string_buffer(n.value)
    _check(load().qieo_checkpoint_save(h, buf, n.value))
    return buf.raw


def qieo_checkpoint_load(h, data: bytes) -> None:
    buf = C.create_string_buffer(bytes(data), len(data))
    _check(load().qieo_checkpoint_load(h, buf, len(data)))


def qieo_get_kernel_time(h):
    ms, n = C.c_double(), C.c_int64()
    _check(load().qieo_get_kernel_time(h, C.byref(ms), C.byref(n)))
    return float(ms.value), int(n.value)


def qieo_get_drawn_vectors(h, first: int, n: int) -> np.ndarray:
    out = np.zeros(max(int(n), 0), dtype=np.int64)
    _check(load().qieo_get_drawn_vectors(h, int(first), int(n), _ptr(out)))
    return out


def qieo_get_generation_times(h, n: int) -> np.ndarray:
    ms = np.zeros(max(0, int(n)), dtype=np.float32)
    cnt = C.c_int32()
    _check(load().qieo_get_generation_times(h, int(n), _ptr(ms), C.byref(cnt)))
    return ms[:cnt.value]


def qieo_measure_integer_ceiling(reps: int = 5) -> qieo_integer_ceiling:
    out = qieo_integer_ceiling()
    _check(load().qieo_measure_integer_ceiling(int(reps), C.byref(out)))
    return out


def qieo_philox(ctr_key) -> np.ndarray:
    ck = np.ascontiguousarray(ctr_key, dtype=np.uint32).reshape(-1, 6)
    out = np.zeros((ck.shape[0], 4), dtype=np.uint32)
    _check(load().qieo_philox(_ptr(ck), _ptr(out), int(ck.shape[0])))
    return out


def qieo_generation_noalloc(d_weights: int, d_values: int, ng: int, capacity: int,
                            params: qieo_params, t: int, d_k: int, d_x: int, d_fitness: int,
                            d_elite: int) -> None:
    """One generation on caller-owned device buffers (all pointer arguments are device
    addresses, e.g. torch.Tensor.data_ptr()); allocates nothing."""
    pr = qieo_problem(int(ng), int(d_weights), int(d_values), int(capacity))
    _check(load().qieo_generation_noalloc(C.byref(pr), C.byref(params), int(t), int(d_k),
                                          int(d_x), int(d_fitness), int(d_elite)))


def qieo_create_batch(handles) -> C.c_void_p:
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    b = C.c_void_p()
    _check(load().qieo_create_batch(arr, len(handles), C.byref(b)))
    return b


def qieo_batch_run(b, generations: int) -> None:
    _check(load().qieo_batch_run(b, int(generations)))


def qieo_destroy_batch(b) -> None:
    _check(load().qieo_destroy_batch(b))


def qieo_run_batch(instances, generations: int) -> None:
    """One call: a temporary batch over the Instance objects, `generations` generations."""
    hs = [i.h for i in instances]
    arr = (C.c_void_p * len(hs))(*[h.value if isinstance(h, C.c_void_p) else h for h in hs])
    _check(load().qieo_run_batch(arr, len(hs), int(generations)))


def qieo_autotune(h, trial_generations: int) -> qieo_launch_shape:
    s = qieo_launch_shape()
    _check(load().qieo_autotune(h, int(trial_generations), C.byref(s)))
    return s


def qieo_server_create(memory_bytes: int = 0, max_active: int = 0, gens_per_step: int = 0):
    cfg = qieo_server_config(int(memory_bytes), int(max_active), int(gens_per_step))
    h = C.c_void_p()
    _check(load().qieo_server_create(C.byref(cfg), C.byref(h)))
    return h


def qieo_server_submit(h, weights, values, capacity: int, params: qieo_params, generations: int) -> int:
    w = np.ascontiguousarray(weights, dtype=np.int32)
    v = np.ascontiguousarray(values, dtype=np.int32)
    pr = qieo_problem(int(w.shape[0]), w.ctypes.data, v.ctypes.data, int(capacity))
    rid = C.c_int64()
    _check(load().qieo_server_submit(h, C.byref(pr), C.byref(params), int(generations), C.byref(rid)))
    return int(rid.value)


def qieo_server_poll(h, rid: int, wait_ms: int = 0, ng: int = 0):
    res = qieo_solve_result()
    bits = np.zeros(max(ng, 1), dtype=np.uint8)
    _check(load().qieo_server_poll(h, int(rid), int(wait_ms), _ptr(bits) if ng else None,
                                   C.byref(res)))
    return res, (bits[:ng] if ng else None)


def qieo_server_get_stats(h) -> qieo_server_stats:
    st = qieo_server_stats()
    _check(load().qieo_server_get_stats(h, C.byref(st)))
    return st


def qieo_server_cancel(h, rid: int) -> None:
    _check(load().qieo_server_cancel(h, int(rid)))


def qieo_server_destroy(h) -> None:
    _check(load().qieo_server_destroy(h))


class Server:
    """Owner of a solve server handle."""

    def __init__(self, memory_bytes: int = 0, max_active: int = 0, gens_per_step: int = 0):
        self.h = qieo_server_create(memory_bytes, max_active, gens_per_step)
        self.ng = {}

    def submit(self, problem, np_: int, generations: int, seed: int = 1, inst: int = 0,
               D: int = 100, lam: int = 1, rule: int = QIEO_RULE_R1, flags: int = 0) -> int:
        p = qieo_default_params()
        p.np, p.seed, p.instance_id = int(np_), int(seed) & 0xFFFFFFFF, int(inst) & 0xFFFFFFFF
        p.dtheta_den, p.penalty_lambda, p.rotate_rule = int(D), int(lam), int(rule)
        p.flags = int(flags)
        rid = qieo_server_submit(self.h, problem.weights, problem.values, problem.capacity, p,
                                 generations)
        self.ng[rid] = int(problem.ng)
        return rid

    def poll(self, rid: int, wait_ms: int = 0):
        return qieo_server_poll(self.h, rid, wait_ms, self.ng.get(rid, 0))

    def cancel(self, rid: int) -> None:
        qieo_server_cancel(self.h, rid)

    def stats(self) -> dict:
        st = qieo_server_get_stats(self.h)
        return {name: getattr(st, name) for name, _ in st._fields_ if name != "reserved"}

    def close(self) -> None:
        if getattr(self, "h", None) is not None:
            qieo_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Owner of a batch handle over Instance objects (which must outlive it)."""

    def __init__(self, instances):
        self.instances = list(instances)
        self.h = qieo_create_batch([i.h for i in self.instances])

    def run(self, generations: int) -> None:
        qieo_batch_run(self.h, generations)

    def close(self) -> None:
        if getattr(self, "h", None) is not None:
            qieo_destroy_batch(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Instance:
    """Convenience owner of one instance handle (destroyed on close / garbage collection).
    row0 >= 0 makes it a row block (qieo_create_row_block) of np_ rows starting at row0."""

    def __init__(self, problem, np_: int, seed: int = 1, inst: int = 0, D: int = 100,
                 lam: int = 1, rule: int = QIEO_RULE_R1, elite_on_host: int = 0,
                 flags: int = 0, stream: int | None = None, row0: int | None = None):
        p = qieo_default_params()
        p.np = int(np_)
        p.dtheta_den = int(D)
        p.penalty_lambda = int(lam)
        p.seed = int(seed) & 0xFFFFFFFF
        p.instance_id = int(inst) & 0xFFFFFFFF
        p.rotate_rule = int(rule)
        p.elite_on_host = int(elite_on_host)
        p.flags = int(flags)
        p.stream = stream
        self.np_, self.ng, self.D = int(np_), int(problem.ng), int(D)
        if row0 is None:
            self.h = qieo_create_instance(problem.weights, problem.values, problem.capacity, p)
        else:
            self.h = qieo_create_row_block(problem.weights, problem.values, problem.capacity, p, row0)

    def close(self) -> None:
        if getattr(self, "h", None) is not None:
            qieo_destroy_instance(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def run(self, generations: int) -> None:
        qieo_run(self.h, generations)

    def reset(self) -> None:
        qieo_reset(self.h)

    def synchronize(self) -> None:
        qieo_synchronize(self.h)

    def set_wait_timeout(self, ns: int) -> None:
        qieo_set_wait_timeout(self.h, ns)

    def best(self):
        return qieo_get_best(self.h, self.ng)

    def state(self):
        return qieo_get_state(self.h, self.np_, self.ng)

    def fitness(self) -> np.ndarray:
        return qieo_get_fitness(self.h, self.np_)

    def alleles(self) -> np.ndarray:
        return qieo_get_alleles(self.h, self.np_, self.ng)

    def allele_row(self, c: int) -> np.ndarray:
        return qieo_get_allele_row(self.h, c, self.ng)

    def history(self, first: int, n: int):
        return qieo_get_elite_history(self.h, first, n)

    def thresholds(self) -> np.ndarray:
        return qieo_get_threshold_table(self.h, self.D)

    def shape(self) -> qieo_launch_shape:
        return qieo_get_launch_shape(self.h)

    def set_shape(self, lanes_per_row: int, warps_per_row: int, grid_ctas: int = 0) -> None:
        qieo_set_launch_shape(self.h, lanes_per_row, warps_per_row, grid_ctas)

    def kernel_time(self):
        return qieo_get_kernel_time(self.h)

    def rows_observe(self, t: int):
        return qieo_rows_observe(self.h, t)

    def rows_rotate(self, elite_bits) -> None:
        qieo_rows_rotate(self.h, elite_bits)

    def generation_times(self, n: int) -> np.ndarray:
        return qieo_get_generation_times(self.h, n)

    def drawn_vectors(self, first: int, n: int) -> np.ndarray:
        """Per generation first .. first + n - 1, the 8-gene vectors that drew (observed by
        Philox draws) in an instance that keeps fixed-vector bits: every vector in a dense
        generation, only the unstable ones in a sparse generation."""
        return qieo_get_drawn_vectors(self.h, first, n)

    def phase_times(self):
        return qieo_get_phase_times(self.h)

    def convergence(self):
        return qieo_get_convergence(self.h)

    def save(self) -> bytes:
        return qieo_checkpoint_save(self.h)

    def load(self, data: bytes) -> None:
        qieo_checkpoint_load(self.h, data)

    def autotune(self, trial_generations: int = 8) -> qieo_launch_shape:
        return qieo_autotune(self.h, trial_generations)
