"""ctypes wrapper of the CPU oracle (qieo_oracle.c).

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT: only the tests, the package smoke check and
the benchmark's CPU-baseline leg import this module. It shares nothing with the GPU
library and imports nothing from it; inputs arrive as plain numpy arrays.

Two builds of the same C file: `serial` (single thread, the oracle proper) and `omp`
(chromosome loops under OpenMP; identical results, used to reach full-size workloads
and to time the host at all cores).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qieo_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIBS: dict[str, C.CDLL] = {}
_LOCK = threading.Lock()


def lib_path(kind: str = "serial") -> str:
    return os.path.join(_BUILD, "libqieo_oracle_omp.so" if kind == "omp" else "libqieo_oracle.so")


def build(force: bool = False) -> None:
    """Compile both builds with gcc (seconds). Plain -O2, no machine-specific flags."""
    os.makedirs(_BUILD, exist_ok=True)
    for kind, extra in (("serial", []), ("omp", ["-fopenmp"])):
        out = lib_path(kind)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        tmp = out + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", *extra,
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, out)


def _lib(kind: str = "serial") -> C.CDLL:
    with _LOCK:
        if kind not in _LIBS:
            if not os.path.exists(lib_path(kind)) or \
                    os.path.getmtime(lib_path(kind)) < os.path.getmtime(_SRC):
                build()
            L = C.CDLL(lib_path(kind))
            P = C.c_void_p
            i32, i64, u32 = C.c_int32, C.c_int64, C.c_uint32
            L.qo_philox4x32_10.argtypes = [P, P, P]
            L.qo_philox4x32_10.restype = None
            L.qo_threshold_table.argtypes = [i32, P]
            L.qo_threshold_table.restype = C.c_int
            L.qo_observe.argtypes = [i32, u32, P]
            L.qo_observe.restype = C.c_int
            L.qo_fitness.argtypes = [i32, P, P, i64, i64, P]
            L.qo_fitness.restype = i64
            L.qo_determine_elite.argtypes = [i32, P]
            L.qo_determine_elite.restype = i32
            L.qo_bruteforce.argtypes = [i32, P, P, i64, i64, P]
            L.qo_bruteforce.restype = i64
            L.qo_run.argtypes = [i32, P, P, i64, i32, i32, i64, u32, u32, i32, i32,
                                 P, P, P, P, P, P, P, P]
            L.qo_run.restype = C.c_int
            L.qo_run_converge.argtypes = [i32, P, P, i64, i32, i32, i64, u32, u32, i32, i32,
                                          P, P, P, P, P, P, P, P, i32, P, P]
            L.qo_run_converge.restype = C.c_int
            L.qo_run_fp64.argtypes = [i32, P, P, i64, i32, i32, i64, u32, u32, i32, i32,
                                      P, P, P, P, P, P, P, P, P, P, P]
            L.qo_run_fp64.restype = C.c_int
            L.qo_rows_observe.argtypes = [i32, P, P, i64, i32, i64, u32, u32, i32, i32, i32,
                                          P, P, P]
            L.qo_rows_observe.restype = C.c_int
            L.qo_rows_rotate.argtypes = [i32, i32, i32, i32, P, P, P]
            L.qo_rows_rotate.restype = C.c_int
            L.qo_set_threads.argtypes = [i32]
            L.qo_set_threads.restype = C.c_int
            L.qo_is_openmp.argtypes = []
            L.qo_is_openmp.restype = C.c_int
            _LIBS[kind] = L
        return _LIBS[kind]


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _lib().qo_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def threshold_table(D: int) -> np.ndarray:
    T = np.zeros(2 * (D // 4) + 1, dtype=np.uint64)
    if _lib().qo_threshold_table(D, _p(T)) != 0:
        raise ValueError("D must be a positive multiple of 4")
    return T


def observe(n: int, u: int, T: np.ndarray) -> int:
    T = np.ascontiguousarray(T, dtype=np.uint64)
    return int(_lib().qo_observe(int(n), int(u), _p(T)))


def fitness(x, w, v, W: int, lam: int = 1) -> int:
    x = np.ascontiguousarray(x, dtype=np.uint8)
    w = np.ascontiguousarray(w, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.int32)
    return int(_lib().qo_fitness(int(w.shape[0]), _p(w), _p(v), int(W), int(lam), _p(x)))


def determine_elite(f) -> int:
    f = np.ascontiguousarray(f, dtype=np.int64)
    return int(_lib().qo_determine_elite(int(f.shape[0]), _p(f)))


def bruteforce(w, v, W: int, lam: int = 1):
    w = np.ascontiguousarray(w, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.int32)
    x = np.zeros(w.shape[0], dtype=np.uint8)
    best = int(_lib().qo_bruteforce(int(w.shape[0]), _p(w), _p(v), int(W), int(lam), _p(x)))
    return best, x


def rows_observe(problem, k_rows, gen: int, c0: int, seed: int = 1, inst: int = 0,
                 D: int = 100, lam: int = 1):
    """QIP + Evaluation of rows c0 .. c0 + nr of a population (k_rows[nr, ng]); returns
    (x[nr, ng], f[nr]). Draws use the global chromosome index."""
    k = np.ascontiguousarray(k_rows, dtype=np.int16)
    nr, ng = k.shape
    w = np.ascontiguousarray(problem.weights, dtype=np.int32)
    v = np.ascontiguousarray(problem.values, dtype=np.int32)
    x = np.zeros((nr, ng), dtype=np.uint8)
    f = np.zeros(nr, dtype=np.int64)
    if _lib().qo_rows_observe(ng, _p(w), _p(v), int(problem.capacity), int(D), int(lam),
                              int(seed) & 0xFFFFFFFF, int(inst) & 0xFFFFFFFF, int(gen), int(c0),
                              int(nr), _p(k), _p(x), _p(f)) != 0:
        raise ValueError("invalid arguments")
    return x, f


def rows_rotate(k_rows: np.ndarray, x_rows, x_elite, D: int = 100, rule: int = 0) -> None:
    """CIP of a row block toward the elite's alleles, in place on k_rows[nr, ng] (int16)."""
    assert k_rows.dtype == np.int16 and k_rows.flags.c_contiguous
    nr, ng = k_rows.shape
    x = np.ascontiguousarray(x_rows, dtype=np.uint8)
    xe = np.ascontiguousarray(x_elite, dtype=np.uint8)
    if _lib().qo_rows_rotate(ng, int(D), int(rule), nr, _p(k_rows), _p(x), _p(xe)) != 0:
        raise ValueError("invalid arguments")


class State:
    """Oracle state of one instance: angle indices k[np, ng], next generation t, the
    best-so-far record, and what the last generation produced."""

    def __init__(self, np_: int, ng: int):
        self.np_, self.ng = np_, ng
        self.k = np.zeros((np_, ng), dtype=np.int16)
        self.t = np.zeros(1, dtype=np.int32)
        self.best = np.array([0, -1, -1], dtype=np.int64)      # fitness, generation, chromosome
        self.best_x = np.zeros(ng, dtype=np.uint8)
        self.x = np.zeros((np_, ng), dtype=np.uint8)
        self.f = np.zeros(np_, dtype=np.int64)
        self.hist_e = np.zeros(0, dtype=np.int32)
        self.hist_f = np.zeros(0, dtype=np.int64)
        # convergence test: run length of equal elite fitness, stopped flag, that fitness
        self.conv = np.zeros(3, dtype=np.int64)

    @property
    def stopped(self) -> bool:
        return bool(self.conv[1])

    def copy(self) -> "State":
        s = State.__new__(State)
        for name, val in self.__dict__.items():
            setattr(s, name, val.copy() if isinstance(val, np.ndarray) else val)
        return s


def run(problem, np_: int, gens: int, seed: int = 1, inst: int = 0, D: int = 100,
        lam: int = 1, rule: int = 0, state: State | None = None, kind: str = "serial",
        threads: int = 0, window: int = 0) -> State:
    """Run `gens` generations of the angle-index form from `state` (a fresh instance if
    None) and return the updated state. `problem` has .weights, .values, .capacity.
    window > 0: stop once the elite fitness has been equal for `window` consecutive
    generations (then `gens` is the cap and the history holds the generations run)."""
    w = np.ascontiguousarray(problem.weights, dtype=np.int32)
    v = np.ascontiguousarray(problem.values, dtype=np.int32)
    ng = int(w.shape[0])
    st = state if state is not None else State(np_, ng)
    he = np.zeros(gens, dtype=np.int32)
    hf = np.zeros(gens, dtype=np.int64)
    L = _lib(kind)
    if kind == "omp":
        L.qo_set_threads(int(threads) if threads else (os.cpu_count() or 1))
    if window > 0:
        done = np.zeros(1, dtype=np.int32)
        rc = L.qo_run_converge(ng, _p(w), _p(v), int(problem.capacity), np_, D, lam,
                               seed & 0xFFFFFFFF, inst & 0xFFFFFFFF, rule, gens, _p(st.k),
                               _p(st.t), _p(st.best), _p(st.best_x), _p(st.x), _p(st.f), _p(he),
                               _p(hf), int(window), _p(st.conv), _p(done))
        n = int(done[0])
    else:
        rc = L.qo_run(ng, _p(w), _p(v), int(problem.capacity), np_, D, lam, seed & 0xFFFFFFFF,
                      inst & 0xFFFFFFFF, rule, gens, _p(st.k), _p(st.t), _p(st.best),
                      _p(st.best_x), _p(st.x), _p(st.f), _p(he), _p(hf))
        n = gens
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    st.hist_e = np.concatenate([st.hist_e, he[:n]])
    st.hist_f = np.concatenate([st.hist_f, hf[:n]])
    return st


def run_fp64(problem, np_: int, gens: int, seed: int = 1, inst: int = 0, D: int = 100,
             lam: int = 1, rule: int = 0):
    """Amplitude-form run from a fresh instance. Returns a dict with alpha, beta, x, f,
    hist_e, hist_f, best, best_x, near_ties, max_norm_err."""
    w = np.ascontiguousarray(problem.weights, dtype=np.int32)
    v = np.ascontiguousarray(problem.values, dtype=np.int32)
    ng = int(w.shape[0])
    a = np.full((np_, ng), 1.0 / np.sqrt(2.0))
    b = np.full((np_, ng), 1.0 / np.sqrt(2.0))
    t = np.zeros(1, dtype=np.int32)
    best = np.array([0, -1, -1], dtype=np.int64)
    best_x = np.zeros(ng, dtype=np.uint8)
    x = np.zeros((np_, ng), dtype=np.uint8)
    f = np.zeros(np_, dtype=np.int64)
    he = np.zeros(gens, dtype=np.int32)
    hf = np.zeros(gens, dtype=np.int64)
    stats = np.zeros(1, dtype=np.int64)
    stats_d = np.zeros(1, dtype=np.float64)
    rc = _lib().qo_run_fp64(ng, _p(w), _p(v), int(problem.capacity), np_, D, lam,
                            seed & 0xFFFFFFFF, inst & 0xFFFFFFFF, rule, gens, _p(a), _p(b),
                            _p(t), _p(best), _p(best_x), _p(x), _p(f), _p(he), _p(hf),
                            _p(stats), _p(stats_d))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return dict(alpha=a, beta=b, x=x, f=f, hist_e=he, hist_f=hf, best=best, best_x=best_x,
                t=int(t[0]), near_ties=int(stats[0]), max_norm_err=float(stats_d[0]))


def set_threads(n: int) -> int:
    return int(_lib("omp").qo_set_threads(int(n)))
