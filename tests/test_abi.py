"""The C-ABI library builds, loads and exports every entry point include/qieo.h declares,
and the binding's structures match the header's layout (no GPU needed: nothing here
launches a kernel)."""
import os
import re
import shutil
import subprocess
import tempfile

import pytest

from paper_2609_30862_gb300 import build as B
from paper_2609_30862_gb300 import qieo as Q

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qieo.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qieo_[a-z_]+)\s*\(", text)))


def test_header_and_binding_agree():
    assert _declared() == sorted(Q.EXPORTS)


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc unavailable")
    B.build()
    return Q.load()


def test_library_exports_every_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (qieo_\w+)", out))
    for name in _declared():
        assert name in exported, name
        assert hasattr(lib, name)


def test_defaults_and_errors_without_gpu(lib):
    p = Q.qieo_default_params()
    assert (p.np, p.dtheta_den, p.penalty_lambda, p.seed, p.rotate_rule) == (64, 100, 1, 1, 0)
    # invalid arguments are rejected on the host before any device call
    with pytest.raises(Q.QieoError) as e:
        Q.qieo_create_instance([1, 2], [3, 4], 2, _params(p, dtheta_den=30))
    assert e.value.status == Q.QIEO_ERR_INVALID and "dtheta_den" in str(e.value)
    with pytest.raises(Q.QieoError) as e:
        Q.qieo_create_instance([1, -2], [3, 4], 2, p)
    assert e.value.status == Q.QIEO_ERR_INVALID
    with pytest.raises(Q.QieoError):
        Q.qieo_create_instance([1, 2], [3, 4], 2, _params(p, np=0))
    with pytest.raises(Q.QieoError):
        Q.qieo_create_instance([1, 2], [3, 4], 2, _params(p, penalty_lambda=0))
    with pytest.raises(Q.QieoError):
        Q.qieo_create_instance([1, 2], [3, 4], -1, p)
    with pytest.raises(Q.QieoError):
        Q.qieo_create_instance([2**31 - 1] * 4, [1] * 4, 1, _params(p, penalty_lambda=2**32))
    with pytest.raises(Q.QieoError) as e:
        Q.qieo_create_instance([1, 2], [3, 4], 2, _params(p, flags=Q.QIEO_FLAG_UNFUSED, elite_on_host=1))
    assert e.value.status == Q.QIEO_ERR_INVALID and "UNFUSED" in str(e.value)
    with pytest.raises(Q.QieoError) as e:
        Q.qieo_create_instance([1, 2], [3, 4], 2,
                               _params(p, flags=Q.QIEO_FLAG_UNFUSED | Q.QIEO_FLAG_COOPERATIVE))
    assert e.value.status == Q.QIEO_ERR_INVALID
    for bad in (dict(flags=Q.QIEO_FLAG_STATE_I8, dtheta_den=124),
                dict(flags=Q.QIEO_FLAG_STATE_I8 | Q.QIEO_FLAG_REGISTER_PREFETCH)):
        with pytest.raises(Q.QieoError) as e:
            Q.qieo_create_instance([1, 2], [3, 4], 2, _params(p, **bad))
        assert e.value.status == Q.QIEO_ERR_INVALID and "STATE_I8" in str(e.value)
    for bad in (dict(flags=Q.QIEO_FLAG_CONVERGE, elite_on_host=1),
                dict(flags=Q.QIEO_FLAG_CONVERGE | Q.QIEO_FLAG_UNFUSED),
                dict(flags=Q.QIEO_FLAG_CONVERGE | Q.QIEO_FLAG_COOPERATIVE)):
        with pytest.raises(Q.QieoError) as e:
            Q.qieo_create_instance([1, 2], [3, 4], 2, _params(p, **bad))
        assert e.value.status == Q.QIEO_ERR_INVALID and "CONVERGE" in str(e.value)
    with pytest.raises(Q.QieoError) as e:
        Q.qieo_run(None, 1)
    assert e.value.status == Q.QIEO_ERR_INVALID
    # the entry points added for measurement and for sharded populations check their
    # arguments on the host before any device call
    for reps in (0, 1001):
        with pytest.raises(Q.QieoError) as e:
            Q.qieo_measure_integer_ceiling(reps)
        assert e.value.status == Q.QIEO_ERR_INVALID and "reps" in str(e.value)
    for call in (lambda: Q.qieo_get_generation_times(None, 4), lambda: Q.qieo_rows_observe(None, 0),
                 lambda: Q.qieo_rows_rotate(None, [0, 1]), lambda: Q.qieo_get_allele_row(None, 0, 4),
                 lambda: Q.qieo_get_drawn_vectors(None, 0, 4)):
        with pytest.raises(Q.QieoError) as e:
            call()
        assert e.value.status == Q.QIEO_ERR_INVALID
    for bad in (dict(row0=-1), dict(row0=0, elite_on_host=1), dict(row0=0, flags=Q.QIEO_FLAG_CONVERGE),
                dict(row0=0, flags=Q.QIEO_FLAG_UNFUSED)):
        kw = dict(bad)
        row0 = kw.pop("row0")
        with pytest.raises(Q.QieoError) as e:
            Q.qieo_create_row_block([1, 2], [3, 4], 2, _params(p, **kw), row0)
        assert e.value.status == Q.QIEO_ERR_INVALID
    for bad in (dict(flags=Q.QIEO_FLAG_TIME_GENERATIONS, elite_on_host=1),
                dict(flags=Q.QIEO_FLAG_TIME_GENERATIONS | Q.QIEO_FLAG_UNFUSED)):
        with pytest.raises(Q.QieoError) as e:
            Q.qieo_create_instance([1, 2], [3, 4], 2, _params(p, **bad))
        assert e.value.status == Q.QIEO_ERR_INVALID and "TIME_GENERATIONS" in str(e.value)


def _params(p, **kw):
    q = Q.qieo_params()
    for name, _ in Q.qieo_params._fields_:
        setattr(q, name, getattr(p, name))
    for k, v in kw.items():
        setattr(q, k, v)
    return q


_LAYOUT_PROG = r"""
#include <stdio.h>
#include <stddef.h>
#include "qieo.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(qieo_problem), sizeof(qieo_params),
         sizeof(qieo_launch_shape), offsetof(qieo_params, stream), offsetof(qieo_problem, capacity));
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(qieo_server_config), sizeof(qieo_solve_result),
         offsetof(qieo_solve_result, submit_s), offsetof(qieo_solve_result, converged), sizeof(qieo_server_stats),
         offsetof(qieo_server_stats, queued), offsetof(qieo_server_stats, max_active));
  return 0;
}
"""


def test_struct_layout_matches_header():
    if shutil.which("gcc") is None:
        pytest.skip("gcc unavailable")
    import ctypes as C
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "l.c")
        open(src, "w").write(_LAYOUT_PROG)
        exe = os.path.join(d, "l")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        got = [int(x) for x in subprocess.check_output([exe]).split()]
    want = [C.sizeof(Q.qieo_problem), C.sizeof(Q.qieo_params), C.sizeof(Q.qieo_launch_shape),
            Q.qieo_params.stream.offset, Q.qieo_problem.capacity.offset,
            C.sizeof(Q.qieo_server_config), C.sizeof(Q.qieo_solve_result),
            Q.qieo_solve_result.submit_s.offset, Q.qieo_solve_result.converged.offset,
            C.sizeof(Q.qieo_server_stats),
            Q.qieo_server_stats.queued.offset, Q.qieo_server_stats.max_active.offset]
    assert got == want
