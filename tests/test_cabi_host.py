"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function include/ecodp.h declares, and rejects
malformed descriptors before touching the device.  Also checks that the
product package never reaches into the oracle."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2104_01284_gb300 import problems as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_2104_01284_gb300 import build
    build.build()
    import paper_2104_01284_gb300.native as N
    return N


def declared_functions():
    hdr = open(os.path.join(ROOT, "include", "ecodp.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(dp_[a-z0-9_]+)\s*\(", hdr)))


def test_exports_every_declared_function(native):
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(native.lib, n), n
    assert set(native.EXPORTED) == set(names)


def test_checked_build_exports_the_same_functions(native):
    """The bounds-checked variant (ECODP_CHECKS) exports the same C ABI and
    reports itself as checked; the production build reports unchecked.
    Neither query touches the device."""
    from paper_2104_01284_gb300 import build
    path = build.build(checks=True)
    chk = C.CDLL(path)
    for n in declared_functions():
        assert hasattr(chk, n), n
    for lib_, want in ((native.lib, 0), (chk, 1)):
        en = C.c_int32(-1)
        assert lib_.dp_debug_checks(C.byref(en), None) == 0
        assert en.value == want


def test_status_strings(native):
    assert native.lib.dp_status_string(0) == b"DP_OK"
    assert native.lib.dp_status_string(4) == b"DP_ERR_INFEASIBLE"


@pytest.mark.parametrize("field,value", [
    ("n_v", 1), ("n_soc", 0), ("n_t", 1), ("n_brake", 3), ("n_te", 0), ("mass", -1.0), ("eta_motor", 1.5),
    ("gamma", 2.0), ("ds", 0.0), ("t_hi", -5.0), ("r0", float("nan")), ("te_lo", -10.0),
])
def test_create_rejects_bad_descriptors(native, field, value):
    from paper_2104_01284_gb300.solver import make_desc
    p = P.config0().replace(**{field: value})
    d, keep = make_desc(p)
    h = C.c_void_p()
    st = native.dp_problem_create(C.byref(d), None, None, C.byref(h))
    assert st == native.DP_ERR_INVALID_ARG
    assert h.value is None
    assert native.lib.dp_last_error()


@pytest.mark.parametrize("lights", [
    dict(light_stage=np.array([0], np.int32)),            # node 0
    dict(light_stage=np.array([10], np.int32)),           # node N
    dict(light_stage=np.array([3, 3], np.int32), cycle=np.array([30.0, 30.0]), red=np.array([5.0, 5.0]),
         offset=np.array([0.0, 0.0])),                     # duplicate
    dict(red=np.array([40.0])),                            # red longer than the cycle
])
def test_create_rejects_bad_lights(native, lights):
    from paper_2104_01284_gb300.solver import make_desc
    p = P.config0().replace(**lights)
    d, keep = make_desc(p)
    h = C.c_void_p()
    assert native.dp_problem_create(C.byref(d), None, None, C.byref(h)) == native.DP_ERR_INVALID_ARG


def test_too_many_controls(native):
    from paper_2104_01284_gb300.solver import make_desc
    p = P.config0().replace(n_te=200, n_tm=100, n_brake=2)
    d, keep = make_desc(p)
    h = C.c_void_p()
    assert native.dp_problem_create(C.byref(d), None, None, C.byref(h)) == native.DP_ERR_INVALID_ARG


def test_product_code_never_uses_the_oracle():
    pkg = os.path.join(ROOT, "paper_2104_01284_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f
                assert "ecodp_oracle" not in src, f


def test_multi_create_rejects_bad_instance(native):
    from paper_2104_01284_gb300.solver import make_desc
    probs = P.config3_small(seed=35, n_instances=3)
    probs[2] = probs[2].replace(n_soc=1)
    descs = (native.ProblemDesc * 3)()
    keep = []
    for b, p in enumerate(probs):
        d, k = make_desc(p)
        descs[b] = d
        keep.append(k)
    h = C.c_void_p()
    st = native.dp_multi_create(descs, 3, None, None, None, C.byref(h))
    assert st == native.DP_ERR_INVALID_ARG and h.value is None
    assert b"instance 2" in native.lib.dp_last_error()
    assert native.dp_multi_create(descs, 0, None, None, None, C.byref(h)) == native.DP_ERR_INVALID_ARG
