"""CPU-side checks of the C ABI: the library loads, exports every entry
point include/flood.h declares, and rejects bad arguments in host code
(no kernel runs here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "flood.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(?:int|void|int64_t|const char\*)\s+\**(\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def capi():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2302_08341_gb300 import capi
    return capi


def test_library_exports_every_declared_symbol(capi):
    names = _declared()
    assert len(names) >= 16
    L = capi.lib()
    for n in names:
        assert hasattr(L, n), f"{n} declared in include/flood.h but not exported"
    assert sorted(capi.EXPORTED) == names


def test_default_params_host_only(capi):
    p = capi.Params.default()
    assert p.dx == 3.0 and p.g == 9.81 and p.alpha == 0.7 and p.dt_cap == 1.0
    assert p.h_eps == 0.0 and p.rain_block == 300.0 and p.limiter == 1
    assert p.east_outflow == 1 and p.south_outflow == 0 and p.reserved == 0


def test_argument_errors_are_reported_before_any_device_work(capi):
    L = capi.lib()
    h = C.c_void_p()
    p = capi.Params.default()
    z = (C.c_float * 4)()
    rc = L.flood_create_grid(C.byref(h), 0, 4, z, z, C.byref(p))
    assert rc == -1 and b"ny and nx" in L.flood_last_error(None)
    rc = L.flood_create_grid(C.byref(h), 2, 2, None, z, C.byref(p))
    assert rc == -1
    bad = capi.Params.default(dx=-1.0)
    rc = L.flood_create_grid(C.byref(h), 2, 2, z, z, C.byref(bad))
    assert rc == -1 and b"flood_params" in L.flood_last_error(None)
    w = (C.c_double * 3)(0.2, 0.3, 0.5)
    idx = (C.c_int32 * 3)()
    assert L.pf_resample_systematic(3, w, 1.0, idx, None) == -1
    assert L.pf_resample_systematic(0, w, 0.5, idx, None) == -1
    assert L.flood_step(None, 1, -1.0, None) == -1
    assert L.flood_destroy(None) == 0
    assert L.flood_launch_count(None) == 0


def test_every_handle_call_refuses_a_null_handle(capi):
    """Each entry point that takes a grid or batch handle returns
    FLOOD_ERR_ARG for a NULL one (no device work); the destroy calls accept
    NULL and the launch counters read 0."""
    L = capi.lib()
    no_handle = {"flood_default_params", "flood_create_grid", "flood_batch_create",
                 "pf_resample_systematic", "flood_storage_static", "flood_storage_static_error"}
    want = {"flood_destroy": 0, "flood_batch_destroy": 0, "flood_launch_count": 0,
            "flood_batch_launch_count": 0}
    text = {"flood_last_error", "flood_batch_last_error"}
    checked = 0
    for name in capi.EXPORTED:
        if name in no_handle or name in text:
            continue
        f = getattr(L, name)
        args = [0 if t in (C.c_int, C.c_int64) else 0.0 if t is C.c_double else None
                for t in f.argtypes]
        assert f(*args) == want.get(name, -1), name
        checked += 1
    assert checked == len(capi.EXPORTED) - len(no_handle) - len(text)
    assert L.flood_last_error(None) == b"grid is NULL"
    assert L.flood_batch_last_error(None) == b"batch is NULL"
