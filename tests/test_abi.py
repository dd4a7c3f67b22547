"""The C-ABI library loads, exports every function include/wgrid.h declares, and rejects bad
arguments with the documented status codes before touching the GPU (runs without a GPU)."""
import ctypes

import pytest

import paper_1403_4209_gb300 as wg
from paper_1403_4209_gb300 import _lib

C = wg.CONST


def test_every_declared_symbol_is_exported():
    names = wg.header_functions()
    assert len(names) >= 19
    for n in names:
        assert hasattr(wg.lib, n), n
        assert ctypes.cast(getattr(wg.lib, n), ctypes.c_void_p).value


def test_status_codes_distinct():
    codes = [v for k, v in C.items() if k.startswith("WG_E_")]
    assert len(set(codes)) == len(codes) and all(c < 0 for c in codes) and C["WG_OK"] == 0


def _err():
    return wg.lib.wg_last_error().decode()


@pytest.mark.parametrize("n,pol,chan,du,msg", [(7, 1, 1, 1.0, "even"), (64, 3, 1, 1.0, "n_pol"),
                                               (64, 1, 0, 1.0, "n_chan"), (64, 1, 1, 0.0, "du")])
def test_grid_create_rejects(n, pol, chan, du, msg):
    d = _lib.GridDesc(n, pol, chan, 0, du, None)
    h = ctypes.c_void_p()
    assert wg.lib.grid_create(ctypes.byref(d), ctypes.byref(h)) == C["WG_E_INVALID_ARG"]
    assert msg in _err() and not h.value


def _table_desc(supports, K=None, beta=8, mode=None, w_max=0.0):
    K = K or len(supports)
    arr = (ctypes.c_int32 * K)(*supports)
    return _lib.TableDesc(K, beta, 7, 0, C["WG_SUPPORT_PRESCRIBED"] if mode is None else mode, C["WG_F32"],
                          w_max, 1.0, 1e-3, ctypes.cast(arr, ctypes.POINTER(ctypes.c_int32))), arr


def test_table_rejects_even_and_oversized_supports():
    h = ctypes.c_void_p()
    d, keep = _table_desc([8])
    assert wg.lib.conv_table_build(ctypes.byref(d), ctypes.byref(h), None) == C["WG_E_INVALID_ARG"]
    d, keep = _table_desc([2049])
    assert wg.lib.conv_table_build(ctypes.byref(d), ctypes.byref(h), None) == C["WG_E_OOB_SUPPORT"]
    d, keep = _table_desc([7, 9], beta=0)
    assert wg.lib.conv_table_build(ctypes.byref(d), ctypes.byref(h), None) == C["WG_E_INVALID_ARG"]
    d, keep = _table_desc([7, 9], w_max=0.0)
    assert wg.lib.conv_table_build(ctypes.byref(d), ctypes.byref(h), None) == C["WG_E_INVALID_ARG"]
    assert "w_max" in _err()


def test_worklist_and_null_handles():
    h = ctypes.c_void_p()
    assert wg.lib.worklist_create(100, 1, 3, ctypes.byref(h)) == C["WG_E_INVALID_ARG"]
    assert wg.lib.worklist_create(0, 1, 1, ctypes.byref(h)) == C["WG_E_INVALID_ARG"]
    vi = _lib.VisIn()
    assert wg.lib.vis_compress(None, None, ctypes.byref(vi), 1, None, None) == C["WG_E_INVALID_ARG"]
    assert wg.lib.grid_vis(None, None, None, None) == C["WG_E_INVALID_ARG"]
    assert wg.lib.degrid_vis(None, None, ctypes.byref(vi), None, 0, None, None) == C["WG_E_INVALID_ARG"]
    assert wg.lib.grid_correct(None, None, 0, None, None) == C["WG_E_INVALID_ARG"]
    st = _lib.Stats()
    assert wg.lib.worklist_stats(None, ctypes.byref(st), None) == C["WG_E_INVALID_ARG"]


def test_errors_raise_in_python():
    with pytest.raises(wg.WgError, match="WG_E_INVALID_ARG"):
        _lib.check(wg.lib.worklist_create(0, 1, 1, ctypes.byref(ctypes.c_void_p())), "worklist_create")


def test_plan_limits_and_null_handles():
    assert C["WG_PLAN_SEG_LEN_MIN"] <= C["WG_PLAN_SEG_LEN_DEFAULT"] <= C["WG_PLAN_SEG_LEN_MAX"]
    assert C["WG_PLAN_SLOTS_MIN"] <= C["WG_PLAN_SLOTS_DEFAULT"] <= C["WG_PLAN_SLOTS_MAX"]
    assert all(C[k] % 32 == 0 for k in C if k.startswith("WG_PLAN_S"))
    assert ctypes.sizeof(_lib.Plan) == 16 and C["WG_PLAN_FIXED_R"] == 1
    pl = _lib.Plan(128, 256, 0, 0)
    assert wg.lib.worklist_plan(None, None, ctypes.byref(pl), None) == C["WG_E_INVALID_ARG"]
    assert "null" in _err()
    assert wg.lib.worklist_get_plan(None, None) == C["WG_E_INVALID_ARG"]
    assert wg.lib.grid_autotune(None, None, None, None, 0, 3, None, None, None) == C["WG_E_INVALID_ARG"]


def test_ceiling_rejects_bad_arguments():
    v = ctypes.c_double(1.0)
    assert wg.lib.ceiling_measure(0, ctypes.byref(v)) == C["WG_E_INVALID_ARG"] and "unknown ceiling" in _err()
    assert wg.lib.ceiling_measure(C["WG_CEIL_SHARED"] + 1, ctypes.byref(v)) == C["WG_E_INVALID_ARG"]
    assert v.value == 0.0
    assert wg.lib.ceiling_measure(C["WG_CEIL_FP32_FMA2"], None) == C["WG_E_INVALID_ARG"]


def test_injected_allocation_failure_returns_oom():
    # the allocation-failure fake fails the next device allocation before the runtime is called,
    # so grid_create and worklist_create report WG_E_OOM and leave no handle (runs without a GPU)
    assert wg.lib.wg_debug_fail_allocations(ctypes.c_int64(0)) == C["WG_OK"]
    try:
        d = _lib.GridDesc(64, 1, 1, 0, 1.0, None)
        h = ctypes.c_void_p()
        assert wg.lib.grid_create(ctypes.byref(d), ctypes.byref(h)) == C["WG_E_OOM"]
        assert "allocate" in _err() and not h.value
        w = ctypes.c_void_p()
        rc = wg.lib.worklist_create(ctypes.c_int64(1000), ctypes.c_int32(2), ctypes.c_int32(4), ctypes.byref(w))
        assert rc == C["WG_E_OOM"]
        assert "work list" in _err() and not w.value
    finally:
        assert wg.lib.wg_debug_fail_allocations(ctypes.c_int64(-1)) == C["WG_OK"]


def test_every_declaration_cites_its_passage():
    # each function's comment block names the thesis passage it follows, or says that the
    # thesis has no counterpart
    import re
    txt = open(_lib.HEADER).read()
    decls = [(m.start(), m.group(1)) for m in
             re.finditer(r"^\s*(?:int|const char\*|uint64_t)\s+(\w+)\s*\(", txt, flags=re.M)]
    prev = 0
    for pos, name in decls:
        comments = " ".join(re.findall(r"/\*.*?\*/", txt[prev:pos], flags=re.S))
        assert re.search(r"Sec\.|Algorithm|eq\.|thesis|no counterpart", comments), name
        prev = pos
