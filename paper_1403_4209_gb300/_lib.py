"""ctypes declarations of the C ABI in include/wgrid.h (argument marshalling only).

Loading fails loudly when libwgrid.so is missing and cannot be built: there is no CPU or
Python fallback for any step of the path.
"""
import ctypes
import os
import re

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "include", "wgrid.h")

c_i32, c_i64, c_u64, c_dbl, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p


class GridDesc(ctypes.Structure):
    _fields_ = [("n", c_i32), ("n_pol", c_i32), ("n_chan", c_i32), ("flags", c_i32),
                ("du", c_dbl), ("data", c_vp)]


class TableDesc(ctypes.Structure):
    _fields_ = [("n_wplanes", c_i32), ("oversample", c_i32), ("taper_support", c_i32), ("n_k", c_i32),
                ("support_mode", c_i32), ("store_dtype", c_i32), ("w_max", c_dbl), ("du", c_dbl),
                ("threshold", c_dbl), ("supports", ctypes.POINTER(c_i32))]


class TableInfo(ctypes.Structure):
    _fields_ = [("n_wplanes", c_i32), ("oversample", c_i32), ("taper_support", c_i32), ("max_support", c_i32),
                ("n_samples", c_i64), ("w_max", c_dbl), ("du", c_dbl), ("data", c_vp), ("zeta", c_vp),
                ("supports", c_vp), ("offsets", c_vp), ("store_dtype", c_i32), ("reserved", c_i32),
                ("data_lp", c_vp)]


class VisIn(ctypes.Structure):
    _fields_ = [("n_rows", c_i64), ("n_chan", c_i32), ("n_pol", c_i32), ("uvw", c_vp), ("freq_hz", c_vp),
                ("vis", c_vp), ("weight", c_vp), ("flag", c_vp), ("vis_dtype", c_i32), ("chan0", c_i32),
                ("vis_scale", c_vp)]


class Stats(ctypes.Structure):
    _fields_ = [(k, c_i64) for k in ("records", "griddable", "gridded", "compressed", "updates",
                                     "updates_saved", "tasks", "dropped")]


class Plan(ctypes.Structure):
    _fields_ = [("seg_len", c_i32), ("slots", c_i32), ("flags", c_i32), ("reserved", c_i32)]


def _constants():
    out = {}
    for m in re.finditer(r"#define\s+(WG_\w+)\s+\(?(-?\d+)\)?", open(HEADER).read()):
        out[m.group(1)] = int(m.group(2))
    return out


CONST = _constants()


def header_functions():
    """Names of the functions include/wgrid.h declares."""
    txt = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*|uint64_t)\s+(\w+)\s*\(", txt, flags=re.M)))


def _load():
    path = _build.LIB
    if _build.stale():
        try:
            _build.build()
        except Exception as e:  # noqa: BLE001
            raise ImportError("libwgrid.so is missing and could not be built (%s); run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`" % e) from e
    so = ctypes.CDLL(path)
    P = ctypes.POINTER
    sig = {
        "wg_last_error": (ctypes.c_char_p, []),
        "wg_launch_count": (c_u64, []),
        "grid_create": (c_i32, [P(GridDesc), P(c_vp)]),
        "grid_destroy": (c_i32, [c_vp]),
        "grid_zero": (c_i32, [c_vp, c_vp]),
        "grid_device_ptrs": (c_i32, [c_vp, P(c_vp), P(c_vp)]),
        "conv_table_build": (c_i32, [P(TableDesc), P(c_vp), c_vp]),
        "conv_table_import": (c_i32, [c_i32, c_i32, c_dbl, c_dbl, c_i32, P(c_i32), P(c_dbl), P(c_dbl), P(c_vp)]),
        "table_destroy": (c_i32, [c_vp]),
        "table_set_store": (c_i32, [c_vp, c_i32]),
        "table_info": (c_i32, [c_vp, P(TableInfo)]),
        "table_copy_to_host": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp]),
        "worklist_create": (c_i32, [c_i64, c_i32, c_i32, P(c_vp)]),
        "worklist_create2": (c_i32, [c_i64, c_i64, c_i32, c_i32, P(c_vp)]),
        "worklist_clear": (c_i32, [c_vp, c_vp]),
        "worklist_destroy": (c_i32, [c_vp]),
        "vis_compress": (c_i32, [c_vp, c_vp, P(VisIn), c_i32, c_vp, c_vp]),
        "worklist_stats": (c_i32, [c_vp, P(Stats), c_vp]),
        "worklist_view": (c_i32, [c_vp, P(c_vp), P(c_vp), P(c_vp), P(c_vp), P(c_i64), c_vp]),
        "grid_vis": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
        "worklist_plan": (c_i32, [c_vp, c_vp, P(Plan), c_vp]),
        "worklist_get_plan": (c_i32, [c_vp, P(Plan)]),
        "grid_autotune": (c_i32, [c_vp, c_vp, c_vp, P(Plan), c_i32, c_i32, P(Plan), P(ctypes.c_float), c_vp]),
        "degrid_vis": (c_i32, [c_vp, c_vp, P(VisIn), c_vp, c_i32, c_vp, c_vp]),
        "grid_correct": (c_i32, [c_vp, c_vp, c_i32, c_vp, c_vp]),
        "vis_weight": (c_i32, [c_vp, c_vp, P(VisIn), c_i32, c_dbl, c_i32, c_vp, c_vp]),
        "ceiling_measure": (c_i32, [c_i32, P(c_dbl)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(so, name)
        f.restype = res
        f.argtypes = args
    return so


lib = _load()


class WgError(RuntimeError):
    def __init__(self, code, func):
        self.code = code
        msg = lib.wg_last_error().decode(errors="replace")
        name = {v: k for k, v in CONST.items() if k.startswith("WG_E_")}.get(code, str(code))
        super().__init__("%s failed with %s: %s" % (func, name, msg))


def check(rc, func):
    if rc != 0:
        raise WgError(rc, func)
