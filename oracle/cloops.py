"""Loads (compiling when needed) the oracle's plain C loops.  Test infrastructure only."""
import ctypes
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    so = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i64, i32 = ctypes.c_int64, ctypes.c_int32
    so.or_grid.argtypes = [i64, P, P, P, P, P, P, i32, i32, P, P]
    so.or_grid.restype = None
    so.or_degrid.argtypes = [i64, P, P, P, P, P, i32, i32, P, P, P]
    so.or_degrid.restype = None
    so.or_compress.argtypes = [i64, i32, i32, i32, i32, P, P, P, P, P, P, P, P, P, P, P, P, P, P]
    so.or_compress.restype = i64
    return so


lib = _load()
