"""Python objects over the C ABI of include/wgrid.h.

Torch tensors provide device memory and the current CUDA stream; every computation runs in
the library's CUDA kernels.  Names follow the C ABI: grid_create -> Grid, conv_table_build ->
ConvTable.build, worklist_create -> WorkList, and vis_compress / grid_vis / degrid_vis /
grid_correct as functions.
"""
import ctypes

import numpy as np
import torch

from ._lib import Plan, CONST, GridDesc, Stats, TableDesc, TableInfo, VisIn, check, lib

c_vp = ctypes.c_void_p

SUPPORT_THRESHOLD = CONST["WG_SUPPORT_THRESHOLD"]
SUPPORT_PRESCRIBED = CONST["WG_SUPPORT_PRESCRIBED"]
DEGRID_PREDICT = CONST["WG_DEGRID_PREDICT"]
DEGRID_ADJOINT = CONST["WG_DEGRID_ADJOINT"]
IMAGE_PER_POL = CONST["WG_IMAGE_PER_POL"]
IMAGE_STOKES_I = CONST["WG_IMAGE_STOKES_I"]
IMAGE_PER_POL_RAW = CONST["WG_IMAGE_PER_POL_RAW"]
IMAGE_TRANSPOSE = CONST["WG_IMAGE_TRANSPOSE"]
IMAGE_STOKES_LINEAR = CONST["WG_IMAGE_STOKES_LINEAR"]
IMAGE_STOKES_CIRCULAR = CONST["WG_IMAGE_STOKES_CIRCULAR"]
PREP_CROSS_SWAP = CONST["WG_PREP_CROSS_SWAP"]
PREP_WSTACK = CONST["WG_PREP_WSTACK"]
PREP_APPEND = CONST["WG_PREP_APPEND"]
IMAGE_WSTACK = CONST["WG_IMAGE_WSTACK"]
PREP_COMPRESS = CONST["WG_PREP_COMPRESS"]
PREP_UNWEIGHTED = CONST["WG_PREP_UNWEIGHTED"]
PREP_INTERLEAVE = CONST["WG_PREP_INTERLEAVE"]


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_vp(s.cuda_stream)


class _DeviceBuffer:
    """Zero-copy description of a library-owned device buffer for torch.as_tensor."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(int(s) for s in shape), "typestr": typestr,
                                         "data": (int(ptr or 0), False), "version": 2}


def _view(ptr, shape, typestr):
    if not ptr or 0 in shape:
        return torch.empty(shape, dtype={"<f8": torch.float64, "<f4": torch.float32, "<i4": torch.int32,
                                         "|u1": torch.uint8}[typestr], device="cuda")
    return torch.as_tensor(_DeviceBuffer(ptr, shape, typestr), device="cuda")


def launch_count() -> int:
    """Kernels this library has launched in this process (cuFFT's own kernels excluded)."""
    return int(lib.wg_launch_count())


CEILINGS = {"fp32_fma2": "WG_CEIL_FP32_FMA2", "fp32_fma": "WG_CEIL_FP32_FMA", "fetch_l1": "WG_CEIL_FETCH_L1",
            "fetch_l2": "WG_CEIL_FETCH_L2", "shared": "WG_CEIL_SHARED"}


def ceiling(kind: str) -> float:
    """Measured roofline ceiling on the current device (ceiling_measure): FLOP/s for
    "fp32_fma2" / "fp32_fma", bytes/s for "fetch_l1" / "fetch_l2" / "shared".  Synchronous."""
    v = ctypes.c_double()
    check(lib.ceiling_measure(CONST[CEILINGS[kind]], ctypes.byref(v)), "ceiling_measure")
    return float(v.value)


class Grid:
    """Complex64 uv-grids [n_chan][N][N][n_pol] (torch tensor `data`) plus FP64 normalisers."""

    def __init__(self, n: int, du: float, n_pol: int = 1, n_chan: int = 1, device=None, compensated: bool = False,
                 storage: torch.Tensor = None):
        """compensated: flushes recover each atomic add's rounding error (WG_GRID_COMPENSATED).
        storage: an existing contiguous complex64 [n_chan][n][n][n_pol] CUDA tensor (e.g. a
        channel slice of a larger grid) that the grid uses instead of allocating; it is not zeroed."""
        self.n, self.du, self.n_pol, self.n_chan = int(n), float(du), int(n_pol), int(n_chan)
        if storage is None:
            self.data = torch.zeros((n_chan, n, n, n_pol), dtype=torch.complex64, device=device or "cuda")
        else:
            if (storage.dtype != torch.complex64 or tuple(storage.shape) != (self.n_chan, self.n, self.n, self.n_pol)
                    or not storage.is_contiguous() or not storage.is_cuda):
                raise ValueError("storage must be a contiguous complex64 CUDA tensor [n_chan][n][n][n_pol]")
            self.data = storage
        d = GridDesc(self.n, self.n_pol, self.n_chan, CONST["WG_GRID_COMPENSATED"] if compensated else 0, self.du,
                     self.data.data_ptr())
        h = c_vp()
        check(lib.grid_create(ctypes.byref(d), ctypes.byref(h)), "grid_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def zero(self, stream=None):
        check(lib.grid_zero(self._h, _stream(stream)), "grid_zero")

    def normaliser(self) -> torch.Tensor:
        """FP64 [n_chan][n_pol] view of N_p (eq. "normalizer")."""
        data, norm = c_vp(), c_vp()
        check(lib.grid_device_ptrs(self._h, ctypes.byref(data), ctypes.byref(norm)), "grid_device_ptrs")
        return _view(norm.value, (self.n_chan, self.n_pol), "<f8")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and lib is not None:
            lib.grid_destroy(h)
            self._h = None


class ConvTable:
    """Oversampled w-projection kernels (C-1 .. C-3 of the thesis, Sec. 4.2.2)."""

    def __init__(self, handle):
        self._h = handle
        info = TableInfo()
        check(lib.table_info(self._h, ctypes.byref(info)), "table_info")
        self.n_wplanes = info.n_wplanes
        self.oversample = info.oversample
        self.taper_support = info.taper_support
        self.max_support = info.max_support
        self.n_samples = info.n_samples
        self.w_max = info.w_max
        self.du = info.du
        sup = np.zeros(self.n_wplanes, np.int32)
        off = np.zeros(self.n_wplanes, np.int32)
        check(lib.table_copy_to_host(self._h, None, None, sup.ctypes.data, off.ctypes.data), "table_copy_to_host")
        self.supports, self.offsets = sup, off
        self._info = info
        self.store = {v: k for k, v in self.STORES.items()}[info.store_dtype]

    @property
    def handle(self):
        return self._h

    STORES = {"f32": CONST["WG_F32"], "bf16": CONST["WG_BF16"], "f16": CONST["WG_F16"]}

    @classmethod
    def build(cls, du: float, n_wplanes: int = 1, w_max: float = 0.0, oversample: int = 8,
              taper_support: int = 7, supports=None, n_k: int = 0, threshold: float = 1e-3, store: str = "f32",
              stacking: bool = False, stream=None):
        """stacking: a w-stacking table (every plane holds the w = 0 kernel; WG_TABLE_WSTACK)."""
        sup_arr = None
        if supports is not None:
            sup_arr = (ctypes.c_int32 * n_wplanes)(*[int(s) for s in supports])
        d = TableDesc(int(n_wplanes), int(oversample), int(taper_support), int(n_k),
                      (SUPPORT_PRESCRIBED if supports is not None else SUPPORT_THRESHOLD)
                      | (CONST["WG_TABLE_WSTACK"] if stacking else 0),
                      cls.STORES[store], float(w_max), float(du), float(threshold),
                      ctypes.cast(sup_arr, ctypes.POINTER(ctypes.c_int32)) if sup_arr is not None else None)
        h = c_vp()
        check(lib.conv_table_build(ctypes.byref(d), ctypes.byref(h), _stream(stream)), "conv_table_build")
        return cls(h)

    @classmethod
    def from_host(cls, n_wplanes, oversample, w_max, du, taper_support, supports, data, zeta):
        """Imports C-1 (complex [sum_k beta^2 S_k^2]), C-2 supports and C-3 zeta from host arrays."""
        sup = np.ascontiguousarray(supports, np.int32)
        dat = np.ascontiguousarray(np.asarray(data, np.complex128)).view(np.float64)
        zet = np.ascontiguousarray(zeta, np.float64)
        h = c_vp()
        check(lib.conv_table_import(int(n_wplanes), int(oversample), float(w_max), float(du), int(taper_support),
                                    sup.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                    dat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    zet.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(h)),
              "conv_table_import")
        return cls(h)

    def set_store(self, store: str):
        """Storage the gridder reads: "f32", "bf16" or "f16" (round to nearest even)."""
        check(lib.table_set_store(self._h, self.STORES[store]), "table_set_store")
        self.store = store

    def lp_samples(self) -> torch.Tensor:
        """The low-precision copy as a device int32 view (one complex bf16/f16 pair per element)."""
        info = TableInfo()
        check(lib.table_info(self._h, ctypes.byref(info)), "table_info")
        return _view(info.data_lp, (int(info.n_samples),), "<i4")

    def to_host(self):
        """(C-1 complex64 numpy, zeta float64, supports int32, offsets int32)."""
        data = np.zeros(self.n_samples, np.complex64)
        zeta = np.zeros(self.n_wplanes * self.oversample ** 2, np.float64)
        check(lib.table_copy_to_host(self._h, data.ctypes.data, zeta.ctypes.data, None, None), "table_copy_to_host")
        return data, zeta, self.supports.copy(), self.offsets.copy()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and lib is not None:
            lib.table_destroy(h)
            self._h = None


class VisBatch:
    """Device inputs I-1..I-5 (Sec. 4.3.2): uvw [rows,3] f64 metres, freq [C] f64 Hz, vis
    [rows,C,P] complex64 (or complex32 = two float16 with per-channel float32 scales
    `vis_scale` [C]: value = scale x vis), weight [rows,C,P] f32, flag [rows,C,P] uint8."""

    def __init__(self, uvw, freq, vis, weight, flag, vis_scale=None):
        def dev(t, dtype):
            t = torch.as_tensor(t)
            if t.dtype != dtype:
                raise TypeError("expected %s, got %s" % (dtype, t.dtype))
            if not t.is_cuda:
                raise ValueError("inputs must be CUDA tensors")
            return t.contiguous()
        self.uvw = dev(uvw, torch.float64)
        self.freq = dev(freq, torch.float64)
        half = torch.as_tensor(vis).dtype == torch.complex32
        self.vis = dev(vis, torch.complex32 if half else torch.complex64)
        self.vis_scale = dev(vis_scale, torch.float32) if half else None
        if half and (self.vis_scale is None or self.vis_scale.shape != (self.vis.shape[1],)):
            raise ValueError("half-precision visibilities need vis_scale of shape [n_chan]")
        self.weight = dev(weight, torch.float32)
        self.flag = dev(flag, torch.uint8)
        rows, C, P = self.vis.shape
        if self.uvw.shape != (rows, 3) or self.freq.shape != (C,) or self.weight.shape != self.vis.shape \
                or self.flag.shape != self.vis.shape:
            raise ValueError("inconsistent input shapes")
        self.rows, self.n_chan, self.n_pol = rows, C, P
        self.struct = VisIn(rows, C, P, self.uvw.data_ptr(), self.freq.data_ptr(), self.vis.data_ptr(),
                            self.weight.data_ptr(), self.flag.data_ptr(),
                            CONST["WG_VIS_COMPLEX_HALF"] if half else CONST["WG_VIS_COMPLEX64"], 0,
                            self.vis_scale.data_ptr() if half else None)


class WorkList:
    """Device outputs of the preparation phase for up to max_records records per batch.
    max_entries: room for that many gridded entries over the batches appended with
    vis_compress(..., append=True) (worklist_create2: no degridding accumulator)."""

    def __init__(self, max_records: int, n_chan: int, n_pol: int, max_entries=None):
        h = c_vp()
        if max_entries is None:
            check(lib.worklist_create(int(max_records), int(n_chan), int(n_pol), ctypes.byref(h)), "worklist_create")
        else:
            check(lib.worklist_create2(int(max_records), int(max_entries), int(n_chan), int(n_pol), ctypes.byref(h)),
                  "worklist_create2")
        self._h = h
        self.n_chan, self.n_pol, self.capacity = n_chan, n_pol, max_records

    def clear(self, stream=None):
        """Empties the work list for a new sequence of appended batches."""
        check(lib.worklist_clear(self._h, _stream(stream)), "worklist_clear")

    @property
    def handle(self):
        return self._h

    def stats(self, stream=None) -> dict:
        st = Stats()
        check(lib.worklist_stats(self._h, ctypes.byref(st), _stream(stream)), "worklist_stats")
        return {k: getattr(st, k) for k, _ in Stats._fields_}

    def plan(self, table: "ConvTable", seg_len: int, slots: int, fixed_r: bool = False, stream=None):
        """Re-plans the prepared batch's gridder tasks: segment length, footprint points per task,
        and whether every support runs with R = slots / 32 points per lane (WG_PLAN_FIXED_R)."""
        pl = Plan(int(seg_len), int(slots), CONST["WG_PLAN_FIXED_R"] if fixed_r else 0, 0)
        check(lib.worklist_plan(self._h, table.handle, ctypes.byref(pl), _stream(stream)), "worklist_plan")

    @property
    def plan_params(self) -> tuple:
        """(seg_len, slots, fixed_r) of the current plan."""
        pl = Plan()
        check(lib.worklist_get_plan(self._h, ctypes.byref(pl)), "worklist_get_plan")
        return int(pl.seg_len), int(pl.slots), bool(pl.flags & CONST["WG_PLAN_FIXED_R"])

    def view(self, n_records: int, stream=None):
        """(entries int32 [n,4], gamma complex64 [n,P], runs int32 [n,2], rec_class uint8 [n_records])."""
        e, g, r, c = c_vp(), c_vp(), c_vp(), c_vp()
        n = ctypes.c_int64()
        check(lib.worklist_view(self._h, ctypes.byref(e), ctypes.byref(g), ctypes.byref(r), ctypes.byref(c),
                                ctypes.byref(n), _stream(stream)), "worklist_view")
        n = int(n.value)
        ent = _view(e.value, (n, 4), "<i4")
        gam = torch.view_as_complex(_view(g.value, (n, self.n_pol, 2), "<f4"))
        runs = _view(r.value, (n, 2), "<i4")
        cls = _view(c.value, (n_records,), "|u1")
        return ent, gam, runs, cls

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and lib is not None:
            lib.worklist_destroy(h)
            self._h = None


def vis_compress(grid: Grid, table: ConvTable, batch: VisBatch, worklist: WorkList, compress: bool = True,
                 unweighted: bool = False, interleave: bool = False, cross_swap: bool = False, wstack: bool = False,
                 append: bool = False, chan0: int = 0, stream=None):
    """Preparation phase.  interleave: all channels of the batch grid onto the one-channel
    `grid` in natural record order, compressing across channels (WG_PREP_INTERLEAVE).
    cross_swap: full-Stokes gridding of quad-pol data (WG_PREP_CROSS_SWAP).
    wstack: w-stacking onto n_chan x K grid channels (WG_PREP_WSTACK, a stacking table).
    append: add the batch's entries after the earlier appended ones (WG_PREP_APPEND); the
    batch grids onto grid channels chan0 .. chan0 + n_chan - 1 and its normaliser terms go
    into the grid now, and one grid_vis then grids every appended batch."""
    flags = ((PREP_COMPRESS if compress else 0) | (PREP_UNWEIGHTED if unweighted else 0)
             | (PREP_INTERLEAVE if interleave else 0) | (PREP_CROSS_SWAP if cross_swap else 0)
             | (PREP_WSTACK if wstack else 0) | (PREP_APPEND if append else 0))
    batch.struct.chan0 = int(chan0) if append else 0
    check(lib.vis_compress(grid.handle, table.handle, ctypes.byref(batch.struct), flags,
                           worklist.handle, _stream(stream)), "vis_compress")


def grid_vis(grid: Grid, table: ConvTable, worklist: WorkList, stream=None):
    check(lib.grid_vis(grid.handle, table.handle, worklist.handle, _stream(stream)), "grid_vis")


def grid_autotune(grid: Grid, table: ConvTable, worklist: WorkList, candidates=None, repeats: int = 3,
                  stream=None) -> tuple:
    """Times grid_vis under each candidate plan (seg_len, slots, fixed_r) on the prepared batch
    (None: the library's default list), keeps the fastest in the work list and zeroes the grid.
    Returns (seg_len, slots, fixed_r, ms per launch)."""
    arr, n = None, 0
    if candidates:
        n = len(candidates)
        arr = (Plan * n)(*[Plan(int(a), int(b), CONST["WG_PLAN_FIXED_R"] if c else 0, 0) for a, b, c in candidates])
    best, ms = Plan(), ctypes.c_float()
    check(lib.grid_autotune(grid.handle, table.handle, worklist.handle, arr, n, int(repeats), ctypes.byref(best),
                            ctypes.byref(ms), _stream(stream)), "grid_autotune")
    return int(best.seg_len), int(best.slots), bool(best.flags & CONST["WG_PLAN_FIXED_R"]), float(ms.value)


def vis_weight(grid: Grid, table: ConvTable, batch: VisBatch, scheme: str = "uniform", robust: float = 0.0,
               interleave: bool = False, wstack: bool = False, out: torch.Tensor = None, stream=None) -> torch.Tensor:
    """Uniform or robust (Briggs) weights for the batch from the density of its griddable records
    per grid cell (WG_WEIGHT_UNIFORM / WG_WEIGHT_ROBUST); returns float32 [rows][chan][pol]."""
    codes = {"uniform": CONST["WG_WEIGHT_UNIFORM"], "robust": CONST["WG_WEIGHT_ROBUST"]}
    if out is None:
        out = torch.empty_like(batch.weight)
    if out.dtype != torch.float32 or out.shape != batch.weight.shape or not out.is_contiguous():
        raise ValueError("out must be a contiguous float32 tensor shaped like the weights")
    check(lib.vis_weight(grid.handle, table.handle, ctypes.byref(batch.struct), codes[scheme], float(robust),
                         (PREP_INTERLEAVE if interleave else 0) | (PREP_WSTACK if wstack else 0),
                         c_vp(out.data_ptr()), _stream(stream)), "vis_weight")
    return out


def degrid_vis(grid: Grid, table: ConvTable, batch: VisBatch, worklist: WorkList, mode: int = DEGRID_PREDICT,
               out: torch.Tensor = None, stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty(batch.vis.shape, dtype=torch.complex64, device=batch.vis.device)
    if out.dtype != torch.complex64 or out.shape != batch.vis.shape or not out.is_contiguous():
        raise ValueError("out must be a contiguous complex64 tensor shaped like the visibilities")
    check(lib.degrid_vis(grid.handle, table.handle, ctypes.byref(batch.struct), worklist.handle, int(mode),
                         c_vp(out.data_ptr()), _stream(stream)), "degrid_vis")
    return out


def grid_correct(grid: Grid, table: ConvTable, mode: int = IMAGE_PER_POL, out: torch.Tensor = None,
                 stream=None) -> torch.Tensor:
    if mode == IMAGE_TRANSPOSE:
        raise ValueError("use image_to_grid for the transpose mode")
    if mode == IMAGE_STOKES_I:
        shape = (grid.n_chan, grid.n, grid.n)
    elif mode == IMAGE_WSTACK:
        shape = (grid.n_chan // table.n_wplanes, grid.n_pol, grid.n, grid.n)
    else:
        shape = (grid.n_chan, grid.n_pol, grid.n, grid.n)
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=grid.data.device)
    if out.dtype != torch.float32 or tuple(out.shape) != shape or not out.is_contiguous():
        raise ValueError("out must be a contiguous float32 tensor of shape %s" % (shape,))
    check(lib.grid_correct(grid.handle, table.handle, int(mode), c_vp(out.data_ptr()), _stream(stream)),
          "grid_correct")
    return out


def image_to_grid(grid: Grid, table: ConvTable, image: torch.Tensor, stream=None) -> Grid:
    """Overwrites grid with the transpose of grid_correct(mode=IMAGE_PER_POL_RAW) applied to a
    float32 [n_chan][n_pol][N][N] image: the sky-to-grid half of the forward model."""
    shape = (grid.n_chan, grid.n_pol, grid.n, grid.n)
    if image.dtype != torch.float32 or tuple(image.shape) != shape or not image.is_contiguous() or not image.is_cuda:
        raise ValueError("image must be a contiguous CUDA float32 tensor of shape %s" % (shape,))
    check(lib.grid_correct(grid.handle, table.handle, IMAGE_TRANSPOSE, c_vp(image.data_ptr()), _stream(stream)),
          "grid_correct")
    return grid
