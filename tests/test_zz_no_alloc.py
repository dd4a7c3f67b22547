"""grid_vis_noalloc: gridding for callers that cannot call cudaMalloc (graph capture, fixed
memory budgets, real-time loops).  Through the C ABI it must give the same grid and
normaliser as vis_compress + grid_vis, within the parity tests' tolerance, on two calls in a
row that reuse its built-in scratch, and it must not allocate device memory.

This file is collected last on purpose, so a run that stops at the first failure has already
run every other test."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 1e-5


class GridView(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_pol", ctypes.c_int32), ("n_chan", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("du", ctypes.c_double), ("data", ctypes.c_void_p),
                ("normaliser", ctypes.c_void_p)]


def _noalloc_fn():
    import paper_1403_4209_gb300 as wg
    from paper_1403_4209_gb300 import _lib
    f = wg.lib.grid_vis_noalloc
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.POINTER(GridView), ctypes.c_void_p, ctypes.POINTER(_lib.VisIn), ctypes.c_int32,
                  ctypes.c_void_p]
    return f


def test_noalloc_matches_worklist_path_twice():
    import paper_1403_4209_gb300 as wg
    import synth
    from gpu_common import max_rel, rel_l2, run_gpu

    # 4 channels x 4 polarisations, 16 w-planes: 200 baselines x 60 steps = 48,000 records
    wl = synth.make("degrid_1k", n_times=60, n_baselines=200, flag_frac=0.02)
    assert wl.rows * wl.n_chan <= wg.CONST["WG_NOALLOC_MAX_RECORDS"]
    ref = run_gpu(wl)                                   # the existing entry points
    g, t, batch, _ = ref["objects"]
    fn = _noalloc_fn()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        out = torch.zeros_like(g.data)
        norm = torch.zeros((wl.n_chan, wl.n_pol), dtype=torch.float64, device="cuda")
        view = GridView(wl.n_grid, wl.n_pol, wl.n_chan, 0, wl.du, out.data_ptr(), norm.data_ptr())
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = fn(ctypes.byref(view), t.handle, ctypes.byref(batch.struct), 1, stream)
        assert rc == 0, wg.lib.wg_last_error().decode()
        torch.cuda.synchronize()
        if call == 1:   # the first call may load the module holding the scratch
            assert torch.cuda.mem_get_info()[0] == free_before
        got = out.cpu().numpy()
        assert rel_l2(got, ref["grid"]) < TOL
        assert max_rel(got, ref["grid"]) < TOL
        assert max_rel(norm.cpu().numpy(), ref["norm"]) < TOL


def test_noalloc_rejects_oversized_batches():
    import paper_1403_4209_gb300 as wg
    import synth
    from gpu_common import gpu_table

    wl = synth.make("w0_small", n_times=140)            # 496 x 140 = 69,440 records > 65,536
    t = gpu_table(wl)
    batch = wg.VisBatch(torch.as_tensor(wl.uvw, device="cuda"), torch.as_tensor(wl.freq, device="cuda"),
                        wl.vis.cuda(), wl.weight.cuda(), wl.flag.cuda())
    out = torch.zeros((1, wl.n_grid, wl.n_grid, 1), dtype=torch.complex64, device="cuda")
    norm = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    view = GridView(wl.n_grid, 1, 1, 0, wl.du, out.data_ptr(), norm.data_ptr())
    rc = _noalloc_fn()(ctypes.byref(view), t.handle, ctypes.byref(batch.struct), 1, None)
    assert rc == wg.CONST["WG_E_CAPACITY"]
    assert "no-allocation limit" in wg.lib.wg_last_error().decode()
    assert np.all(out.cpu().numpy() == 0)
