"""grid_vis_noalloc: gridding for callers that cannot call cudaMalloc (code recording into a CUDA
graph, processes on a fixed device-memory budget, real-time loops).  Through the C ABI it must
give the same grid and normaliser as vis_compress + grid_vis, and as the FP64 oracle, within the
parity tests' tolerance, on two calls in a row that reuse its built-in scratch, with no entry
dropped by the device-side bounds checks and no device memory allocated.

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
                ("normaliser", ctypes.c_void_p), ("dropped", ctypes.c_void_p)]


def _noalloc_fn():
    import paper_1403_4209_gb300 as wg
    from paper_1403_4209_gb300 import _lib
    f = wg.lib.grid_vis_noalloc
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.POINTER(GridView), ctypes.c_void_p, ctypes.POINTER(_lib.VisIn), ctypes.c_int32,
                  ctypes.c_void_p]
    return f


def _call(wl, table, batch, compress, out, norm, dropped, stream):
    import paper_1403_4209_gb300 as wg
    view = GridView(wl.n_grid, wl.n_pol, wl.n_chan, 0, wl.du, out.data_ptr(), norm.data_ptr(),
                    None if dropped is None else dropped.data_ptr())
    rc = _noalloc_fn()(ctypes.byref(view), table.handle, ctypes.byref(batch.struct), compress, stream)
    assert rc == 0, wg.lib.wg_last_error().decode()
    assert wg.lib.wg_last_error().decode() == ""


@pytest.mark.parametrize("compress", [True, False], ids=["compress", "no-compress"])
def test_noalloc_matches_worklist_path_and_oracle_twice(compress):
    import synth
    from gpu_common import max_rel, rel_l2, run_gpu, run_oracle

    import paper_1403_4209_gb300 as wg
    # 4 channels x 4 polarisations, 16 w-planes: 200 baselines x 60 steps = 48,000 records
    wl = synth.make("degrid_1k", n_times=60, n_baselines=200, flag_frac=0.02)
    assert wl.rows * wl.n_chan <= wg.CONST["WG_NOALLOC_MAX_RECORDS"]
    ref = run_gpu(wl, compress=compress)                # the existing entry points
    orc = run_oracle(wl, compress=compress)              # the FP64 oracle on the same inputs
    g, t, batch, _ = ref["objects"]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    dropped = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    for call in range(2):
        out = torch.zeros_like(g.data)
        norm = torch.zeros((wl.n_chan, wl.n_pol), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        _call(wl, t, batch, 1 if compress else 0, out, norm, dropped, stream)
        torch.cuda.synchronize()
        if call == 1:   # the first call may load the module holding the scratch
            assert torch.cuda.mem_get_info()[0] == free_before
        assert int(dropped.item()) == 0
        got, got_n = out.cpu().numpy(), norm.cpu().numpy()
        for want, want_n in ((ref["grid"], ref["norm"]), (orc["grid"], orc["norm"])):
            assert rel_l2(got, want) < TOL
            assert max_rel(got, want) < TOL
            assert max_rel(got_n, want_n) < TOL


def test_noalloc_half_vis_at_element_alignment():
    """Half-precision visibilities need only 4-byte alignment, as vis_compress accepts them."""
    import synth
    from gpu_common import gpu_table, max_rel, rel_l2

    import paper_1403_4209_gb300 as wg
    wl = synth.make("degrid_1k", n_times=30, n_baselines=150, n_chan=2, flag_frac=0.02)
    t = gpu_table(wl)
    vis_h, scale = synth.to_half_vis(wl.vis.cuda())
    buf = torch.empty(vis_h.numel() + 1, dtype=torch.complex32, device="cuda")
    buf[1:].copy_(vis_h.reshape(-1))
    shifted = buf[1:].view(vis_h.shape)               # 4 bytes past an 8-byte boundary
    assert shifted.data_ptr() % 8 == 4
    dev = "cuda"
    uvw, freq = torch.as_tensor(wl.uvw, device=dev), torch.as_tensor(wl.freq, device=dev)
    b = wg.VisBatch(uvw, freq, shifted, wl.weight.to(dev), wl.flag.to(dev), vis_scale=scale)
    g = wg.Grid(wl.n_grid, wl.du, wl.n_pol, wl.n_chan)
    w = wg.WorkList(wl.rows * wl.n_chan, wl.n_chan, wl.n_pol)
    wg.vis_compress(g, t, b, w)
    wg.grid_vis(g, t, w)
    out = torch.zeros_like(g.data)
    norm = torch.zeros((wl.n_chan, wl.n_pol), dtype=torch.float64, device=dev)
    dropped = torch.full((1,), -1, dtype=torch.int64, device=dev)
    _call(wl, t, b, 1, out, norm, dropped, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert int(dropped.item()) == 0
    want = g.data.cpu().numpy()
    assert rel_l2(out.cpu().numpy(), want) < TOL and max_rel(out.cpu().numpy(), want) < TOL
    assert max_rel(norm.cpu().numpy(), g.normaliser().cpu().numpy()) < TOL


def test_noalloc_rejects_oversized_batches_and_bad_cells():
    import synth
    from gpu_common import gpu_table

    import paper_1403_4209_gb300 as wg
    wl = synth.make("w0_small", n_times=140)            # 496 x 140 = 69,440 records > 65,536
    t = gpu_table(wl)
    batch = wg.VisBatch(torch.as_tensor(wl.uvw, device="cuda"), torch.as_tensor(wl.freq, device="cuda"),
                        wl.vis.cuda(), wl.weight.cuda(), wl.flag.cuda())
    out = torch.zeros((1, wl.n_grid, wl.n_grid, 1), dtype=torch.complex64, device="cuda")
    norm = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    view = GridView(wl.n_grid, 1, 1, 0, wl.du, out.data_ptr(), norm.data_ptr(), None)
    rc = _noalloc_fn()(ctypes.byref(view), t.handle, ctypes.byref(batch.struct), 1, None)
    assert rc == wg.CONST["WG_E_CAPACITY"]
    assert "no-allocation limit" in wg.lib.wg_last_error().decode()
    for du in (float("nan"), float("inf"), 0.0, -wl.du):
        view = GridView(wl.n_grid, 1, 1, 0, du, out.data_ptr(), norm.data_ptr(), None)
        rc = _noalloc_fn()(ctypes.byref(view), t.handle, ctypes.byref(batch.struct), 1, None)
        assert rc == wg.CONST["WG_E_INVALID_ARG"]
        assert "du" in wg.lib.wg_last_error().decode()
    torch.cuda.synchronize()
    assert np.all(out.cpu().numpy() == 0)
