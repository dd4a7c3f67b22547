"""Precision variants (reduced-precision kernel tables, half-precision visibilities with
per-channel scales, compensated flushes) against the FP64 oracle on the w-projection slice.

The oracle grids the original complex64 visibilities with its FP64 table, so each variant's
error includes its own storage rounding.  Bars follow the storage precision: FP32 paths 1e-5
(rel-L2 and max-abs/max|grid|); FP16 tables or visibilities (11-bit significands, relative
rounding 2^-11 per value) 2e-3; BF16 tables (8-bit significands, 2^-8) 1e-2.  The measured errors
are printed (run with -s).
"""
import numpy as np
import pytest
import torch

import paper_1403_4209_gb300 as wg
import synth
from gpu_common import max_rel, rel_l2, run_oracle

pytestmark = pytest.mark.gpu

VARIANTS = [  # name, table storage, half visibilities, compensated flush, rel-L2 bar
    ("fp32", "f32", False, False, 1e-5),
    ("fp32 + compensated", "f32", False, True, 1e-5),
    ("f16 table + compensated", "f16", False, True, 2e-3),
    ("bf16 table + compensated", "bf16", False, True, 1e-2),
    ("f16 vis + compensated", "f32", True, True, 2e-3),
    ("f16 table + f16 vis + compensated", "f16", True, True, 3e-3),
    ("bf16 table + f16 vis + compensated", "bf16", True, True, 1e-2),
]


def _grid(wl, store, half, comp, plan=None):
    dev = "cuda"
    t = wg.ConvTable.build(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports,
                           store=store)
    g = wg.Grid(wl.n_grid, wl.du, wl.n_pol, wl.n_chan, compensated=comp)
    if half:
        vis, scale = synth.to_half_vis(wl.vis)
        batch = wg.VisBatch(torch.as_tensor(wl.uvw, device=dev), torch.as_tensor(wl.freq, device=dev),
                            vis.to(dev), wl.weight.to(dev), wl.flag.to(dev), vis_scale=scale.to(dev))
    else:
        batch = wg.VisBatch(torch.as_tensor(wl.uvw, device=dev), torch.as_tensor(wl.freq, device=dev),
                            wl.vis.to(dev), wl.weight.to(dev), wl.flag.to(dev))
    wlst = wg.WorkList(wl.rows * wl.n_chan, wl.n_chan, wl.n_pol)
    wg.vis_compress(g, t, batch, wlst)
    if plan is not None:
        wlst.plan(t, *plan)
    wg.grid_vis(g, t, wlst)
    torch.cuda.synchronize()
    assert wlst.stats()["dropped"] == 0
    return g.data.cpu().numpy()


def test_precision_variants_against_oracle():
    wl = synth.make("wproj_2k", n_times=24, n_chan=2, n_baselines=300, flag_frac=0.01)
    ref = run_oracle(wl)["grid"]
    rows = []
    for name, store, half, comp, bar in VARIANTS:
        got = _grid(wl, store, half, comp)
        e2, ea = rel_l2(got, ref), max_rel(got, ref)
        rows.append((name, e2, ea))
        assert e2 < bar and ea < bar * 10, (name, e2, ea)
    print("\nvariant, rel-L2, max-abs/max|grid| (vs FP64 oracle)")
    for name, e2, ea in rows:
        print("  %-36s %.3e  %.3e" % (name, e2, ea))
    # compensation never makes the FP32 path worse
    assert rows[1][1] <= rows[0][1] * 1.05


@pytest.mark.parametrize("store,dtype", [("bf16", torch.bfloat16), ("f16", torch.float16)])
def test_low_precision_table_is_round_to_nearest(store, dtype):
    wl = synth.make("w0_small", n_times=2)
    t = wg.ConvTable.build(wl.du, 1, 0.0, 8, 7, supports=[7], store=store)
    data, _, _, _ = t.to_host()
    ref = torch.view_as_real(torch.as_tensor(data)).to(dtype)               # torch's RNE conversion
    got = t.lp_samples().cpu().view(dtype).reshape(-1, 2)
    assert torch.equal(got.view(torch.int16), ref.view(torch.int16))


@pytest.mark.parametrize("name,store,half,comp,bar", VARIANTS)
def test_precision_variants_fixed_r(name, store, half, comp, bar):
    # the same bars under the fixed R = 8 plan, which every table type and the compensated
    # flush run with their own kernel
    wl = synth.make("wproj_2k", n_times=24, n_chan=2, n_baselines=300, flag_frac=0.01)
    ref = run_oracle(wl)["grid"]
    got = _grid(wl, store, half, comp, plan=(256, 256, True))
    assert rel_l2(got, ref) < bar and max_rel(got, ref) < bar * 10, name
