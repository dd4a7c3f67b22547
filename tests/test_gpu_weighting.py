"""Uniform and robust weighting on the GPU (vis_weight) against the FP64 oracle
(oracle/weighting.py): every new weight within 1e-5 relative (the density grid is summed in
FP32 atomics); records that are not griddable keep their weights exactly.  Workloads: the
w-projection geometry (300 baselines x 40 steps x 2 channels, 5 % flags, random weights
U(0.5, 2)) per channel, and the narrow-channel mfs geometry interleaved onto one grid."""
import numpy as np
import pytest
import torch

import oracle
import paper_1403_4209_gb300 as wg
import synth
from gpu_common import gpu_table, oracle_table
from oracle.weighting import reweight

pytestmark = pytest.mark.gpu


def _case(name, interleave):
    wl = synth.make(name, n_times=40, n_chan=2 if not interleave else 4, n_baselines=300, flag_frac=0.05)
    rng = np.random.default_rng(12)
    w = rng.uniform(0.5, 2.0, wl.weight.shape).astype(np.float32)
    dev = "cuda"
    t = gpu_table(wl)
    g = wg.Grid(wl.n_grid, wl.du, wl.n_pol, 1 if interleave else wl.n_chan)
    b = wg.VisBatch(torch.as_tensor(wl.uvw, device=dev), torch.as_tensor(wl.freq, device=dev), wl.vis.to(dev),
                    torch.as_tensor(w, device=dev), wl.flag.to(dev))
    ot = oracle_table(wl)
    pl = oracle.place(wl.uvw, wl.freq, wl.du, wl.n_grid, ot, flag=wl.flag.numpy())
    return wl, w, g, t, b, pl


@pytest.mark.parametrize("name,interleave", [("wproj_2k", False), ("mfs_2k", True)])
@pytest.mark.parametrize("scheme,robust", [("uniform", 0.0), ("robust", 0.0), ("robust", -1.0), ("robust", 1.5)])
def test_weights_match_oracle(name, interleave, scheme, robust):
    wl, w, g, t, b, pl = _case(name, interleave)
    got = wg.vis_weight(g, t, b, scheme=scheme, robust=robust, interleave=interleave).cpu().numpy().reshape(-1, wl.n_pol)
    exp = reweight(pl, w, wl.flag.numpy(), wl.n_grid, scheme, robust=robust, interleave=interleave)
    sel = pl.griddable
    assert np.array_equal(got[~sel], w.reshape(-1, wl.n_pol)[~sel])
    assert np.max(np.abs(got[sel] - exp[sel]) / np.maximum(np.abs(exp[sel]), 1e-30)) < 1e-5
    assert sel.sum() > 0.5 * sel.size


def test_in_place_weights_and_gridding_with_them():
    wl, w, g, t, b, pl = _case("wproj_2k", False)
    wg.vis_weight(g, t, b, scheme="uniform", out=b.weight)             # in place
    wk = wg.WorkList(wl.rows * wl.n_chan, wl.n_chan, wl.n_pol)
    wg.vis_compress(g, t, b, wk)
    wg.grid_vis(g, t, wk)
    torch.cuda.synchronize()
    ot = oracle_table(wl)
    uw = reweight(pl, w, wl.flag.numpy(), wl.n_grid, "uniform").reshape(w.shape)
    G = oracle.grid_plain(pl, ot, wl.vis.numpy(), uw, wl.flag.numpy(), wl.n_grid)
    got = g.data.cpu().numpy()
    assert np.linalg.norm(got - G) / np.linalg.norm(G) < 1e-5
