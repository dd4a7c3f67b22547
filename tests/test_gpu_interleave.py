"""Channel interleaving on the GPU (WG_PREP_INTERLEAVE: all channels onto one grid, compression
over the natural record order) against the FP64 oracle, bit-exact for the classification,
statistics, entries and runs, within the FP32 bar (1e-5) for gamma, N_p, the grid and the
degridded visibilities.  Workload: the narrow-channel mfs_2k geometry (12.2 kHz channels at
150 MHz) sliced to 200 baselines x 30 steps x 5 channels, 2 % flags."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import paper_1403_4209_gb300 as wg
import synth
from gpu_common import gpu_table, max_rel, oracle_table, rel_l2
from oracle.grid import compress, degrid, grid_plain, normaliser, stats

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    wl = synth.make("mfs_2k", n_times=30, n_chan=5, n_baselines=200, flag_frac=0.02)
    dev = "cuda"
    t = gpu_table(wl)
    g = wg.Grid(wl.n_grid, wl.du, wl.n_pol, 1)
    b = wg.VisBatch(torch.as_tensor(wl.uvw, device=dev), torch.as_tensor(wl.freq, device=dev), wl.vis.to(dev),
                    wl.weight.to(dev), wl.flag.to(dev))
    w = wg.WorkList(wl.rows * wl.n_chan, wl.n_chan, wl.n_pol)
    wg.vis_compress(g, t, b, w, interleave=True)
    wg.grid_vis(g, t, w)
    torch.cuda.synchronize()
    ot = oracle_table(wl)
    vis, wt, f = wl.vis.numpy(), wl.weight.numpy(), wl.flag.numpy()
    pl = oracle.place(wl.uvw, wl.freq, wl.du, wl.n_grid, ot, flag=f)
    og, oc, lrec, llast, gamma = compress(pl, vis, wt, f, interleave=True)
    ref = {"pl": pl, "g": og, "c": oc, "lrec": lrec, "llast": llast, "gamma": gamma, "table": ot,
           "grid": grid_plain(pl, ot, vis, wt, f, wl.n_grid, interleave=True),
           "norm": normaliser(pl, ot, wt, f, interleave=True), "stats": stats(pl, og, oc)}
    return wl, (g, t, b, w), ref


def test_interleaved_classification_and_lists_bit_exact(case):
    wl, (g, t, b, w), ref = case
    n = wl.rows * wl.n_chan
    ent, gam, runs, cls = (x.cpu().numpy() for x in w.view(n))
    assert np.array_equal(cls & 1, ref["g"].astype(np.uint8))
    assert np.array_equal((cls >> 1) & 1, ref["c"].astype(np.uint8))
    assert ref["c"].sum() > 0
    st = w.stats()
    assert st["gridded"] == ref["stats"]["gridded"] and st["compressed"] == ref["stats"]["compressed"]
    assert st["updates"] == ref["stats"]["updates"] * wl.n_pol and st["dropped"] == 0
    pl = ref["pl"]
    # one list in record order: entries, their runs (first and last record) and channel 0
    assert np.array_equal(runs[:, 0], ref["lrec"]) and np.array_equal(runs[:, 1], ref["llast"])
    assert np.all((ent[:, 3] >> 16) == 0)
    assert np.array_equal(ent[:, 2], pl.z[ref["lrec"]])
    assert max_rel(gam, ref["gamma"]) < 1e-5


def test_interleaved_grid_and_normaliser(case):
    wl, (g, t, b, w), ref = case
    got = g.data.cpu().numpy()
    assert got.shape[0] == 1
    assert rel_l2(got, ref["grid"]) < 1e-5 and max_rel(got, ref["grid"]) < 1e-5
    assert max_rel(g.normaliser().cpu().numpy(), ref["norm"]) < 1e-5


def test_interleaved_degrid_fans_out_over_records(case):
    wl, (g, t, b, w), ref = case
    out = wg.degrid_vis(g, t, b, w, mode=wg.DEGRID_ADJOINT)
    torch.cuda.synchronize()
    G = g.data.cpu().numpy().astype(np.complex128)
    exp = degrid(ref["pl"], ref["table"], G, wl.weight.numpy(), wl.flag.numpy(), adjoint=True, interleave=True)
    got = out.cpu().numpy().reshape(-1, wl.n_pol)
    assert np.max(np.abs(got - exp)) <= 1e-5 * np.max(np.abs(exp))


def test_interleave_needs_a_one_channel_grid(case):
    wl, (g, t, b, w), ref = case
    g2 = wg.Grid(wl.n_grid, wl.du, wl.n_pol, wl.n_chan)
    with pytest.raises(wg.WgError, match="SHAPE"):
        wg.vis_compress(g2, t, b, w, interleave=True)
