"""GPU parity at the full size of the w-projection workload, in the launch configuration that
bench.py times.

The batch is the whole workload: 2016 baselines x 3600 steps x 16 channels (120-180 MHz) x 4
polarisations, 116.1 M records, 2048^2 grids, 32 sqrt(w)-spaced planes with supports 9..65,
beta = 8, compression on.  Every channel goes through one vis_compress and one grid_vis under
the plan that grid_autotune picks from the benchmark's candidate list, exactly as in the
benchmark step.

The FP64 oracle then redoes one whole channel of that batch (its 7.26 M records) from the same
seeded inputs, and the test compares, element by element:
  * the class bits of every record and the channel's gridded entries and runs (bit-exact);
  * gamma and N_p (within 1e-5 relative);
  * the channel's 2048^2 x 4 grid (rel-L2 and max-abs within 1e-5);
  * degridding of a seeded sample of the channel's records, each computed one by one by the
    oracle from its own FP64 grid (within 1e-5 of the largest value).
Counts that hold at any size are checked over all 16 channels.
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import paper_1403_4209_gb300 as wg
import synth
from bench import STEP_PLANS
from gpu_common import max_rel, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5
CHAN = 15            # 180 MHz: the longest baselines in wavelengths and the largest |w|
N_DEGRID = 4096      # sampled records for the degridding check

_PER_RECORD = ("x", "y", "fu", "fv", "k", "psi", "w", "S", "x0", "y0", "z", "zeta_idx", "griddable", "chan")


def test_wproj_full_size_one_channel_against_oracle():
    dev = "cuda"
    wl = synth.make("wproj_2k", device=dev)
    assert (wl.rows, wl.n_chan, wl.n_pol, wl.n_grid, wl.n_wplanes) == (2016 * 3600, 16, 4, 2048, 32)
    tab = wg.ConvTable.build(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports)
    g = wg.Grid(wl.n_grid, wl.du, wl.n_pol, wl.n_chan, device=dev)
    batch = wg.VisBatch(torch.as_tensor(wl.uvw, device=dev), torch.as_tensor(wl.freq, device=dev), wl.vis,
                        wl.weight, wl.flag)
    wlst = wg.WorkList(wl.rows * wl.n_chan, wl.n_chan, wl.n_pol)
    # the benchmark's set-up, then one benchmark step: zero, vis_compress, grid_vis
    wg.vis_compress(g, tab, batch, wlst)
    wg.grid_autotune(g, tab, wlst, candidates=STEP_PLANS, repeats=1)
    g.zero()
    wg.vis_compress(g, tab, batch, wlst)
    wg.grid_vis(g, tab, wlst)
    torch.cuda.synchronize()
    assert wlst.plan_params in [(a, b, c) for a, b, c in STEP_PLANS]

    # all channels: counts that hold at any size
    st = wlst.stats()
    assert st["dropped"] == 0
    assert st["records"] == wl.rows * wl.n_chan
    assert st["gridded"] + st["compressed"] == st["griddable"]
    ent, gam, runs, cls = wlst.view(wl.rows * wl.n_chan)
    ent, runs, cls = ent.cpu().numpy(), runs.cpu().numpy(), cls.cpu().numpy()
    assert ent.shape[0] == st["gridded"]
    sup = np.asarray(wl.supports, np.int64)
    assert int((sup[ent[:, 3] & 0xFFF] ** 2).sum()) * wl.n_pol == st["updates"]
    echan = (ent[:, 3] >> 16) & 0xFFFF
    assert np.all(np.diff(echan) >= 0)                 # channel-major
    sel = echan == CHAN
    e_c, runs_c = ent[sel], runs[sel]
    gam_c = gam.cpu().numpy()[sel]
    cls_c = cls.reshape(wl.rows, wl.n_chan)[:, CHAN]
    grid_c = g.data[CHAN].cpu().numpy()
    norm_c = g.normaliser()[CHAN].cpu().numpy()
    del ent, runs, cls, gam

    # degridding of the whole batch (predict mode); a seeded sample of channel CHAN's records
    rows_s = np.sort(np.random.default_rng(1403).choice(wl.rows, N_DEGRID, replace=False))
    out = wg.degrid_vis(g, tab, batch, wlst)
    out_s = out[torch.as_tensor(rows_s, device=dev), CHAN].cpu().numpy()
    del out

    # the oracle on channel CHAN alone, from the same seeded inputs
    vis = wl.vis[:, CHAN:CHAN + 1].cpu().numpy()
    w = wl.weight[:, CHAN:CHAN + 1].cpu().numpy()
    f = wl.flag[:, CHAN:CHAN + 1].cpu().numpy()
    ot = oracle.build_table(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports)
    pl = oracle.place(wl.uvw, np.asarray(wl.freq)[CHAN:CHAN + 1], wl.du, wl.n_grid, ot, flag=f)
    og, oc, lrec, llast, ogamma = oracle.compress(pl, vis, w, f)

    # classes (bit0 g, bit1 c, bit2 griddable, bit3 take-conjugate), entries, runs: bit-exact
    assert np.array_equal(cls_c & 1, og.astype(np.uint8))
    assert np.array_equal((cls_c >> 1) & 1, oc.astype(np.uint8))
    assert np.array_equal((cls_c >> 2) & 1, pl.griddable.astype(np.uint8))
    assert np.array_equal((cls_c >> 3) & 1, (pl.psi < 0).astype(np.uint8))
    assert e_c.shape[0] == lrec.shape[0]
    assert np.array_equal(e_c[:, 0] & 0xFFFF, pl.x0[lrec])
    assert np.array_equal((e_c[:, 0] >> 16) & 0xFFFF, pl.y0[lrec])
    assert np.array_equal(e_c[:, 2], pl.z[lrec])
    assert np.array_equal(e_c[:, 3] & 0xFFF, pl.k[lrec])
    S = pl.S[lrec]
    assert np.array_equal(e_c[:, 1] & 0xFFFF, (-pl.x0[lrec]) % S)
    assert np.array_equal((e_c[:, 1] >> 16) & 0xFFFF, (-pl.y0[lrec]) % S)
    assert np.array_equal(runs_c, np.stack([lrec, llast], 1))     # one channel: record index = row
    assert int(oc.sum()) > 0

    # gamma, normaliser and the channel's grid against FP64
    assert max_rel(gam_c, ogamma) < TOL
    assert max_rel(norm_c, oracle.normaliser(pl, ot, w, f)[0]) < TOL
    ref = oracle.grid_compressed(pl, ot, vis, w, f, wl.n_grid)
    assert rel_l2(grid_c, ref[0]) < TOL
    assert max_rel(grid_c, ref[0]) < TOL

    # degridding: each sampled record one by one from the oracle's own grid
    sub = dataclasses.replace(pl, rows=N_DEGRID, C=1, **{k: getattr(pl, k)[rows_s] for k in _PER_RECORD})
    ref_d = oracle.degrid(sub, ot, ref)
    assert np.array_equal(out_s[~sub.griddable], np.zeros_like(out_s[~sub.griddable]))
    assert max_rel(out_s, ref_d) < TOL
