"""Batching through WG_PREP_APPEND (Sec. 5.4: many channels in one gridder launch): channel
groups prepared one after another into one work list, each onto its slice of one grid, then a
single grid_vis over all of them.  The grid and the normaliser must equal those of the whole
batch prepared at once and those of the FP64 oracle, within the parity bar; the statistics
must add up over the groups; a work list holding appended batches refuses degridding; and
entries past the work list's entry capacity are dropped and counted, not written."""
import numpy as np
import pytest
import torch

import synth
from gpu_common import gpu_table, max_rel, rel_l2, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _groups(wl, size):
    """The workload's channels as consecutive groups of `size` channels (device tensors)."""
    dev = "cuda"
    out = []
    for c0 in range(0, wl.n_chan, size):
        sl = slice(c0, c0 + size)
        out.append((c0, torch.as_tensor(wl.freq[sl], device=dev), wl.vis[:, sl].contiguous().to(dev),
                    wl.weight[:, sl].contiguous().to(dev), wl.flag[:, sl].contiguous().to(dev)))
    return out


def _append_all(wg, g, t, wlst, uvw, groups):
    wlst.clear()
    for c0, freq, vis, w, f in groups:
        b = wg.VisBatch(uvw, freq, vis, w, f)
        wg.vis_compress(g, t, b, wlst, append=True, chan0=c0)
    wg.grid_vis(g, t, wlst)
    torch.cuda.synchronize()


def test_appended_groups_match_one_batch_and_the_oracle():
    import paper_1403_4209_gb300 as wg
    wl = synth.make("wproj_2k", n_chan=4, n_times=60, n_baselines=300, flag_frac=0.02)
    ref = run_gpu(wl)                         # the whole batch at once
    orc = run_oracle(wl)
    t = ref["objects"][1]
    uvw = torch.as_tensor(wl.uvw, device="cuda")
    groups = _groups(wl, 2)
    g = wg.Grid(wl.n_grid, wl.du, wl.n_pol, wl.n_chan)
    wlst = wg.WorkList(wl.rows * 2, 2, wl.n_pol, max_entries=wl.rows * wl.n_chan)
    for rep in range(2):                      # the work list is cleared and reused
        g.zero()
        _append_all(wg, g, t, wlst, uvw, groups)
        got, got_n = g.data.cpu().numpy(), g.normaliser().cpu().numpy()
        for want, want_n in ((ref["grid"], ref["norm"]), (orc["grid"], orc["norm"])):
            assert rel_l2(got, want) < TOL and max_rel(got, want) < TOL
            assert max_rel(got_n, want_n) < TOL
        st = wlst.stats()
        assert st["dropped"] == 0
        for k in ("records", "griddable", "gridded", "compressed", "updates", "updates_saved"):
            assert st[k] == ref["stats"][k], (rep, k)
        assert st["gridded"] == orc["stats"]["gridded"] and st["compressed"] == orc["stats"]["compressed"]


def test_append_rules():
    import paper_1403_4209_gb300 as wg
    wl = synth.make("wproj_2k", n_chan=4, n_times=20, n_baselines=100)
    t = gpu_table(wl)
    uvw = torch.as_tensor(wl.uvw, device="cuda")
    groups = _groups(wl, 2)
    g = wg.Grid(wl.n_grid, wl.du, wl.n_pol, wl.n_chan)
    wlst = wg.WorkList(wl.rows * 2, 2, wl.n_pol, max_entries=wl.rows * wl.n_chan)
    c0, freq, vis, w, f = groups[1]
    b = wg.VisBatch(uvw, freq, vis, w, f)
    with pytest.raises(RuntimeError, match="exceed the grid"):        # channels 3..4 of 4
        wg.vis_compress(g, t, b, wlst, append=True, chan0=3)
    _append_all(wg, g, t, wlst, uvw, groups)
    out = torch.empty_like(vis)
    with pytest.raises(RuntimeError, match="APPEND"):                 # no degridding accumulator
        wg.degrid_vis(g, t, b, wlst, out=out)
    # a work list holding a batch prepared without the flag must be cleared before appending
    w2 = wg.WorkList(wl.rows * 2, 2, wl.n_pol)
    g2 = wg.Grid(wl.n_grid, wl.du, wl.n_pol, 2)
    wg.vis_compress(g2, t, b, w2)
    with pytest.raises(RuntimeError, match="worklist_clear"):
        wg.vis_compress(g, t, b, w2, append=True, chan0=2)


def test_entries_past_the_capacity_are_dropped_and_counted():
    import paper_1403_4209_gb300 as wg
    wl = synth.make("wproj_2k", n_chan=4, n_times=20, n_baselines=100)
    t = gpu_table(wl)
    uvw = torch.as_tensor(wl.uvw, device="cuda")
    groups = _groups(wl, 2)
    g = wg.Grid(wl.n_grid, wl.du, wl.n_pol, wl.n_chan)
    full = wg.WorkList(wl.rows * 2, 2, wl.n_pol, max_entries=wl.rows * wl.n_chan)
    _append_all(wg, g, t, full, uvw, groups)
    n_all = full.stats()["gridded"]
    cap = n_all // 3
    g.zero()
    small = wg.WorkList(wl.rows * 2, 2, wl.n_pol, max_entries=cap)
    _append_all(wg, g, t, small, uvw, groups)
    st = small.stats()
    assert st["dropped"] > 0
    ent, _, _, _ = small.view(wl.rows * 2)
    assert 0 < ent.shape[0] <= cap
    assert np.isfinite(g.data.cpu().numpy()).all()
