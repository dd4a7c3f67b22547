"""GPU parity of the batched workload at its own geometry (8192^2 grids, 64 sqrt(w)-spaced
w-planes with supports 9..129, one polarisation, compression on), in the launch configuration
bench.py uses for it (the plan picked by grid_autotune from the batch candidates).

The slice: 4 channels (331-350 MHz, the largest |w| in wavelengths) x 24 time steps x 300
baselines of the 256-station, 10 km log-radial layout.  The steps are the window around the
track's largest |w|; 100 of the baselines are the ones with the largest |w| in that window, so
the records reach the outermost plane (support 129), and 200 are spread over the baseline list.
2 % of the polarisation samples are flagged.

The CUDA path runs the full 64-plane table; the FP64 oracle builds only the planes the slice's
records use (each plane's kernels are computed independently of the others, Algorithm
"convgen"), which bounds its host time to about a minute.  Compared element by element:
  * every record's class bits, the gridded entries and their runs (bit-exact);
  * gamma and N_p (within 1e-5 relative);
  * the four 8192^2 grids (rel-L2 and max-abs within 1e-5 of max|grid|);
  * the kernel table on the planes in use (within 2e-7 of max|C|, FP32 rounding of FP64);
  * degridding of a seeded sample of records, each computed by the oracle from its own FP64
    grid (within 1e-5 of the largest value).
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import paper_1403_4209_gb300 as wg
import synth
from bench import BATCH_PLANS
from gpu_common import max_rel, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5
N_DEGRID = 2048
_PER_RECORD = ("x", "y", "fu", "fv", "k", "psi", "w", "S", "x0", "y0", "z", "zeta_idx", "griddable", "chan")


@pytest.fixture(scope="module")
def case():
    bl, t0 = synth.outer_w_slice("batch_8k", n_times=24, n_top=100, n_spread=200)
    wl = synth.make("batch_8k", baselines=bl, n_times=24, t_start=t0, n_chan=4, chan0=60, flag_frac=0.02)
    assert (wl.n_pol, wl.n_grid, wl.n_wplanes, max(wl.supports)) == (1, 8192, 64, 129)
    dev = "cuda"
    tab = wg.ConvTable.build(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports)
    g = wg.Grid(wl.n_grid, wl.du, wl.n_pol, wl.n_chan, device=dev)
    batch = wg.VisBatch(torch.as_tensor(wl.uvw, device=dev), torch.as_tensor(wl.freq, device=dev), wl.vis.to(dev),
                        wl.weight.to(dev), wl.flag.to(dev))
    wlst = wg.WorkList(wl.rows * wl.n_chan, wl.n_chan, wl.n_pol)
    # the benchmark's set-up for a channel group: autotune on the batch, then zero, prepare, grid
    wg.vis_compress(g, tab, batch, wlst)
    wg.grid_autotune(g, tab, wlst, candidates=BATCH_PLANS, repeats=1)
    g.zero()
    wg.vis_compress(g, tab, batch, wlst)
    wg.grid_vis(g, tab, wlst)
    torch.cuda.synchronize()
    assert wlst.plan_params in [(a, b, c) for a, b, c in BATCH_PLANS]
    st = wlst.stats()
    ent, gam, runs, cls = (x.cpu().numpy() for x in wlst.view(wl.rows * wl.n_chan))
    rows_s = np.sort(np.random.default_rng(1404).choice(wl.rows * wl.n_chan, N_DEGRID, replace=False))
    out = wg.degrid_vis(g, tab, batch, wlst)
    got = {"stats": st, "entries": ent, "gamma": gam, "runs": runs, "cls": cls,
           "grid": g.data.cpu().numpy(), "norm": g.normaliser().cpu().numpy(),
           "degrid": out.reshape(-1, wl.n_pol)[torch.as_tensor(rows_s, device=dev)].cpu().numpy(),
           "table": tab.to_host()}
    del out, g, wlst, batch
    torch.cuda.empty_cache()

    # the oracle: placement needs only the table's layout; then the planes the records use
    vis, w, f = wl.vis.numpy(), wl.weight.numpy(), wl.flag.numpy()
    layout = oracle.build_table(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support,
                                supports=wl.supports, planes=())
    used = np.unique(oracle.place(wl.uvw, wl.freq, wl.du, wl.n_grid, layout, flag=f).k)
    used = used[used < wl.n_wplanes]
    ot = oracle.build_table(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support,
                            supports=wl.supports, planes=used)
    pl = oracle.place(wl.uvw, wl.freq, wl.du, wl.n_grid, ot, flag=f)
    og, oc, lrec, llast, ogamma = oracle.compress(pl, vis, w, f)
    ref = {"pl": pl, "g": og, "c": oc, "lrec": lrec, "llast": llast, "gamma": ogamma, "table": ot, "used": used,
           "grid": oracle.grid_plain(pl, ot, vis, w, f, wl.n_grid), "norm": oracle.normaliser(pl, ot, w, f),
           "stats": oracle.stats(pl, og, oc), "rows_s": rows_s}
    return wl, got, ref


def test_batch8k_slice_reaches_the_outer_planes(case):
    wl, got, ref = case
    pl = ref["pl"]
    S = pl.S[pl.griddable]
    assert S.max() == 129 and S.min() <= 15
    assert len(ref["used"]) >= 48
    assert int(ref["c"].sum()) > 0 and int(ref["g"].sum()) > 0


def test_batch8k_classes_entries_runs_bit_exact(case):
    wl, got, ref = case
    pl, st = ref["pl"], got["stats"]
    cls = got["cls"]
    assert st["dropped"] == 0
    assert np.array_equal(cls & 1, ref["g"].astype(np.uint8))
    assert np.array_equal((cls >> 1) & 1, ref["c"].astype(np.uint8))
    assert np.array_equal((cls >> 2) & 1, pl.griddable.astype(np.uint8))
    assert np.array_equal((cls >> 3) & 1, (pl.psi < 0).astype(np.uint8))
    assert st["records"] == wl.rows * wl.n_chan and st["griddable"] == int(pl.griddable.sum())
    assert st["gridded"] == ref["stats"]["gridded"] and st["compressed"] == ref["stats"]["compressed"]
    assert st["updates"] == ref["stats"]["updates"] * wl.n_pol
    ent, runs, lrec = got["entries"], got["runs"], ref["lrec"]
    assert ent.shape[0] == lrec.shape[0]
    assert np.array_equal(ent[:, 0] & 0xFFFF, pl.x0[lrec])
    assert np.array_equal((ent[:, 0] >> 16) & 0xFFFF, pl.y0[lrec])
    assert np.array_equal(ent[:, 2], pl.z[lrec])
    assert np.array_equal(ent[:, 3] & 0xFFF, pl.k[lrec])
    assert np.array_equal((ent[:, 3] >> 16) & 0xFFFF, pl.chan[lrec])
    S = pl.S[lrec]
    assert np.array_equal(ent[:, 1] & 0xFFFF, (-pl.x0[lrec]) % S)
    assert np.array_equal((ent[:, 1] >> 16) & 0xFFFF, (-pl.y0[lrec]) % S)
    C = wl.n_chan
    assert np.array_equal(runs, np.stack([lrec // C, ref["llast"] // C], 1))
    assert max_rel(got["gamma"], ref["gamma"]) < TOL


def test_batch8k_grid_and_normaliser(case):
    wl, got, ref = case
    assert max_rel(got["norm"], ref["norm"]) < TOL
    G, R = got["grid"], ref["grid"]
    assert rel_l2(G, R) < TOL
    assert max_rel(G, R) < TOL
    for c in range(wl.n_chan):                     # every channel's grid, not only the largest
        assert rel_l2(G[c], R[c]) < TOL


def test_batch8k_table_on_the_planes_in_use(case):
    wl, got, ref = case
    data, zeta, sup, off = got["table"]
    ot = ref["table"]
    assert np.array_equal(sup, ot.supports) and np.array_equal(off, ot.offsets)
    peak = 0.0
    err = 0.0
    for k in ref["used"]:
        n = wl.oversample ** 2 * int(sup[k]) ** 2
        a, b = data[off[k]:off[k] + n], ot.data[off[k]:off[k] + n]
        peak = max(peak, float(np.max(np.abs(b))))
        err = max(err, float(np.max(np.abs(a - b))))
        zk = slice(int(k) * wl.oversample ** 2, (int(k) + 1) * wl.oversample ** 2)
        assert np.max(np.abs(zeta[zk] - ot.zeta[zk])) <= 1e-10 * np.max(np.abs(ot.zeta[zk]))
    assert err <= 2e-7 * peak


def test_batch8k_degrid_sample(case):
    wl, got, ref = case
    pl, rows_s = ref["pl"], ref["rows_s"]
    sub = dataclasses.replace(pl, rows=N_DEGRID, C=1, **{k: getattr(pl, k)[rows_s] for k in _PER_RECORD})
    want = oracle.degrid(sub, ref["table"], ref["grid"])
    out = got["degrid"]
    assert np.array_equal(out[~sub.griddable], np.zeros_like(out[~sub.griddable]))
    assert max_rel(out, want) < TOL
