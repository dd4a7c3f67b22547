"""Shared helpers for the GPU parity tests: run one seeded workload through the CUDA path (via
the C ABI) and through the FP64 oracle, independently.  Nothing the CUDA path computes is fed
to the oracle."""
import numpy as np
import torch

import oracle


def gpu_table(wl, n_k=0, supports="prescribed", threshold=1e-3):
    import paper_1403_4209_gb300 as wg
    sup = wl.supports if supports == "prescribed" else None
    return wg.ConvTable.build(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=sup,
                              n_k=n_k, threshold=threshold)


def oracle_table(wl, n_k=None, supports="prescribed", threshold=1e-3):
    sup = wl.supports if supports == "prescribed" else None
    return oracle.build_table(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=sup,
                              n_k=n_k, threshold=threshold)


def run_gpu(wl, table=None, compress=True, n_k=0):
    import paper_1403_4209_gb300 as wg
    dev = "cuda"
    t = table if table is not None else gpu_table(wl, n_k=n_k)
    g = wg.Grid(wl.n_grid, wl.du, wl.n_pol, wl.n_chan)
    batch = wg.VisBatch(torch.as_tensor(wl.uvw, device=dev), torch.as_tensor(wl.freq, device=dev),
                        wl.vis.to(dev), wl.weight.to(dev), wl.flag.to(dev))
    wlst = wg.WorkList(max(1, wl.rows * wl.n_chan), wl.n_chan, wl.n_pol)
    wg.vis_compress(g, t, batch, wlst, compress=compress)
    wg.grid_vis(g, t, wlst)
    torch.cuda.synchronize()
    st = wlst.stats()
    ent, gam, runs, cls = wlst.view(wl.rows * wl.n_chan)
    return {"grid": g.data.cpu().numpy(), "norm": g.normaliser().cpu().numpy(), "stats": st,
            "entries": ent.cpu().numpy(), "gamma": gam.cpu().numpy(), "runs": runs.cpu().numpy(),
            "rec_class": cls.cpu().numpy(), "objects": (g, t, batch, wlst)}


def run_oracle(wl, table=None, compress=True, n_k=None):
    t = table if table is not None else oracle_table(wl, n_k=n_k)
    vis, w, f = wl.vis.cpu().numpy(), wl.weight.cpu().numpy(), wl.flag.cpu().numpy()
    pl = oracle.place(wl.uvw, wl.freq, wl.du, wl.n_grid, t, flag=f)
    grid = oracle.grid_plain(pl, t, vis, w, f, wl.n_grid)
    if compress:
        g, c, lrec, llast, gamma = oracle.compress(pl, vis, w, f)
    else:
        g, c = pl.griddable.copy(), np.zeros_like(pl.griddable)
        idx = np.nonzero(pl.griddable)[0]
        lrec = idx[np.lexsort((idx // wl.n_chan, idx % wl.n_chan))]   # channel-major, then row
        llast = lrec.copy()
        q = oracle.weighted_vis(pl, vis, w, f)
        gamma = q[lrec]
    st = oracle.stats(pl, g, c)
    norm = oracle.normaliser(pl, t, w, f)
    return {"grid": grid, "norm": norm, "stats": st, "pl": pl, "g": g, "c": c, "lrec": lrec, "llast": llast,
            "gamma": gamma, "table": t}


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def max_rel(a, b):
    m = np.max(np.abs(b)) if b.size else 0.0
    return np.max(np.abs(a - b)) / (m if m > 0 else 1.0) if a.size else 0.0
