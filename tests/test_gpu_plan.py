"""Gridder plans (segment length x footprint points per task x per-support or fixed points per
lane): every plan grids the same sums and degrids the same visibilities (the degridder runs the
gridder's tasks), the task count is the one the plan defines, and grid_autotune keeps a
candidate plan and leaves the grid zeroed.

Workload: the w-projection geometry sliced to 300 baselines x 24 steps x 2 channels (32
w-planes, supports 7..45), compressed.  The grid agrees with the FP64 oracle within the FP32
bar of the parity tests (1e-5 rel-L2) under every plan; the task count is compared exactly
with one recomputed on the host from the work list's entries and the table's supports.
Degridding a seeded random grid agrees with the oracle's per-record sums within 1e-5 of their
largest magnitude (FP32 sums of up to 2025 terms), for 4, 2 and 1 polarisations.
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import paper_1403_4209_gb300 as wg
import synth
from gpu_common import max_rel, rel_l2, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

PLANS = [(32, 64, False), (64, 128, False), (128, 256, False), (256, 192, False), (256, 256, False),
         (96, 160, False), (128, 256, True), (64, 128, True), (256, 256, True), (128, 192, True)]


@pytest.fixture(scope="module")
def case():
    wl = synth.make("wproj_2k", n_times=24, n_chan=2, n_baselines=300, flag_frac=0.01)
    return wl, run_oracle(wl), run_gpu(wl)


def _tasks(entries, supports, seg_len, slots):
    n = len(entries)
    k = entries[:, 3] & 0xFFF
    nb = -(-np.asarray(supports)[k] ** 2 // slots)
    return int(sum(nb[i:i + seg_len].max() for i in range(0, n, seg_len)))


@pytest.mark.parametrize("seg_len,slots,fixed_r", PLANS)
def test_plan_grids_the_same_sums(case, seg_len, slots, fixed_r):
    wl, ref, gpu = case
    g, t, batch, wlst = gpu["objects"]
    wlst.plan(t, seg_len, slots, fixed_r)
    assert wlst.plan_params == (seg_len, slots, fixed_r)
    g.zero()
    wg.grid_vis(g, t, wlst)
    torch.cuda.synchronize()
    st = wlst.stats()
    got = g.data.cpu().numpy()
    assert rel_l2(got, ref["grid"]) < 1e-5 and max_rel(got, ref["grid"]) < 1e-4
    assert st["dropped"] == 0
    assert st["tasks"] == _tasks(gpu["entries"], t.supports, seg_len, slots)
    assert max_rel(g.normaliser().cpu().numpy(), ref["norm"]) < 1e-5    # FP32 per-tile partials


def _random_grid(shape, seed):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)


def _degrid_check(wl, pl, table, g, t, batch, wlst, mode, seed):
    y = _random_grid(tuple(g.data.shape), seed)
    want = oracle.degrid(pl, table, y.astype(np.complex128), wl.weight.numpy(), wl.flag.numpy(),
                         adjoint=(mode == wg.DEGRID_ADJOINT))
    g.data.copy_(torch.as_tensor(y))
    got = wg.degrid_vis(g, t, batch, wlst, mode=mode).cpu().numpy().reshape(-1, wl.n_pol)
    assert wlst.stats()["dropped"] == 0
    assert np.array_equal(got[~pl.griddable], np.zeros_like(got[~pl.griddable]))
    assert max_rel(got, want) < 1e-5


@pytest.mark.parametrize("seg_len,slots,fixed_r", PLANS)
def test_plan_degrids_the_same_sums(case, seg_len, slots, fixed_r):
    wl, ref, gpu = case
    g, t, batch, wlst = gpu["objects"]
    wlst.plan(t, seg_len, slots, fixed_r)
    _degrid_check(wl, ref["pl"], ref["table"], g, t, batch, wlst, wg.DEGRID_PREDICT, 11)


@pytest.mark.parametrize("pols", [[0, 3], [0]])
@pytest.mark.parametrize("seg_len,slots,fixed_r", [(128, 256, True), (64, 128, True), (96, 160, False)])
def test_plan_degrids_fewer_polarisations(pols, seg_len, slots, fixed_r):
    full = synth.make("wproj_2k", n_times=16, n_chan=2, n_baselines=200, flag_frac=0.02)
    wl = dataclasses.replace(full, vis=full.vis[..., pols].contiguous(), weight=full.weight[..., pols].contiguous(),
                             flag=full.flag[..., pols].contiguous())
    gpu = run_gpu(wl)
    g, t, batch, wlst = gpu["objects"]
    wlst.plan(t, seg_len, slots, fixed_r)
    ref = run_oracle(wl)
    _degrid_check(wl, ref["pl"], ref["table"], g, t, batch, wlst, wg.DEGRID_ADJOINT, 12)


def test_plan_rejects_bad_parameters(case):
    _, _, gpu = case
    g, t, batch, wlst = gpu["objects"]
    for seg_len, slots in [(16, 128), (512, 128), (100, 128), (128, 32), (128, 288), (128, 100)]:
        with pytest.raises(wg.WgError, match="INVALID_ARG"):
            wlst.plan(t, seg_len, slots)


def test_autotune_keeps_a_candidate_and_zeroes_the_grid(case):
    wl, ref, gpu = case
    g, t, batch, wlst = gpu["objects"]
    cands = [(64, 128, False), (128, 256, True), (128, 256, False)]
    seg, slots, fixed_r, ms = wg.grid_autotune(g, t, wlst, candidates=cands, repeats=2)
    assert (seg, slots, fixed_r) in cands and ms > 0
    torch.cuda.synchronize()
    assert not torch.any(g.data != 0) and not torch.any(g.normaliser() != 0)
    wg.grid_vis(g, t, wlst)
    torch.cuda.synchronize()
    assert rel_l2(g.data.cpu().numpy(), ref["grid"]) < 1e-5
    # the plan carries over to the next batch prepared on this work list
    wg.vis_compress(g, t, batch, wlst)
    assert wlst.plan_params == (seg, slots, fixed_r)
    assert wlst.stats()["tasks"] == _tasks(gpu["entries"], t.supports, seg, slots)
