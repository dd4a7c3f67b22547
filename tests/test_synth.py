"""The seeded synthetic workloads have the shapes that the benchmark and the parity tests are
quoted on.  They stand in for the thesis's LOFAR data sets.  The test checks station and
baseline counts, time steps, channel frequencies, polarisations, grid side, w-planes, the odd
support schedule, and oversampling.  It also checks that every record of slices across the
whole array and the whole track is griddable (the cell-size and w_max rules), that
auto-correlations are excluded, that the records are baseline-major and time-minor, and
that the same call gives the same inputs."""
import numpy as np
import pytest

import oracle
import synth
from oracle.table import Table

# name: baselines, steps, channels, first and last frequency (Hz), pols, grid side, planes,
#       first and last support
SPEC = {
    "w0_small": (496, 256, 1, 150e6, 150e6, 1, 512, 1, 7, 7),
    "wproj_2k": (2016, 3600, 16, 120e6, 180e6, 4, 2048, 32, 9, 65),
    "degrid_1k": (2016, 600, 4, 120e6, 180e6, 4, 1024, 16, 9, 33),
    "batch_8k": (32640, 1800, 64, 50e6, 350e6, 1, 8192, 64, 9, 129),
    "mfs_2k": (2016, 3600, 16, 150e6, 150e6 + 15 * 195312.5 / 16, 4, 2048, 32, 9, 65),
}


def _placement_table(wl):
    """A table with the workload's planes and supports (sample values are not needed to place)."""
    sup = np.asarray(wl.supports, np.int32)
    off = np.concatenate([[0], np.cumsum(wl.oversample ** 2 * sup.astype(np.int64) ** 2)[:-1]])
    planes = oracle.table.w_plane_values(wl.n_wplanes, wl.w_max)
    return Table(wl.oversample, sup, off.astype(np.int64), np.zeros(1, complex), np.zeros(1), planes, wl.w_max)


@pytest.mark.parametrize("name", sorted(SPEC))
def test_workload_shapes_and_rules(name):
    nb, T, C, f0, f1, P, N, K, s0, s1 = SPEC[name]
    across = synth.make(name, n_times=2)                    # every baseline, every channel
    along = synth.make(name, n_baselines=2, n_chan=1)       # whole tracks of two baselines
    assert across.n_baselines == nb and along.n_times == T
    assert across.rows == nb * 2 and along.rows == 2 * T
    assert across.n_chan == C and across.n_pol == P
    assert abs(across.freq[0] - f0) <= 1e-9 * f0 and abs(across.freq[-1] - f1) <= 1e-9 * f1
    if C > 1:
        d = np.diff(across.freq)
        assert np.all(d > 0) and np.max(np.abs(d - d[0])) <= 1e-6 * d[0]
    assert (across.n_grid, across.n_wplanes, across.oversample) == (N, K, 8)
    sup = np.asarray(across.supports)
    assert sup[0] == s0 and sup[-1] == s1 and np.all(sup % 2 == 1) and np.all(np.diff(sup) >= 0)
    # slices share the whole workload's cell size and w_max
    assert (along.du, along.w_max) == (across.du, across.w_max)
    # no auto-correlations: every baseline has a non-zero length
    assert np.all(np.abs(across.uvw).max(axis=1) > 0)
    # every footprint fits the grid and every |w| lies inside the last plane (flags are 0)
    for wl in (across, along):
        pl = oracle.place(wl.uvw, wl.freq, wl.du, wl.n_grid, _placement_table(wl), flag=wl.flag.numpy())
        assert pl.griddable.all()
    # baseline-major, time-minor: each baseline's track moves by a small step per time step
    tr = along.uvw.reshape(2, T, 3)
    step = np.abs(np.diff(tr, axis=1)).max()
    assert step <= 0.01 * np.abs(tr).max()


def test_seeded_inputs_repeat():
    a = synth.make("wproj_2k", n_times=8, n_chan=2, n_baselines=50, flag_frac=0.02)
    b = synth.make("wproj_2k", n_times=8, n_chan=2, n_baselines=50, flag_frac=0.02)
    assert np.array_equal(a.uvw, b.uvw)
    assert np.array_equal(a.vis.numpy(), b.vis.numpy()) and np.array_equal(a.flag.numpy(), b.flag.numpy())
    assert a.flag.numpy().any() and not a.flag.numpy().all()
