"""Host-side behaviour of the binding and of the input generator that needs no GPU: a grid view
must be a contiguous complex64 CUDA tensor of its shape (checked before the library is called),
and half-precision visibilities carry per-channel scales max|vis| / 60000 that bring them
back within float16 rounding."""
import numpy as np
import pytest
import torch

import paper_1403_4209_gb300 as wg
import synth


@pytest.mark.parametrize("storage", [
    torch.zeros((1, 16, 16, 1), dtype=torch.complex64),                 # host memory
    torch.zeros((1, 16, 16, 1), dtype=torch.complex128),                # wrong type
    torch.zeros((2, 16, 16, 1), dtype=torch.complex64),                 # wrong shape
])
def test_grid_storage_is_checked_before_the_library(storage):
    with pytest.raises(ValueError, match="storage"):
        wg.Grid(16, 1.0, 1, 1, storage=storage)


def test_half_visibilities_and_scales():
    wl = synth.make("wproj_2k", n_times=4, n_chan=3, n_baselines=40)
    vh, scale = synth.to_half_vis(wl.vis)
    assert vh.dtype == torch.complex32 and scale.dtype == torch.float32 and scale.shape == (3,)
    v = wl.vis.numpy()
    amax = np.abs(v).max(axis=(0, 2))
    assert np.allclose(scale.numpy(), amax / 60000.0, rtol=1e-6)
    back = vh.to(torch.complex64).numpy() * scale.numpy()[None, :, None]
    # float16 keeps 11 significant bits: relative rounding <= 2^-11 of each component
    err = np.abs(back - v)
    assert np.all(err <= 2.0 ** -11 * (np.abs(v.real) + np.abs(v.imag)) + 1e-12)
