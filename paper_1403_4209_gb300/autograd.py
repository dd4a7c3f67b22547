"""Differentiable sky -> visibility model: degridding forward, hand-written gridding backward.

SkyModel(x) = A x: a real image x [n_chan][n_pol][N][N] is divided by the grid-correction
function (taper x sinc of the image finaliser, Sec. 4.7), transformed to a grid with the centred
forward FFT (grid_correct's transpose mode) and degridded (degrid_vis, PREDICT) into visibilities
[rows][n_chan][n_pol] for the fixed uvw, frequencies and flags given at construction.

The backward pass is the exact adjoint A^H under the real inner product, with no tracing: the
incoming gradient is gridded with unit weights (vis_compress with WG_PREP_UNWEIGHTED + grid_vis),
transformed back and divided by taper x sinc (grid_correct, IMAGE_PER_POL_RAW).  Kernel samples
are read from the table on every pass; nothing is stored per visibility.  With torch's
convention for complex outputs, the gradient of sum |A x - v|^2 is 2 A^H (A x - v).
"""
import torch

from .api import (DEGRID_PREDICT, IMAGE_PER_POL_RAW, Grid, VisBatch, WorkList, degrid_vis, grid_correct, grid_vis,
                  image_to_grid, vis_compress)


class SkyModel:
    def __init__(self, table, uvw: torch.Tensor, freq: torch.Tensor, weight: torch.Tensor, flag: torch.Tensor,
                 n_grid: int, du: float, compress: bool = True):
        rows, C, P = weight.shape
        self.table = table
        self.compress = compress
        self.shape = (C, P, n_grid, n_grid)
        self.grid_fwd = Grid(n_grid, du, P, C, device=weight.device)
        self.grid_adj = Grid(n_grid, du, P, C, device=weight.device)
        self.wl_fwd = WorkList(max(1, rows * C), C, P)
        self.wl_adj = WorkList(max(1, rows * C), C, P)
        zeros = torch.zeros((rows, C, P), dtype=torch.complex64, device=weight.device)
        self.batch = VisBatch(uvw, freq, zeros, weight, flag)
        vis_compress(self.grid_fwd, table, self.batch, self.wl_fwd, compress=compress)

    def forward_vis(self, image: torch.Tensor) -> torch.Tensor:
        image_to_grid(self.grid_fwd, self.table, image.detach().contiguous())
        return degrid_vis(self.grid_fwd, self.table, self.batch, self.wl_fwd, mode=DEGRID_PREDICT)

    def adjoint_image(self, vis: torch.Tensor) -> torch.Tensor:
        b = VisBatch(self.batch.uvw, self.batch.freq, vis.detach().contiguous(), self.batch.weight, self.batch.flag)
        vis_compress(self.grid_adj, self.table, b, self.wl_adj, compress=self.compress, unweighted=True)
        self.grid_adj.zero()
        grid_vis(self.grid_adj, self.table, self.wl_adj)
        return grid_correct(self.grid_adj, self.table, mode=IMAGE_PER_POL_RAW)

    def __call__(self, image: torch.Tensor) -> torch.Tensor:
        return DegridFn.apply(image, self)


class DegridFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, image, model):
        if tuple(image.shape) != model.shape or image.dtype != torch.float32:
            raise ValueError("image must be float32 of shape %s" % (model.shape,))
        ctx.model = model
        return model.forward_vis(image)

    @staticmethod
    def backward(ctx, vis_grad):
        return ctx.model.adjoint_image(vis_grad), None
