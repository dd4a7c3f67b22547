"""Grid correction, Algorithm "finalizer" (thesis Sec. 4.7), FP64.  Test infrastructure only.

  1. inverse FFT of each polarised grid (centred: u = 0 at N/2 maps to l = 0 at N/2;
     exponent +j2pi(ul + vm), the inverse of the measurement equation's sign);
  2. real part, divided by the normaliser N_p (Jy/beam, Sec. 4.3.2); Stokes I as the mean
     of the parallel hands (polarisations 0 and P-1);
  3. divide by the taper c(l) c(m) = psi_0(c, 2 du l) psi_0(c, 2 du m) (eq. "convgrid");
  4. divide by sinc(pi l du / beta) sinc(pi m du / beta) (eq. "coversampled").

Step 2 with Stokes conversion (grid_correct_stokes): each polarisation's complex image is
normalised by its own N_p, then combined, for linear feeds (XX, XY, YX, YY) as
I = (XX + YY)/2, Q = (XX - YY)/2, U = (XY + YX)/2, V = -j (XY - YX)/2, and for circular feeds
(RR, RL, LR, LL) as I = (RR + LL)/2, V = (RR - LL)/2, Q = (RL + LR)/2, U = -j (RL - LR)/2,
keeping the real part (one Hermitian half is gridded).  Dual polarisation gives I and Q
(linear) or I and V (circular); single polarisation gives I.

Pixel k of an image axis sits at l = (k - N/2) / (N du).
"""
import numpy as np

from .pswf import psi0, bandwidth


def taper_1d(n_grid: int, taper_support: int) -> np.ndarray:
    k = np.arange(n_grid)
    eta = 2.0 * (k - n_grid // 2) / n_grid
    return psi0(bandwidth(taper_support), eta)


def sinc_1d(n_grid: int, beta: int) -> np.ndarray:
    k = np.arange(n_grid)
    x = np.pi * (k - n_grid // 2) / (n_grid * beta)
    return np.where(x == 0, 1.0, np.sin(x) / np.where(x == 0, 1.0, x))


def dirty_complex(grid: np.ndarray) -> np.ndarray:
    """Step 1: [C, N, N, P] -> complex [C, P, N, N] (not normalised)."""
    C, N, _, P = grid.shape
    g = np.moveaxis(grid, 3, 1)
    return np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(g, axes=(-2, -1)), axes=(-2, -1)),
                           axes=(-2, -1)) * (N * N)


def dirty_per_pol(grid: np.ndarray) -> np.ndarray:
    """Step 1 and the real part: [C, N, N, P] -> [C, P, N, N] (not normalised)."""
    return dirty_complex(grid).real


def grid_correct_stokes(grid: np.ndarray, norm: np.ndarray, beta: int, taper_support: int,
                        feeds: str) -> np.ndarray:
    """[C, N, N, P] -> [C, S, N, N]: the Stokes images (I, Q, U, V for P = 4)."""
    C, N, _, P = grid.shape
    nz = np.where(norm != 0, norm, 1.0)
    z = dirty_complex(grid) * np.where(norm != 0, 1.0 / nz, 0.0)[:, :, None, None]
    if P == 1:
        st = [z[:, 0].real]
    elif P == 2:
        st = [0.5 * (z[:, 0] + z[:, 1]).real, 0.5 * (z[:, 0] - z[:, 1]).real]       # I, Q or I, V
    elif feeds == "linear":
        st = [0.5 * (z[:, 0] + z[:, 3]).real, 0.5 * (z[:, 0] - z[:, 3]).real,
              0.5 * (z[:, 1] + z[:, 2]).real, 0.5 * (-1j * (z[:, 1] - z[:, 2])).real]
    elif feeds == "circular":
        st = [0.5 * (z[:, 0] + z[:, 3]).real, 0.5 * (z[:, 1] + z[:, 2]).real,
              0.5 * (-1j * (z[:, 1] - z[:, 2])).real, 0.5 * (z[:, 0] - z[:, 3]).real]
    else:
        raise ValueError(feeds)
    img = np.stack(st, axis=1)
    t = taper_1d(N, taper_support) * sinc_1d(N, beta)
    return img / (t[None, None, :, None] * t[None, None, None, :])


def grid_correct(grid: np.ndarray, norm: np.ndarray, beta: int, taper_support: int,
                 stokes_i: bool = False) -> np.ndarray:
    C, N, _, P = grid.shape
    img = dirty_per_pol(grid) / norm[:, :, None, None]
    t = taper_1d(N, taper_support) * sinc_1d(N, beta)
    img = img / (t[None, None, :, None] * t[None, None, None, :])
    if stokes_i:
        return 0.5 * (img[:, 0] + img[:, P - 1]) if P > 1 else img[:, 0]
    return img
