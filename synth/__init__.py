"""Seeded synthetic interferometer inputs, shaped like the thesis's LOFAR workloads.

This module produces *inputs only*: station layouts, Earth-rotation uvw tracks,
channel frequencies, and visibilities from the measurement equation (Sec. 1.3,
eq. "measurmentrewritten") for a handful of point sources plus Gaussian noise.
It holds none of the gridding method's arithmetic (no placement, no kernels, no
compression) and is shared by the CUDA path's tests/bench and the oracle.

Record order is baseline-major, time-minor (Sec. 2.5 and Sec. 4.3: records of a
baseline are grouped and sorted by time).  Auto-correlations are excluded.

uvw follows the textbook equatorial rotation (Thompson, Moran & Swenson eq. 4.1):
station offsets in local East/North/Up are rotated to equatorial (X, Y, Z) at the
array latitude, then projected for hour angle H and declination dec.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np
import torch

C0 = 299_792_458.0          # speed of light [m/s]
OMEGA_EARTH = 7.2921159e-5  # sidereal rotation rate [rad/s]
LOFAR_LAT_DEG = 52.9


# ----------------------------------------------------------------------------------
# station layouts (ENU metres)
# ----------------------------------------------------------------------------------
def stations_uniform_disk(n: int, diameter_m: float, rng: np.random.Generator) -> np.ndarray:
    r = 0.5 * diameter_m * np.sqrt(rng.random(n))
    t = 2 * np.pi * rng.random(n)
    up = rng.normal(0.0, 1.0, n)
    return np.stack([r * np.cos(t), r * np.sin(t), up], axis=1)


def stations_gaussian(n: int, extent_m: float, rng: np.random.Generator) -> np.ndarray:
    """2-D Gaussian density whose radius extent_m/2 holds 95% of the stations."""
    sigma = 0.5 * extent_m / math.sqrt(2.0 * math.log(20.0))
    e = rng.normal(0.0, sigma, n)
    nn = rng.normal(0.0, sigma, n)
    up = rng.normal(0.0, 1.0, n)
    return np.stack([e, nn, up], axis=1)


def stations_log_radial(n: int, r_max_m: float, rng: np.random.Generator,
                        r_min_m: float = 30.0) -> np.ndarray:
    r = np.exp(rng.uniform(math.log(r_min_m), math.log(r_max_m), n))
    t = 2 * np.pi * rng.random(n)
    up = rng.normal(0.0, 2.0, n)
    return np.stack([r * np.cos(t), r * np.sin(t), up], axis=1)


def baseline_pairs(n_st: int) -> np.ndarray:
    i, j = np.triu_indices(n_st, k=1)
    return np.stack([i, j], axis=1)


def uvw_tracks(enu: np.ndarray, n_times: int, dt_s: float, dec_deg: float,
               lat_deg: float = LOFAR_LAT_DEG, baselines: Optional[np.ndarray] = None) -> np.ndarray:
    """uvw in metres, shape [n_baselines * n_times, 3], baseline-major, time-minor.

    Hour angle runs symmetrically about transit."""
    if baselines is None:
        baselines = baseline_pairs(enu.shape[0])
    lat = math.radians(lat_deg)
    dec = math.radians(dec_deg)
    b = enu[baselines[:, 1]] - enu[baselines[:, 0]]          # [B, 3] ENU
    E, N, U = b[:, 0], b[:, 1], b[:, 2]
    X = -math.sin(lat) * N + math.cos(lat) * U
    Y = E
    Z = math.cos(lat) * N + math.sin(lat) * U
    t = (np.arange(n_times) - 0.5 * (n_times - 1)) * dt_s
    H = OMEGA_EARTH * t                                        # [T]
    sH, cH = np.sin(H)[None, :], np.cos(H)[None, :]
    X, Y, Z = X[:, None], Y[:, None], Z[:, None]
    u = sH * X + cH * Y
    v = -math.sin(dec) * cH * X + math.sin(dec) * sH * Y + math.cos(dec) * Z
    w = math.cos(dec) * cH * X - math.cos(dec) * sH * Y + math.sin(dec) * Z
    uvw = np.stack([u, v, w], axis=-1).reshape(-1, 3)
    return np.ascontiguousarray(uvw, dtype=np.float64)


# ----------------------------------------------------------------------------------
# sky and visibilities
# ----------------------------------------------------------------------------------
@dataclasses.dataclass
class Sky:
    flux: np.ndarray   # [S] Jy
    l: np.ndarray      # [S] direction cosines
    m: np.ndarray


def point_sources(n: int, rng: np.random.Generator, flux=(0.1, 1.0), max_offset_deg=1.0) -> Sky:
    flux_v = rng.uniform(flux[0], flux[1], n)
    off = np.radians(rng.uniform(-max_offset_deg, max_offset_deg, (n, 2)))
    return Sky(flux_v, np.sin(off[:, 0]), np.sin(off[:, 1]))


def visibilities(uvw_m: np.ndarray, freq_hz: np.ndarray, sky: Sky, n_pol: int,
                 noise_sigma: float, seed: int, device: str = "cpu",
                 rows_per_block: int = 1 << 18) -> torch.Tensor:
    """complex64 [rows, C, P]: V(u,v,w) = sum_s S_s exp(-j2pi(u l + v m + w(n-1))) + noise.

    The parallel-hand polarisations (0 and P-1) carry the unpolarised sky; cross
    hands carry noise only.  Computed in float64 on `device`, stored complex64."""
    rows = uvw_m.shape[0]
    C = freq_hz.shape[0]
    out = torch.empty((rows, C, n_pol), dtype=torch.complex64, device=device)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    lam_inv = torch.as_tensor(freq_hz / C0, dtype=torch.float64, device=device)
    fl = torch.as_tensor(sky.flux, dtype=torch.float64, device=device)
    ll = torch.as_tensor(sky.l, dtype=torch.float64, device=device)
    mm = torch.as_tensor(sky.m, dtype=torch.float64, device=device)
    nm1 = -(ll * ll + mm * mm) / (1.0 + torch.sqrt(1.0 - ll * ll - mm * mm))
    for r0 in range(0, rows, rows_per_block):
        r1 = min(rows, r0 + rows_per_block)
        uvw = torch.as_tensor(uvw_m[r0:r1], dtype=torch.float64, device=device)
        # phase per (row, chan, src)
        geo = (uvw[:, 0:1] * ll[None, :] + uvw[:, 1:2] * mm[None, :]
               + uvw[:, 2:3] * nm1[None, :])                              # [R, S] metres
        ph = -2.0 * math.pi * geo[:, None, :] * lam_inv[None, :, None]     # [R, C, S]
        v = (fl[None, None, :] * torch.exp(1j * ph)).sum(-1)               # [R, C]
        blk = torch.zeros((r1 - r0, C, n_pol), dtype=torch.complex128, device=device)
        blk[:, :, 0] = v
        if n_pol > 1:
            blk[:, :, n_pol - 1] = v
        if noise_sigma > 0:
            nr = torch.randn((r1 - r0, C, n_pol), generator=g, device=device, dtype=torch.float64)
            ni = torch.randn((r1 - r0, C, n_pol), generator=g, device=device, dtype=torch.float64)
            blk = blk + noise_sigma * torch.complex(nr, ni)
        out[r0:r1] = blk.to(torch.complex64)
    return out


# ----------------------------------------------------------------------------------
# workload descriptions (shapes of the thesis's experiments on its LOFAR data sets)
# ----------------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    uvw: np.ndarray            # [rows, 3] float64 metres
    freq: np.ndarray           # [C] float64 Hz
    vis: torch.Tensor          # [rows, C, P] complex64
    weight: torch.Tensor       # [rows, C, P] float32
    flag: torch.Tensor         # [rows, C, P] uint8
    n_grid: int
    du: float                  # cell size, wavelengths
    n_wplanes: int
    w_max: float               # wavelengths
    oversample: int
    supports: list             # prescribed odd supports per w-plane
    taper_support: int
    n_baselines: int
    n_times: int

    @property
    def rows(self):
        return self.uvw.shape[0]

    @property
    def n_chan(self):
        return self.freq.shape[0]

    @property
    def n_pol(self):
        v = self.vis[0] if isinstance(self.vis, list) else self.vis
        return v.shape[2]

    @property
    def chan_groups(self):
        """[(c0, c1)] channel ranges of the per-group tensors (one range if not grouped)."""
        if not isinstance(self.vis, list):
            return [(0, self.n_chan)]
        out, c0 = [], 0
        for v in self.vis:
            out.append((c0, c0 + v.shape[1]))
            c0 += v.shape[1]
        return out


def support_schedule(s_min: int, s_max: int, k_planes: int) -> list:
    """Odd supports growing linearly over the w-planes: the smallest odd integer
    >= s_min + (s_max - s_min) * k / (K - 1)."""
    out = []
    for k in range(k_planes):
        t = s_min + (s_max - s_min) * (k / (k_planes - 1) if k_planes > 1 else 0.0)
        s = int(math.ceil(t - 1e-9))
        if s % 2 == 0:
            s += 1
        out.append(s)
    return out


def cell_and_wmax(uvw_m: np.ndarray, freq_hz: np.ndarray, n_grid: int, s_max: int):
    """Cell size so that every footprint fits the grid, and w_max = max |w| [wavelengths]."""
    lam_inv = freq_hz.max() / C0
    uvmax = float(np.abs(uvw_m[:, :2]).max()) * lam_inv
    du = 2.0 * uvmax / (n_grid - s_max - 2)
    w_max = float(np.abs(uvw_m[:, 2]).max()) * lam_inv
    return du, w_max


def _flags(rows, C, P, frac, seed, device):
    if frac <= 0:
        return torch.zeros((rows, C, P), dtype=torch.uint8, device=device)
    g = torch.Generator(device=device)
    g.manual_seed(seed + 7)
    f = (torch.rand((rows, C, P), generator=g, device=device) < frac).to(torch.uint8)
    # a few fully flagged records as well
    allf = (torch.rand((rows, C, 1), generator=g, device=device) < frac).to(torch.uint8)
    return torch.maximum(f, allf.expand(rows, C, P)).contiguous()


_SEEDS = {"w0_small": 1000, "wproj_2k": 1001, "degrid_1k": 1002, "batch_8k": 1004, "mfs_2k": 1005}


def _spec(name: str, rng: np.random.Generator):
    """Station layout (the first draws from rng) and the fixed parameters of a named workload."""
    if name == "w0_small":
        enu = stations_uniform_disk(32, 2000.0, rng)
        T, dt, dec = 256, 10.0, 45.0
        freq = np.array([150e6])
        P, N, K, beta, S_lo, S_hi, taper = 1, 512, 1, 8, 7, 7, 7
        noise = 0.01
    elif name == "wproj_2k":
        enu = stations_gaussian(64, 3000.0, rng)
        T, dt, dec = 3600, 1.0, 45.0
        freq = np.linspace(120e6, 180e6, 16)
        P, N, K, beta, S_lo, S_hi, taper = 4, 2048, 32, 8, 8, 64, 7
        noise = 0.01
    elif name == "mfs_2k":
        enu = stations_gaussian(64, 3000.0, rng)
        T, dt, dec = 3600, 1.0, 45.0
        freq = 150e6 + 195312.5 / 16 * np.arange(16)
        P, N, K, beta, S_lo, S_hi, taper = 4, 2048, 32, 8, 8, 64, 7
        noise = 0.01
    elif name == "degrid_1k":
        enu = stations_gaussian(64, 3000.0, rng)
        T, dt, dec = 600, 6.0, 45.0
        freq = np.linspace(120e6, 180e6, 4)
        P, N, K, beta, S_lo, S_hi, taper = 4, 1024, 16, 8, 8, 32, 7
        noise = 0.01
    elif name == "batch_8k":
        enu = stations_log_radial(256, 10000.0, rng)
        T, dt, dec = 1800, 2.0, 45.0
        freq = np.linspace(50e6, 350e6, 64)
        P, N, K, beta, S_lo, S_hi, taper = 1, 8192, 64, 8, 8, 128, 7
        noise = 0.01
    else:
        raise KeyError(name)
    return enu, T, dt, dec, freq, P, N, K, beta, S_lo, S_hi, taper, noise


def full_tracks(name: str):
    """The full workload's uvw tracks [baselines, times, 3] in metres and its channel
    frequencies [C] in Hz (the same seeded layout as make(name)); for choosing slices."""
    rng = np.random.default_rng(_SEEDS[name])
    enu, T, dt, dec, freq, *_ = _spec(name, rng)
    uvw = uvw_tracks(enu, T, dt, dec, baselines=baseline_pairs(enu.shape[0]))
    return uvw.reshape(-1, T, 3), np.asarray(freq, dtype=np.float64)


def outer_w_slice(name: str, n_times: int, n_top: int, n_spread: int, stride: int = 97):
    """A slice that reaches the workload's outermost w-planes: the n_times steps around the
    largest |w| of the track, the n_top baselines with the largest |w| in those steps, and
    n_spread further baselines taken every `stride` along the baseline list.  Returns
    (sorted baseline indices, first time step) for make(baselines=..., t_start=...)."""
    tracks, _ = full_tracks(name)
    B, T, _ = tracks.shape
    aw = np.abs(tracks[:, :, 2])
    t_star = int(np.argmax(aw.max(axis=0)))
    t0 = min(max(0, t_star - n_times // 2), T - n_times)
    w_win = aw[:, t0:t0 + n_times].max(axis=1)
    top = np.argsort(w_win)[::-1][:n_top]
    rest = np.setdiff1d(np.arange(0, B, stride), top)[:n_spread]
    return np.sort(np.concatenate([top, rest])), t0


def make(name: str, device: str = "cpu", flag_frac: float = 0.0, n_times: Optional[int] = None,
         n_chan: Optional[int] = None, n_baselines: Optional[int] = None,
         chan_group: Optional[int] = None, chan0: int = 0, baselines=None,
         t_start: Optional[int] = None) -> Workload:
    """Build one of the named workloads.

    name: "w0_small"   : plain w=0 gridding, 32 stations in a 2 km disk, 496 baselines x 256
                         steps at 10 s, dec +45, 150 MHz, 1 pol, N=512, S=7, beta=8, K=1.
          "wproj_2k"   : 64 stations in a 3 km Gaussian layout, 2016 baselines x 3600 steps at
                         1 s, 16 channels 120-180 MHz, 4 pols, N=2048, K=32 sqrt(w)-spaced
                         planes with supports 9..65, beta=8.
          "degrid_1k"  : 64 stations, 600 steps, 4 channels 120-180 MHz, 4 pols, N=1024, K=16.
          "batch_8k"   : 256 stations log-radial to 10 km, 1800 steps, 64 channels
                         50-350 MHz, 1 pol, N=8192, K=64, supports 9..129.
          "mfs_2k"     : the wproj_2k geometry with 16 narrow channels (12.2 kHz apart from
                         150 MHz, a LOFAR subband split 16 ways), for channel interleaving.
    n_times / n_chan / n_baselines shrink a workload to a seeded slice of the same geometry;
    chan0 is the first channel of an n_chan slice.  `baselines` (indices into the workload's
    baseline list, in the order given) replaces the first n_baselines; `t_start` is the first
    time step of an n_times slice (default: the block centred on transit).
    chan_group: vis, weight and flag become lists of [rows, chan_group, P] tensors, one per
    group of consecutive channels, each drawn with its own seed (seed + 7919 * group index);
    the (all-ones) weight tensor is shared by the groups."""
    seed = _SEEDS[name]
    rng = np.random.default_rng(seed)
    enu, T, dt, dec, freq, P, N, K, beta, S_lo, S_hi, taper, noise = _spec(name, rng)
    sky = point_sources(5, rng)
    pairs = baseline_pairs(enu.shape[0])
    supports = support_schedule(S_lo, S_hi, K)
    # geometry of the FULL workload fixes cell size and w_max, so slices share it
    uvw_full = uvw_tracks(enu, T, dt, dec, baselines=pairs)
    du, w_max = cell_and_wmax(uvw_full, freq, N, max(supports))
    b_idx = np.arange(len(pairs))
    if baselines is not None:
        b_idx = np.asarray(baselines, dtype=np.int64).reshape(-1)
        if b_idx.size and (b_idx.min() < 0 or b_idx.max() >= len(pairs)):
            raise ValueError("baseline index out of range")
        pairs = pairs[b_idx]
    elif n_baselines is not None:
        pairs = pairs[:n_baselines]
        b_idx = b_idx[:n_baselines]
    T_used = T if n_times is None else n_times
    if n_times is not None or n_baselines is not None or baselines is not None:
        # a contiguous block of time steps (centred on transit unless t_start is given) for the
        # chosen baselines
        t0 = (T - T_used) // 2 if t_start is None else int(t_start)
        if t0 < 0 or t0 + T_used > T:
            raise ValueError("time slice [%d, %d) outside the %d steps" % (t0, t0 + T_used, T))
        t_idx = np.arange(t0, t0 + T_used)
        uvw = uvw_full.reshape(-1, T, 3)[b_idx][:, t_idx]
        uvw = np.ascontiguousarray(uvw.reshape(-1, 3))
    else:
        uvw = uvw_full
    if n_chan is not None or chan0:
        freq = freq[chan0:None if n_chan is None else chan0 + n_chan]
    rows, C = uvw.shape[0], freq.shape[0]
    if chan_group is None:
        vis = visibilities(uvw, freq, sky, P, noise, seed, device=device)
        weight = torch.ones((rows, C, P), dtype=torch.float32, device=device)
        flag = _flags(rows, C, P, flag_frac, seed, device)
    else:
        if C % chan_group:
            raise ValueError("chan_group=%d must divide the %d channels" % (chan_group, C))
        ones = torch.ones((rows, chan_group, P), dtype=torch.float32, device=device)
        vis, weight, flag = [], [], []
        for gi, c0 in enumerate(range(0, C, chan_group)):
            sg = seed + 7919 * gi
            vis.append(visibilities(uvw, freq[c0:c0 + chan_group], sky, P, noise, sg, device=device))
            weight.append(ones)
            flag.append(_flags(rows, chan_group, P, flag_frac, sg, device))
    return Workload(name, uvw, freq.astype(np.float64), vis, weight, flag, N, du, K, w_max, beta,
                    supports, taper, len(pairs), T_used)


def to_half_vis(vis: torch.Tensor, headroom: float = 60000.0):
    """complex32 visibilities and per-channel float32 scales max|vis| / headroom, so that the
    scaled values stay inside the float16 range (storage format of the precision variant)."""
    C = vis.shape[1]
    amax = vis.abs().amax(dim=(0, 2)) if vis.numel() else torch.zeros(C, device=vis.device)
    scale = torch.where(amax > 0, amax / headroom, torch.ones_like(amax)).to(torch.float32)
    import warnings
    with warnings.catch_warnings():   # complex32 is a storage format here; no arithmetic on it
        warnings.simplefilter("ignore", UserWarning)
        return (vis / scale[None, :, None]).to(torch.complex32), scale
