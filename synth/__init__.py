"""Seeded synthetic interferometric workloads.

This module only makes inputs: antenna layouts, Earth-rotation uv tracks, a
sky model, its visibilities and their noise.  It holds none of the imaging
method's arithmetic (no gridding, no FFT imaging, no wavelets, no solver), so
that the FP64 oracle and the CUDA path can both be fed from it without sharing
any of the code they are compared on.

Conventions (shared as *data*, stated here once):

* Visibility rows are time-major: row = t * n_baselines + b, baselines are the
  antenna pairs i < j (no autocorrelations).
* u, v, w are in wavelengths.  ``pixel_size`` is in radians.
* Image pixel (p, q) (row p, column q) sits at l = (q - N/2) * pixel_size,
  m = (p - N/2) * pixel_size; the sky model is defined on that pixel grid.
* A visibility is V(u, v) = sum_pixels x[p, q] exp(-2 pi i (u l + v m)), the
  measurement equation of the paper (Sect. 2, Eq. RIME) with the direction
  dependent terms and w dropped, as the paper's reduced 2-D form allows.

The workloads mirror the paper's simulation (Sect. 4.1: 64 dishes, 4 h at
120 s, declination of the Galactic centre, noise from a complex Gaussian) at
the sizes of the five benchmark configurations; the MeerKAT mosaic and
antenna file the paper uses are not available, so layouts and skies are drawn
at random from the stated seed.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

C_LIGHT = 299_792_458.0


@dataclasses.dataclass
class Workload:
    """One synthetic observation (one or more channels)."""

    name: str
    npix: int
    pixel_size: float           # radians
    u: np.ndarray               # [nchan, nvis] float64, wavelengths
    v: np.ndarray               # [nchan, nvis] float64, wavelengths
    vis: np.ndarray             # [nchan, nvis] complex128 (noisy)
    flags: Optional[np.ndarray]  # [nchan, nvis] uint8 (1 = flagged) or None
    truth: np.ndarray           # [npix, npix] float64, pixel-sampled sky
    ell_px: float               # partition centre (pixel units of the N x N DFT grid)
    delta_px: float             # partition half width
    freqs: np.ndarray           # [nchan] Hz
    noise_sigma: np.ndarray     # [nchan] complex noise std (|n| rms)

    @property
    def nchan(self) -> int:
        return self.u.shape[0]

    @property
    def nvis(self) -> int:
        return self.u.shape[1]


# --------------------------------------------------------------------------
# array layouts
# --------------------------------------------------------------------------
def layout_uniform_disc(n_ant: int, radius_m: float, rng: np.random.Generator) -> np.ndarray:
    """East/north positions (metres), uniform in a disc."""
    r = radius_m * np.sqrt(rng.random(n_ant))
    th = 2 * np.pi * rng.random(n_ant)
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)


def layout_log_radial(n_ant: int, r_min: float, r_max: float,
                      rng: np.random.Generator) -> np.ndarray:
    """East/north positions with log-uniform radius (dense core, sparse arms)."""
    r = np.exp(rng.uniform(np.log(r_min), np.log(r_max), n_ant))
    th = 2 * np.pi * rng.random(n_ant)
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)


def baselines(enu: np.ndarray) -> np.ndarray:
    """Baseline vectors (east, north, up) for all pairs i < j."""
    n = enu.shape[0]
    i, j = np.triu_indices(n, k=1)
    d = enu[j] - enu[i]
    return np.concatenate([d, np.zeros((d.shape[0], 1))], axis=1)


def earth_rotation_uv(bl_enu: np.ndarray, hour_angles: np.ndarray, dec: float,
                      lat: float, freq: float):
    """uvw tracks (wavelengths) by the textbook ENU -> equatorial rotation.

    Rows are time-major.  Returns u, v, w of shape [n_times * n_bl].
    """
    e, n, up = bl_enu[:, 0], bl_enu[:, 1], bl_enu[:, 2]
    X = -math.sin(lat) * n + math.cos(lat) * up
    Y = e
    Z = math.cos(lat) * n + math.sin(lat) * up
    H = hour_angles[:, None]
    sd, cd = math.sin(dec), math.cos(dec)
    u = np.sin(H) * X + np.cos(H) * Y
    v = -sd * np.cos(H) * X + sd * np.sin(H) * Y + cd * Z
    w = cd * np.cos(H) * X - cd * np.sin(H) * Y + sd * Z
    lam = C_LIGHT / freq
    return (u / lam).ravel(), (v / lam).ravel(), (w / lam).ravel()


# --------------------------------------------------------------------------
# sky
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Sky:
    pts_pq: np.ndarray      # [np, 2] int pixel positions (row p, col q)
    pts_flux: np.ndarray    # [np]
    blob_pq: np.ndarray     # [nb, 2] float pixel centres
    blob_sigma: np.ndarray  # [nb] pixel std
    blob_peak: np.ndarray   # [nb]


def random_sky(npix: int, n_points: int, n_blobs: int, rng: np.random.Generator,
               margin: float = 0.25) -> Sky:
    """Point sources at integer pixels (log-uniform flux 0.01-1) plus
    Gaussian blobs (FWHM 2-6 px, log-uniform peak 0.01-1).  Sources are kept
    inside the central (1 - 2 margin) of the field."""
    lo, hi = int(npix * margin), int(npix * (1 - margin))
    pts = rng.integers(lo, hi, size=(n_points, 2))
    flux = np.exp(rng.uniform(np.log(0.01), np.log(1.0), n_points))
    bpq = rng.uniform(lo, hi, size=(n_blobs, 2)).round()
    fwhm = rng.uniform(2.0, 6.0, n_blobs)
    sig = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    peak = np.exp(rng.uniform(np.log(0.01), np.log(1.0), n_blobs))
    return Sky(pts, flux, bpq, sig, peak)


def sky_image(sky: Sky, npix: int) -> np.ndarray:
    """Pixel-sampled truth image."""
    img = np.zeros((npix, npix))
    np.add.at(img, (sky.pts_pq[:, 0], sky.pts_pq[:, 1]), sky.pts_flux)
    p = np.arange(npix)[:, None]
    q = np.arange(npix)[None, :]
    for (bp, bq), s, a in zip(sky.blob_pq, sky.blob_sigma, sky.blob_peak):
        img += a * np.exp(-((p - bp) ** 2 + (q - bq) ** 2) / (2 * s * s))
    return img


def sky_visibilities(sky: Sky, u: np.ndarray, v: np.ndarray, npix: int,
                     pixel_size: float, device: str = "cpu",
                     chunk: int = 1 << 22) -> np.ndarray:
    """Exact visibilities of the sky: a phase term per point source plus the
    analytic Fourier transform of each (pixel-unit) Gaussian blob.

    The heavy sum runs in float64 through torch on ``device`` (CPU threads or a
    GPU), chunked over rows.  This is simulation of the instrument, not part of
    the imaging method.
    """
    import torch

    dev = torch.device(device)
    l_pts = (sky.pts_pq[:, 1] - npix // 2) * pixel_size
    m_pts = (sky.pts_pq[:, 0] - npix // 2) * pixel_size
    l_b = (sky.blob_pq[:, 1] - npix // 2) * pixel_size
    m_b = (sky.blob_pq[:, 0] - npix // 2) * pixel_size
    lt = torch.tensor(np.concatenate([l_pts, l_b]), dtype=torch.float64, device=dev)
    mt = torch.tensor(np.concatenate([m_pts, m_b]), dtype=torch.float64, device=dev)
    amp_p = torch.tensor(sky.pts_flux, dtype=torch.float64, device=dev)
    sig_b = torch.tensor(sky.blob_sigma * pixel_size, dtype=torch.float64, device=dev)
    # integral of a Gaussian with pixel-unit peak a: a * 2 pi s_px^2
    amp_b = torch.tensor(sky.blob_peak * 2 * np.pi * sky.blob_sigma ** 2,
                         dtype=torch.float64, device=dev)
    npts = len(l_pts)
    out = np.empty(u.shape[0], dtype=np.complex128)
    two_pi = 2 * np.pi
    for s in range(0, u.shape[0], chunk):
        uu = torch.tensor(u[s:s + chunk], dtype=torch.float64, device=dev)
        vv = torch.tensor(v[s:s + chunk], dtype=torch.float64, device=dev)
        re = torch.zeros_like(uu)
        im = torch.zeros_like(uu)
        # sources in small groups to bound the temporary size
        for g in range(0, lt.shape[0], 16):
            ph = -two_pi * (uu[:, None] * lt[None, g:g + 16] + vv[:, None] * mt[None, g:g + 16])
            a = torch.empty(ph.shape[1], dtype=torch.float64, device=dev)
            idx = torch.arange(g, g + ph.shape[1], device=dev)
            isp = idx < npts
            a[isp] = amp_p[idx[isp]]
            a = a[None, :].expand(uu.shape[0], -1).clone()
            nb = (~isp).sum().item()
            if nb:
                bi = idx[~isp] - npts
                q2 = (uu * uu + vv * vv)[:, None]
                env = amp_b[bi][None, :] * torch.exp(-2 * np.pi ** 2 * sig_b[bi][None, :] ** 2 * q2)
                a[:, ~isp] = env
            re += (a * torch.cos(ph)).sum(1)
            im += (a * torch.sin(ph)).sum(1)
        out[s:s + chunk] = re.cpu().numpy() + 1j * im.cpu().numpy()
    return out


def add_noise(vis: np.ndarray, snr: float, rng: np.random.Generator):
    """Complex Gaussian noise with |n| rms = rms(|v|) / snr."""
    sigma = math.sqrt(np.mean(np.abs(vis) ** 2)) / snr
    n = (rng.standard_normal(vis.shape) + 1j * rng.standard_normal(vis.shape)) * (sigma / math.sqrt(2))
    return vis + n, sigma


# --------------------------------------------------------------------------
# the five benchmark workloads
# --------------------------------------------------------------------------
DEC = math.radians(-30.0)
LAT = math.radians(-30.7)


def _single_channel(name, n_ant, layout, n_dumps, span_h, npix, n_points, n_blobs,
                    split_frac, delta_px, freq, seed, device, snr=30.0,
                    max_rows=None):
    rng = np.random.default_rng(seed)
    enu = layout(rng)
    bl = baselines(enu)
    # dump centres over the span, hour angle in radians
    ha = (np.arange(n_dumps) + 0.5) / n_dumps * span_h - span_h / 2
    u, v, _ = earth_rotation_uv(bl, ha * (2 * np.pi / 24.0), DEC, LAT, freq)
    if max_rows is not None:
        u, v = u[:max_rows], v[:max_rows]
    uvmax = float(np.max(np.hypot(u, v)))
    pixel_size = 1.0 / (3.0 * uvmax)      # r_max = N/3 pixels
    sky = random_sky(npix, n_points, n_blobs, rng)
    truth = sky_image(sky, npix)
    vis = sky_visibilities(sky, u, v, npix, pixel_size, device=device)
    vis, sig = add_noise(vis, snr, rng)
    r_max = npix / 3.0
    return Workload(name=name, npix=npix, pixel_size=pixel_size,
                    u=u[None, :], v=v[None, :], vis=vis[None, :], flags=None,
                    truth=truth, ell_px=split_frac * r_max, delta_px=delta_px,
                    freqs=np.array([freq]), noise_sigma=np.array([sig]))


def small_fp64(seed: int = 0, device: str = "cpu") -> Workload:
    """128 x 128, 32 antennas in a 2 km disc, 64 dumps over 4 h, 31,744 rows,
    20 points + 3 blobs, split at 25 % of max |uv|."""
    return _single_channel(
        "small-128px-31744vis", 32, lambda r: layout_uniform_disc(32, 1000.0, r),
        64, 4.0, 128, 20, 3, 0.25, 3.0, 1.28e9, seed, device)


def ska_mid_like(seed: int = 0, device: str = "cpu", max_rows=None) -> Workload:
    """1024 x 1024, 197 dishes log-radial 50 m .. 150 km, 480 dumps over 8 h,
    9,266,880 rows, 200 points + 20 blobs, split at 10 % of max |uv|."""
    return _single_channel(
        "ska-mid-like-1024px-9266880vis", 197,
        lambda r: layout_log_radial(197, 50.0, 150e3, r),
        480, 8.0, 1024, 200, 20, 0.10, 3.0, 1.28e9, seed, device, max_rows=max_rows)


def ska_low_like(seed: int = 0, nchan: int = 4, n_dumps: int = 240, span_h: float = 4.0,
                 f_lo: float = 50e6, f_hi: float = 350e6) -> Workload:
    """4096 x 4096, 512 stations log-radial 35 m .. 65 km, 240 dumps over 4 h,
    4 channels over 50-350 MHz: 125,583,360 rows.  uv scale with frequency,
    the pixel size is fixed by the top channel.  The visibilities are seeded
    complex Gaussian values, not a sky: this workload serves operator timing
    and precision comparisons, where only the geometry matters and every form
    sees the same values."""
    rng = np.random.default_rng(seed)
    enu = layout_log_radial(512, 35.0, 65e3, rng)
    bl = baselines(enu)
    ha = (np.arange(n_dumps) + 0.5) / n_dumps * span_h - span_h / 2
    u0, v0, _ = earth_rotation_uv(bl, ha * (2 * np.pi / 24.0), DEC, LAT, 1.0)
    freqs = np.linspace(f_lo, f_hi, nchan)
    uvmax = float(np.max(np.hypot(u0, v0))) * f_hi
    pixel_size = 1.0 / (3.0 * uvmax)
    u = np.stack([u0 * f for f in freqs])
    v = np.stack([v0 * f for f in freqs])
    buf = np.empty(u.shape + (2,))
    rng.standard_normal(out=buf)
    buf *= 1.0 / math.sqrt(2.0)
    vis = buf.view(np.complex128)[..., 0]
    npix = 4096
    return Workload(name=f"ska-low-like-{npix}px-{u.size}vis", npix=npix,
                    pixel_size=pixel_size, u=u, v=v, vis=vis, flags=None,
                    truth=np.zeros((1, 1)), ell_px=0.10 * npix / 3.0, delta_px=3.0,
                    freqs=freqs, noise_sigma=np.ones(nchan))


def c1_style(npix: int, seed: int, device: str = "cpu") -> Workload:
    """The small workload's recipe at another image size (the learned warm
    start's training and evaluation skies): 32 antennas in a 2 km disc, 64
    dumps over 4 h (31,744 rows), split at 25 % of max |uv|, with the point
    and blob counts scaled with the image area (20 + 3 at 128 pixels)."""
    area = (npix / 128.0) ** 2
    return _single_channel(
        f"c1-style-{npix}px-seed{seed}", 32, lambda r: layout_uniform_disc(32, 1000.0, r),
        64, 4.0, npix, max(1, int(round(20 * area))), max(1, int(round(3 * area))),
        0.25, 3.0, 1.28e9, seed, device)


def paper_like(npix: int, seed: int = 0, split_frac: float = 0.205, delta_px: float = 3.0,
               device: str = "cpu") -> Workload:
    """The paper's simulation setting in kind (Sect. 4.1: 64 dishes, 4 h at
    120 s, one channel; 2016 baselines x 120 dumps = 241,920 rows), with a
    MeerKAT-like log-radial layout (29 m .. 8 km) in place of the array file
    the paper uses, and a random sky of points and blobs scaled with the
    image area (50 + 6 at 512 pixels).  The paper's partition centres 20, 35,
    55 px of its 512-pixel images are 0.117, 0.205, 0.322 of the longest
    baseline's radius (N/3 pixels here)."""
    area = (npix / 512.0) ** 2
    return _single_channel(
        f"paper-like-{npix}px-seed{seed}", 64, lambda r: layout_log_radial(64, 29.0, 8000.0, r),
        120, 4.0, npix, max(1, int(round(50 * area))), max(1, int(round(6 * area))),
        split_frac, delta_px, 1.28e9, seed, device)


def tiny(npix: int = 32, n_ant: int = 8, n_dumps: int = 6, seed: int = 1,
         device: str = "cpu", split_frac: float = 0.3, delta_px: float = 1.5,
         n_points: int = 4, n_blobs: int = 1) -> Workload:
    """Small cases for pins and parity tests (seconds on the oracle)."""
    return _single_channel(
        f"tiny-{npix}px", n_ant, lambda r: layout_uniform_disc(n_ant, 1000.0, r),
        n_dumps, 4.0, npix, n_points, n_blobs, split_frac, delta_px, 1.28e9, seed, device)


def multi_channel(npix: int = 1024, nchan: int = 64, f_lo: float = 350e6,
                  f_hi: float = 1050e6, seed: int = 0, device: str = "cpu",
                  n_ant: int = 197, n_dumps: int = 480, span_h: float = 8.0,
                  flag_max: float = 0.5, with_vis: bool = False) -> Workload:
    """Many channels of one layout: uv scale with frequency, pixel size fixed by
    the top channel, per-channel random flag fraction U(0, flag_max)."""
    rng = np.random.default_rng(seed)
    enu = layout_log_radial(n_ant, 50.0, 150e3, rng)
    bl = baselines(enu)
    ha = (np.arange(n_dumps) + 0.5) / n_dumps * span_h - span_h / 2
    freqs = np.linspace(f_lo, f_hi, nchan)
    u0, v0, _ = earth_rotation_uv(bl, ha * (2 * np.pi / 24.0), DEC, LAT, 1.0)
    uvmax = float(np.max(np.hypot(u0, v0))) * f_hi
    pixel_size = 1.0 / (3.0 * uvmax)
    u = np.stack([u0 * f for f in freqs])
    v = np.stack([v0 * f for f in freqs])
    frac = rng.uniform(0.0, flag_max, nchan)
    flags = (rng.random(u.shape) < frac[:, None]).astype(np.uint8)
    sky = random_sky(npix, 200, 20, rng)
    truth = sky_image(sky, npix)
    vis = np.zeros(u.shape, np.complex128)
    sig = np.zeros(nchan)
    if with_vis:
        for c in range(nchan):
            vc = sky_visibilities(sky, u[c], v[c], npix, pixel_size, device=device)
            vis[c], sig[c] = add_noise(vc, 30.0, rng)
    return Workload(name=f"multichannel-{nchan}x{npix}px", npix=npix,
                    pixel_size=pixel_size, u=u, v=v, vis=vis, flags=flags,
                    truth=truth, ell_px=0.10 * npix / 3.0, delta_px=3.0,
                    freqs=freqs, noise_sigma=sig)


def random_uv(n: int, npix: int, pixel_size: float, rng: np.random.Generator,
              frac_of_grid: float = 0.45) -> tuple:
    """Uniformly random (u, v) with |g| up to frac_of_grid of the oversampled
    grid half-width; used by the edge-case tests (points near the grid edge)."""
    uvmax = frac_of_grid / pixel_size
    u = rng.uniform(-uvmax, uvmax, n)
    v = rng.uniform(-uvmax, uvmax, n)
    return u, v
