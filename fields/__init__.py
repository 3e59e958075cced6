"""Seeded synthetic permeability fields and right-hand sides.

These generators feed both the CUDA path and the CPU oracle.  They hold none
of the method's arithmetic: they only draw random numbers and lay out
geometry.  Every array uses the cell order ``i + nx*(j + ny*k)`` (i fastest),
i.e. numpy shape ``(nz, ny, nx)``.

Fields (all isotropic, K = kappa * I, returned as float64 ``(nz, ny, nx)``):

* ``grf_lognormal``: log-permeability is a Gaussian random field with
  exponential covariance exp(-r/ell), synthesised with random Fourier modes
  (Shinozuka's spectral method: wave vectors drawn from the covariance's
  spectral density, which for the 3-D exponential kernel is a multivariate
  Student-t with one degree of freedom scaled by 1/ell).  Every cell value is
  computable independently, so the same seed gives the same field at any
  resolution.
* ``inclusions``: background 1 with random spheres and full-length
  axis-aligned square channels at a high value.
* ``layered_channels``: layered lognormal field with sinuous binary channels
  (the layer/channel geometry of the SPE10-like two-phase benchmark).

Right-hand sides: ``rhs_corners`` (+1 / -1 in opposite corner cells),
``rhs_line_sources`` (four corner line sources, one opposite centre line) and
``rhs_random`` (iid normal, mean removed).
"""
from __future__ import annotations

import math

import numpy as np
import torch

__all__ = [
    "grf_modes", "grf_values", "grf_lognormal", "grf_lognormal_device", "inclusions", "layered_channels",
    "rhs_corners", "rhs_line_sources", "rhs_random", "contrast_rescale",
]


def grf_modes(seed: int, corr_len: float = 0.1, n_modes: int = 1024):
    """Draw the random Fourier modes (wave vectors and phases) of a unit-variance
    GRF with covariance exp(-|x-y|/corr_len) in 3-D."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n_modes, 3))
    u = rng.chisquare(1.0, size=(n_modes, 1))
    k = g / np.sqrt(u) / corr_len
    phi = rng.uniform(0.0, 2.0 * math.pi, size=n_modes)
    return k, phi


def grf_values(shape, seed: int, corr_len: float = 0.1, n_modes: int = 1024,
               device: str = "cpu", chunk: int = 1 << 18) -> np.ndarray:
    """Unit-variance GRF sampled at cell centres of the unit cube grid ``shape``
    = (nz, ny, nx).  Evaluated with torch in float64 on ``device`` (chunked)."""
    nz, ny, nx = shape
    k, phi = grf_modes(seed, corr_len, n_modes)
    kt = torch.tensor(k, dtype=torch.float64, device=device)          # [M,3]
    pt = torch.tensor(phi, dtype=torch.float64, device=device)        # [M]
    n = nx * ny * nz
    out = torch.empty(n, dtype=torch.float64, device=device)
    scale = math.sqrt(2.0 / n_modes)
    for s in range(0, n, chunk):
        idx = torch.arange(s, min(n, s + chunk), device=device, dtype=torch.int64)
        i = idx % nx
        j = (idx // nx) % ny
        kk = idx // (nx * ny)
        x = torch.stack([(i + 0.5) / nx, (j + 0.5) / ny, (kk + 0.5) / nz], dim=1).to(torch.float64)
        out[s:s + idx.numel()] = scale * torch.cos(x @ kt.T + pt).sum(dim=1)
    return out.reshape(nz, ny, nx).cpu().numpy()


def grf_lognormal_device(shape, seed: int, contrast: float = 1e6, corr_len: float = 0.1, n_modes: int = 1024,
                         device: str = "cuda", dtype=torch.float32, chunk: int = 1 << 22) -> torch.Tensor:
    """The lognormal field of ``grf_lognormal`` (same modes for the same seed),
    evaluated and rescaled to ``max/min = contrast`` on ``device`` in ``dtype``
    and returned there: for grids too large to stage through the host.  In
    float32 the values differ from the float64 field by the rounding of the
    phases (a different, equally seeded realisation)."""
    nz, ny, nx = shape
    k, phi = grf_modes(seed, corr_len, n_modes)
    kt = torch.tensor(k, dtype=dtype, device=device)
    pt = torch.tensor(phi, dtype=dtype, device=device)
    n = nx * ny * nz
    out = torch.empty(n, dtype=dtype, device=device)
    scale = math.sqrt(2.0 / n_modes)
    for s in range(0, n, chunk):
        idx = torch.arange(s, min(n, s + chunk), device=device, dtype=torch.int64)
        i = idx % nx
        j = (idx // nx) % ny
        kk = idx // (nx * ny)
        x = torch.stack([(i + 0.5) / nx, (j + 0.5) / ny, (kk + 0.5) / nz], dim=1).to(dtype)
        out[s:s + idx.numel()] = scale * torch.cos(x @ kt.T + pt).sum(dim=1)
    lo, hi = out.min(), out.max()
    out.sub_(lo).div_(hi - lo).mul_(math.log(contrast)).exp_()
    return out.reshape(nz, ny, nx)


def contrast_rescale(y: np.ndarray, contrast: float) -> np.ndarray:
    """Affinely map y onto log-permeability so that kappa spans exactly
    [1, contrast]."""
    lo, hi = float(y.min()), float(y.max())
    t = (y - lo) / (hi - lo) if hi > lo else np.zeros_like(y)
    return np.exp(t * math.log(contrast))


def grf_lognormal(shape, seed: int, contrast: float | None = 1e3, sigma: float | None = None,
                  corr_len: float = 0.1, n_modes: int = 1024, device: str = "cpu") -> np.ndarray:
    """Lognormal permeability.  Either ``contrast`` (affine rescale of log-kappa
    so max/min equals it exactly) or ``sigma`` (kappa = exp(sigma * Y))."""
    y = grf_values(shape, seed, corr_len, n_modes, device)
    if sigma is not None:
        return np.exp(sigma * y)
    return contrast_rescale(y, contrast)


def inclusions(n: int, seed: int, n_spheres: int = 200, n_channels: int = 20,
               k_hi: float = 1e6, r_min_cells: float = 1.5, r_max_cells: float = 6.0) -> np.ndarray:
    """Background kappa = 1, ``n_spheres`` random-radius spheres and ``n_channels``
    2x2-cell square channels along a random axis across the whole domain at
    ``k_hi``, on an n^3 unit-cube grid."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    kappa = np.ones((n, n, n), dtype=np.float64)
    c = (np.arange(n) + 0.5) * h
    zc, yc, xc = np.meshgrid(c, c, c, indexing="ij")
    centres = rng.uniform(0.0, 1.0, size=(n_spheres, 3))
    radii = rng.uniform(r_min_cells * h, r_max_cells * h, size=n_spheres)
    for (cx, cy, cz), r in zip(centres, radii):
        lo = np.maximum(((np.array([cz, cy, cx]) - r) / h).astype(int) - 1, 0)
        hi = np.minimum(((np.array([cz, cy, cx]) + r) / h).astype(int) + 2, n)
        sl = tuple(slice(a, b) for a, b in zip(lo, hi))
        d2 = (xc[sl] - cx) ** 2 + (yc[sl] - cy) ** 2 + (zc[sl] - cz) ** 2
        kappa[sl][d2 <= r * r] = k_hi
    for _ in range(n_channels):
        axis = int(rng.integers(0, 3))
        a0, b0 = (int(v) for v in rng.integers(0, n - 1, size=2))
        if axis == 0:      # along x: fixed (z, y)
            kappa[a0:a0 + 2, b0:b0 + 2, :] = k_hi
        elif axis == 1:    # along y: fixed (z, x)
            kappa[a0:a0 + 2, :, b0:b0 + 2] = k_hi
        else:              # along z: fixed (y, x)
            kappa[:, a0:a0 + 2, b0:b0 + 2] = k_hi
    return kappa


def layered_channels(shape, seed: int, n_layers: int = 85, lattice=(60, 220),
                     channel_layers: int = 50, contrast_range=(1e6, 1e8)) -> np.ndarray:
    """Layered field: ``n_layers`` z-layers, each a 2-D lognormal field drawn on a
    ``lattice`` (x, y) grid and upsampled laterally; the lowest
    ``channel_layers`` layers carry sinuous binary channels.  Overall contrast
    is drawn from ``contrast_range``."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    lx, ly = lattice
    contrast = float(np.exp(rng.uniform(np.log(contrast_range[0]), np.log(contrast_range[1]))))
    layer_of_k = (np.arange(nz) * n_layers) // nz
    kappa = np.empty(shape, dtype=np.float64)
    xi = np.minimum((np.arange(nx) * lx) // nx, lx - 1)
    yi = np.minimum((np.arange(ny) * ly) // ny, ly - 1)
    # background log-permeability per layer (smoothed lattice noise)
    bg = []
    for _ in range(n_layers):
        z = rng.standard_normal((ly, lx))
        # separable 1-2-1 smoothing, a few passes
        for _ in range(3):
            z = (np.roll(z, 1, 0) + 2 * z + np.roll(z, -1, 0)) / 4
            z = (np.roll(z, 1, 1) + 2 * z + np.roll(z, -1, 1)) / 4
        z = (z - z.mean()) / (z.std() + 1e-30)
        bg.append(z[np.ix_(yi, xi)])
    log_bg_span = 0.5 * math.log(contrast)       # background spans half the decades
    for k in range(nz):
        kappa[k] = np.exp(np.clip(bg[layer_of_k[k]], -3, 3) / 6.0 * log_bg_span)
    # channels in the lowest layers
    k_ch = math.sqrt(contrast) * float(kappa.max())
    ygrid = (np.arange(ny) + 0.5) / ny
    xgrid = (np.arange(nx) + 0.5) / nx
    for layer in range(n_layers - channel_layers, n_layers):
        ks = np.nonzero(layer_of_k == layer)[0]
        if ks.size == 0:
            continue
        for _ in range(int(rng.integers(2, 5))):
            x0 = rng.uniform(0, 1)
            amp = rng.uniform(0.02, 0.15)
            lam = rng.uniform(0.2, 0.8)
            ph = rng.uniform(0, 2 * math.pi)
            width = rng.integers(3, 9) / nx
            xc_y = x0 + amp * np.sin(2 * math.pi * ygrid / lam + ph)
            mask = np.abs(xgrid[None, :] - xc_y[:, None]) <= width / 2
            for k in ks:
                kappa[k][mask] = k_ch
    kappa /= kappa.min()
    return kappa


def rhs_corners(shape) -> np.ndarray:
    """+1 in cell (0,0,0), -1 in the opposite corner cell (zero mean)."""
    f = np.zeros(shape, dtype=np.float64)
    f.flat[0] = 1.0
    f.flat[-1] = -1.0
    return f


def rhs_line_sources(shape) -> np.ndarray:
    """Four vertical line sources at the x-y corners and one opposite-sign line
    source at the x-y centre, zero mean (a five-spot well pattern)."""
    nz, ny, nx = shape
    f = np.zeros(shape, dtype=np.float64)
    for (j, i) in [(0, 0), (0, nx - 1), (ny - 1, 0), (ny - 1, nx - 1)]:
        f[:, j, i] += 1.0
    f[:, ny // 2, nx // 2] -= 4.0
    return f


def rhs_random(shape, n_rhs: int, seed: int) -> np.ndarray:
    """``n_rhs`` iid standard-normal right-hand sides with the mean removed;
    shape (n_rhs, nz, ny, nx)."""
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((n_rhs,) + tuple(shape))
    f -= f.reshape(n_rhs, -1).mean(axis=1).reshape((n_rhs, 1, 1, 1))
    return f


# ------------------------------------------------------------------ batched workload
LOGNORMAL_BATCH_GRIDS = (64, 64, 96, 96, 128, 128, 192, 192)


def lognormal_batch(n_rhs: int = 16, grids=LOGNORMAL_BATCH_GRIDS, device: str = "cpu"):
    """Inputs of the batched workload, one problem at a time: problem i is a
    grids[i]^3 unit-cube grid with kappa = exp(sigma_i Y), Y the exponential-
    covariance Gaussian field (correlation length 0.1, seed 10 + i) and
    sigma_i = 2 + 2 i / (len(grids) - 1), and ``n_rhs`` iid N(0, 1) zero-mean
    right-hand sides (seed 100 + i).  Yields (kappa, rhs) with rhs of shape
    (n_rhs, N, N, N)."""
    k = len(grids)
    for i, N in enumerate(grids):
        sigma = 2.0 + 2.0 * i / max(1, k - 1)
        kappa = grf_lognormal((N, N, N), seed=10 + i, contrast=None, sigma=sigma, device=device)
        yield kappa, rhs_random((N, N, N), n_rhs, seed=100 + i)
