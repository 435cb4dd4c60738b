"""Image-quality measures of a reconstruction against its phantom.

The paper judges its reconstructions by mean absolute error, root mean square
error and the structural similarity index against the original phantom
(Sec. IV, Table 2).  This module computes the same three measures for the
Cartesian image the library's resample produces (point sampling, Sec. II.B),
against the seeded phantom sampled at the same pixel centres.  It is host-side
measurement only: it holds none of the reconstruction method's arithmetic.

Readings (the paper gives no formulas for its measures):
  * MAE and RMSE are taken over the pixels whose centre lies inside the disk
    (2D) or the cylinder (3D), where the grid has cells; outside, both images
    are 0 by construction.
  * SSIM follows Wang, Bovik, Sheikh and Simoncelli (IEEE TIP 13(4), 2004):
    local means, variances and covariance under an 11 x 11 Gaussian window of
    standard deviation 1.5, constants C1 = (0.01 L)^2 and C2 = (0.03 L)^2 with
    L the phantom's value range, averaged over every window position that lies
    wholly inside the image; a 3D image is the mean over its slabs.
"""
from __future__ import annotations

import numpy as np

from . import synth

WIN = 11
SIGMA = 1.5
K1, K2 = 0.01, 0.03


def pixel_centres(spec: dict, nx: int, ny: int):
    """x [nx], y [ny] and z [slabs] of the pixel centres of the resampled image:
    the square [-R, R]^2 split into nx x ny pixels, one image per slab at the
    slab's mid-height."""
    R = spec["n_rings"] * spec["r"]
    x = -R + (np.arange(nx) + 0.5) * (2.0 * R / nx)
    y = -R + (np.arange(ny) + 0.5) * (2.0 * R / ny)
    if spec["geometry"] == synth.CONE_3D:
        z = spec["z_min"] + (np.arange(spec["n_slabs"]) + 0.5) * spec["h"]
    else:
        z = np.zeros(1)
    return x, y, z


def phantom_image(spec: dict, nx: int, ny: int) -> np.ndarray:
    """The workload's phantom at the pixel centres, [slabs][ny][nx], 0 where
    the centre lies outside the grid's disk."""
    bodies = synth.phantom_for(spec)
    x, y, z = pixel_centres(spec, nx, ny)
    R = spec["n_rings"] * spec["r"]
    X, Y = np.meshgrid(x, y)
    inside = np.hypot(X, Y) < R
    out = np.zeros((len(z), ny, nx))
    for s, zz in enumerate(z):
        v = synth.sample_phantom_on_points(bodies, X, Y, np.full_like(X, zz))
        out[s] = np.where(inside, v, 0.0)
    return out


def disk_mask(spec: dict, nx: int, ny: int) -> np.ndarray:
    x, y, _ = pixel_centres(spec, nx, ny)
    X, Y = np.meshgrid(x, y)
    return np.hypot(X, Y) < spec["n_rings"] * spec["r"]


def mae(a: np.ndarray, b: np.ndarray, mask: np.ndarray | None = None) -> float:
    d = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))
    return float(d[..., mask].mean() if mask is not None else d.mean())


def rmse(a: np.ndarray, b: np.ndarray, mask: np.ndarray | None = None) -> float:
    d = (np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2
    return float(np.sqrt(d[..., mask].mean() if mask is not None else d.mean()))


def gaussian_window(n: int = WIN, sigma: float = SIGMA) -> np.ndarray:
    """1D Gaussian weights of length n, centred, summing to 1."""
    t = np.arange(n) - (n - 1) / 2.0
    g = np.exp(-0.5 * (t / sigma) ** 2)
    return g / g.sum()


def _filter_valid(img: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Separable weighted window sums over every wholly-inside position."""
    n = len(g)
    v = np.lib.stride_tricks.sliding_window_view(img, n, axis=0) @ g
    return np.lib.stride_tricks.sliding_window_view(v, n, axis=1) @ g


def ssim2d(ref: np.ndarray, img: np.ndarray, data_range: float) -> float:
    """Mean SSIM of one 2D image against a reference (both at least 11 x 11)."""
    x = np.asarray(ref, np.float64)
    y = np.asarray(img, np.float64)
    g = gaussian_window()
    mx, my = _filter_valid(x, g), _filter_valid(y, g)
    sxx = _filter_valid(x * x, g) - mx * mx
    syy = _filter_valid(y * y, g) - my * my
    sxy = _filter_valid(x * y, g) - mx * my
    c1, c2 = (K1 * data_range) ** 2, (K2 * data_range) ** 2
    s = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
    return float(s.mean())


def ssim(ref: np.ndarray, img: np.ndarray, data_range: float | None = None) -> float:
    """SSIM of an image [ny][nx] or a stack [slabs][ny][nx] against the reference;
    data_range defaults to the reference's max - min."""
    ref = np.asarray(ref, np.float64)
    img = np.asarray(img, np.float64)
    if data_range is None:
        data_range = float(ref.max() - ref.min()) or 1.0
    if ref.ndim == 2:
        return ssim2d(ref, img, data_range)
    return float(np.mean([ssim2d(r, i, data_range) for r, i in zip(ref, img)]))


def report(spec: dict, image: np.ndarray) -> dict:
    """MAE, RMSE (inside the disk) and SSIM of a resampled image [slabs][ny][nx]
    against the workload's phantom."""
    image = np.asarray(image, np.float64)
    ns, ny, nx = image.shape
    ref = phantom_image(spec, nx, ny)
    m = disk_mask(spec, nx, ny)
    return {"mae": mae(ref, image, m), "rmse": rmse(ref, image, m), "ssim": ssim(ref, image),
            "phantom_range": float(ref.max() - ref.min()), "pixels": [ns, ny, nx]}
