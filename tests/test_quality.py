"""Pins of the image-quality measures (Table 2's MAE, RMSE and SSIM) against
closed forms and a direct evaluation of SSIM's definition on a single window."""
import math

import numpy as np

from paper_2208_12964_gb300 import quality, synth


def test_mae_rmse_closed_form():
    a = np.zeros((4, 4))
    b = np.zeros((4, 4))
    b[0, :2] = [3.0, -4.0]
    assert quality.mae(a, b) == 7.0 / 16
    assert abs(quality.rmse(a, b) - math.sqrt(25.0 / 16)) < 1e-15
    m = np.zeros((4, 4), bool)
    m[0, :2] = True
    assert quality.mae(a, b, m) == 3.5 and abs(quality.rmse(a, b, m) - math.sqrt(12.5)) < 1e-15


def test_ssim_identity_symmetry_and_constants():
    rng = np.random.default_rng(0)
    x = rng.random((40, 37))
    y = x + 0.1 * rng.standard_normal(x.shape)
    assert abs(quality.ssim(x, x) - 1.0) < 1e-12
    assert abs(quality.ssim(x, y, 1.0) - quality.ssim(y, x, 1.0)) < 1e-12
    assert quality.ssim(x, y) < quality.ssim(x, x + 0.01 * (y - x))
    # constant images: every local variance and covariance vanishes, leaving
    # the luminance term (2 c1 c2 + C1) / (c1^2 + c2^2 + C1)
    c1v, c2v, L = 0.3, 0.7, 1.0
    C1 = (0.01 * L) ** 2
    got = quality.ssim(np.full((20, 20), c1v), np.full((20, 20), c2v), L)
    assert abs(got - (2 * c1v * c2v + C1) / (c1v ** 2 + c2v ** 2 + C1)) < 1e-12


def test_ssim_single_window_matches_definition():
    """An 11 x 11 image has one window position: SSIM there is the formula of
    Wang et al. with Gaussian-weighted moments, evaluated here term by term."""
    rng = np.random.default_rng(1)
    x = rng.random((11, 11))
    y = 0.5 * x + 0.3 * rng.random((11, 11))
    t = np.arange(11) - 5.0
    g1 = np.exp(-t * t / (2 * 1.5 ** 2))
    w = np.outer(g1, g1)
    w /= w.sum()
    mx, my = (w * x).sum(), (w * y).sum()
    vx = (w * (x - mx) ** 2).sum()
    vy = (w * (y - my) ** 2).sum()
    cxy = (w * (x - mx) * (y - my)).sum()
    L = 2.0
    C1, C2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    ref = (2 * mx * my + C1) * (2 * cxy + C2) / ((mx * mx + my * my + C1) * (vx + vy + C2))
    assert abs(quality.ssim(x, y, L) - ref) < 1e-12


def test_phantom_image_of_a_centred_disk():
    spec = synth.parallel_workload(16, 4, 33)
    disk = [dict(kind="ellipse", dens=2.0, c=(0.0, 0.0, 0.0), axes=(0.5, 0.5, 1.0), rot=np.eye(3))]
    x, y, _ = quality.pixel_centres(spec, 64, 64)
    X, Y = np.meshgrid(x, y)
    v = synth.sample_phantom_on_points(disk, X, Y)
    inside = np.hypot(X, Y) <= 0.5
    assert np.all(v[inside] == 2.0) and np.all(v[~inside] == 0.0)
    assert abs(inside.sum() * (2.0 / 64) ** 2 - math.pi * 0.25) < 0.05
    img = quality.phantom_image(spec, 32, 32)
    assert img.shape == (1, 32, 32) and img.max() > 0 and np.all(img[0][~quality.disk_mask(spec, 32, 32)] == 0)
