"""Pins of the oracle's error measures (Section IV-C) against hand-evaluated cases, an
independent library implementation of Gaussian derivative filters, closed forms of the
filters on ramps and constants, and symmetries."""
import numpy as np
import pytest

from oracle import quality



def test_sad_mse_hand_evaluated():
    a = np.array([[0.0, 0.5], [1.0, 0.25]])
    Fg = np.zeros((2, 2, 3))
    Fe = np.zeros((2, 2, 3))
    Fe[0, 0] = [9, 9, 9]          # alpha 0: not counted
    Fe[0, 1] = [0.1, -0.2, 0.3]   # alpha 0.5
    Fe[1, 0] = [5, 5, 5]          # alpha 1: not counted
    Fe[1, 1] = [0.4, 0.0, -0.4]   # alpha 0.25
    r = quality.measures(Fe, Fg, a)
    assert r["pixels"] == 2
    assert r["sad"] == pytest.approx(0.5 * 0.6 + 0.25 * 0.8, abs=1e-15)
    assert r["mse"] == pytest.approx(0.5 * (0.01 + 0.04 + 0.09) + 0.25 * (0.16 + 0.16), abs=1e-15)


def test_gradient_matches_scipy_gaussian_derivative():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(5)
    F = rng.random((23, 31, 3))
    gx, gy = quality.gradient(F)
    for c in range(3):
        sx = ndimage.gaussian_filter(F[..., c], quality.SIGMA, order=(0, 1), mode="nearest",
                                     truncate=quality.TRUNCATE)
        sy = ndimage.gaussian_filter(F[..., c], quality.SIGMA, order=(1, 0), mode="nearest",
                                     truncate=quality.TRUNCATE)
        assert np.abs(gx[..., c] - sx).max() < 1e-12
        assert np.abs(gy[..., c] - sy).max() < 1e-12


def test_filter_taps():
    k, g, dg = quality.gaussian_kernels()
    assert len(k) == 13 and k[0] == -6                # radius floor(4 * 1.4 + 0.5) = 6
    assert g.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(g, g[::-1]) and np.allclose(dg, -dg[::-1])
    # the derivative of a unit ramp: sum k^2 g(k) / sigma^2, the discrete Gaussian's
    # variance over sigma^2, close to 1 (the taps cut at 6 sigma/1.4 lose about 1e-4)
    assert abs(np.sum(k * k * g) / quality.SIGMA ** 2 - 1.0) < 1e-3


def test_ramp_and_constant_gradients():
    h, w = 30, 40
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    slopes = np.array([0.5, -1.0, 2.0])
    F = x[..., None] * slopes + 0.3 * y[..., None]
    gx, gy = quality.gradient(F)
    inner = (slice(7, h - 7), slice(7, w - 7))
    _, g, _ = quality.gaussian_kernels()
    k = np.arange(-6, 7)
    unit = np.sum(k * k * g) / quality.SIGMA ** 2
    assert np.abs(gx[inner] - slopes * unit).max() < 1e-12
    assert np.abs(gy[inner] - 0.3 * unit).max() < 1e-12
    # a constant image has zero gradient everywhere, borders included
    cx, cy = quality.gradient(np.full((9, 11, 3), 0.7))
    assert np.abs(cx).max() < 1e-15 and np.abs(cy).max() < 1e-15


def test_grad_of_a_ramp_difference_and_symmetries():
    rng = np.random.default_rng(9)
    h, w = 40, 50
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    Fg = rng.random((h, w, 3))
    Fe = Fg + 0.01 * x[..., None]                     # the difference is a ramp in x
    a = np.zeros((h, w))
    a[10:30, 10:40] = rng.uniform(0.1, 0.9, (20, 30))  # fractional only away from borders
    r = quality.measures(Fe, Fg, a)
    k = np.arange(-6, 7)
    _, g, _ = quality.gaussian_kernels()
    unit = np.sum(k * k * g) / quality.SIGMA ** 2
    assert r["grad"] == pytest.approx(a.sum() * 3 * (0.01 * unit) ** 2, rel=1e-9)
    # swapping estimate and truth, and transposing everything, change nothing
    s = quality.measures(Fg, Fe, a)
    t = quality.measures(Fe.transpose(1, 0, 2), Fg.transpose(1, 0, 2), a.T)
    for key in ("sad", "mse", "grad"):
        assert s[key] == pytest.approx(r[key], rel=1e-12)
        assert t[key] == pytest.approx(r[key], rel=1e-12)


def test_only_fractional_alpha_counts():
    rng = np.random.default_rng(3)
    Fe, Fg = rng.random((12, 9, 3)), rng.random((12, 9, 3))
    a = (rng.random((12, 9)) > 0.5).astype(np.float64)   # 0 or 1 only
    r = quality.measures(Fe, Fg, a)
    assert r["sad"] == 0 and r["mse"] == 0 and r["grad"] == 0 and r["pixels"] == 0
