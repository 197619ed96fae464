"""Pins of the tangent-aligned (anisotropic) contour variant of the oracle:
closed forms of the rotated Gaussian, a straight stroke worked by hand, the
k_sigma ellipse box of the bin rule, brute force = tiled, and central
differences of the loss through the tangent."""
import math

import numpy as np
import pytest
import torch

import scenes
from oracle import pipeline as op
from oracle import raster as rs

DT = torch.float64


def test_alpha_axis_aligned_and_rotated_closed_forms():
    rng = np.random.default_rng(201)
    px = torch.tensor(rng.uniform(-6, 6, 50), dtype=DT)
    py = torch.tensor(rng.uniform(-6, 6, 50), dtype=DT)
    mu = torch.tensor([[0.3, -0.2]], dtype=DT)
    o = torch.tensor([0.8], dtype=DT)
    sn = torch.tensor([1.1], dtype=DT)
    st = 2.7
    # tangent along +x: along = dx, across = dy
    a = rs.alpha(px, py, mu, sn, o, 1.0, torch.tensor([[st, 1.0, 0.0]], dtype=DT))[:, 0]
    dx, dy = px - 0.3, py + 0.2
    ref = 0.8 * torch.exp(-dx * dx / (2 * st * st) - dy * dy / (2 * 1.1 * 1.1))
    assert torch.allclose(a, ref, rtol=1e-15, atol=0)
    # tangent along +y: along = dy, across = -dx
    a = rs.alpha(px, py, mu, sn, o, 1.0, torch.tensor([[st, 0.0, 1.0]], dtype=DT))[:, 0]
    ref = 0.8 * torch.exp(-dy * dy / (2 * st * st) - dx * dx / (2 * 1.1 * 1.1))
    assert torch.allclose(a, ref, rtol=1e-15, atol=0)
    # equal deviations reproduce the isotropic Gaussian whatever the angle
    th = 0.7
    a = rs.alpha(px, py, mu, sn, o, 1.0, torch.tensor([[1.1, math.cos(th), math.sin(th)]], dtype=DT))[:, 0]
    assert torch.allclose(a, rs.alpha(px, py, mu, sn, o, 1.0)[:, 0], rtol=1e-14, atol=0)


def test_alpha_rotation_invariance():
    """Rotating the pixel offsets and the tangent by the same angle leaves alpha
    unchanged."""
    rng = np.random.default_rng(202)
    d = torch.tensor(rng.uniform(-5, 5, (40, 2)), dtype=DT)
    th, phi = 0.4, 1.9
    shp = torch.tensor([[3.0, math.cos(th), math.sin(th)]], dtype=DT)
    R = torch.tensor([[math.cos(phi), -math.sin(phi)], [math.sin(phi), math.cos(phi)]], dtype=DT)
    shp2 = torch.tensor([[3.0, math.cos(th + phi), math.sin(th + phi)]], dtype=DT)
    mu = torch.zeros(1, 2, dtype=DT)
    s, o = torch.tensor([0.9], dtype=DT), torch.tensor([1.0], dtype=DT)
    a1 = rs.alpha(d[:, 0], d[:, 1], mu, s, o, 1.0, shp)
    d2 = d @ R.T
    a2 = rs.alpha(d2[:, 0], d2[:, 1], mu, s, o, 1.0, shp2)
    assert torch.allclose(a1, a2, rtol=1e-13, atol=0)


def _segment(x0, y0, x1, y1, width=3.0, delta_c=0.5):
    key = np.array([[x0, y0, width, 1.0], [x1, y1, width, 1.0]])
    return scenes.from_curves([dict(p=1, key=key, tau=[1.0])], 48, 48,
                              sample=dict(delta_c=delta_c, contour_mode=1, kappa=2))


def test_straight_stroke_worked_example():
    """A degree-1 stroke from (5, 7) to (41, 22): length 39, M = ceil(0.5 * 39)
    = 20 samples; every Gaussian has the segment direction (36, 15)/39 as its
    tangent, sigma_t = 39 / ((M - 1) rho) and sigma_n = 3 / rho."""
    sc = _segment(5.0, 7.0, 41.0, 22.0)
    g = op.gaussians_fp32(sc)
    pl = g["plans"][0]
    assert pl.m_contour == 20
    sh = g["shape"]
    assert sh.shape == (20 + 2 * 2, 4)
    assert np.allclose(sh[:, 1], 36 / 39, rtol=0, atol=1e-7) and np.allclose(sh[:, 2], 15 / 39, rtol=0, atol=1e-7)
    assert np.allclose(sh[:, 0], 39 / (19 * 2.0), rtol=1e-6)
    assert np.allclose(g["rec"][:, 2], 1.5, rtol=1e-6)


def test_bins_hold_every_pixel_above_alpha_min():
    """The k_sigma = 3.5 ellipse box: every pixel with alpha >= 1/255 of a
    tangent-aligned Gaussian lies in its tile rectangle."""
    rng = np.random.default_rng(203)
    G = 300
    mu = rng.uniform(0, 64, (G, 2)).astype(np.float32)
    sn = rng.uniform(0.3, 2.0, G).astype(np.float32)
    th = rng.uniform(0, 2 * np.pi, G)
    shape = np.stack([rng.uniform(0.3, 6.0, G), np.cos(th), np.sin(th)], 1).astype(np.float32)
    o = rng.uniform(0.05, 1.0, G).astype(np.float32)
    T = 8
    xlo, xhi, ylo, yhi, valid = rs.tile_rects(mu, sn, o, T, 3.5, 1 / 255, 8, 8, shape)
    yy, xx = np.mgrid[0:64, 0:64]
    px = torch.tensor(xx.reshape(-1) + 0.5, dtype=DT)
    py = torch.tensor(yy.reshape(-1) + 0.5, dtype=DT)
    a = rs.alpha(px, py, torch.tensor(mu, dtype=DT), torch.tensor(sn, dtype=DT), torch.tensor(o, dtype=DT),
                 0.99, torch.tensor(shape, dtype=DT)).numpy()
    tx, ty = xx.reshape(-1) // T, yy.reshape(-1) // T
    for i in range(G):
        hit = a[:, i] >= 1 / 255
        if not hit.any():
            continue
        assert valid[i]
        assert np.all((tx[hit] >= xlo[i]) & (tx[hit] <= xhi[i]) & (ty[hit] >= ylo[i]) & (ty[hit] <= yhi[i]))


@pytest.mark.parametrize("thresholds", ["production", "parity"])
def test_brute_equals_tiled(thresholds):
    sc = scenes.small_open(204, n_curves=3, size=40, delta_c=0.6).with_sample(contour_mode=1)
    if thresholds == "production":
        sc = sc.with_raster(**scenes.RASTER_DEFAULTS)
    k, t, c = op.leaves(sc, False)
    with torch.no_grad():
        brute, _ = op.render(sc, k, t, c, mode="brute")
        tiled, _ = op.render(sc, k, t, c, mode="tiled")
    assert (brute - tiled).abs().max() <= (1e-12 if thresholds == "production" else 1e-6)


@pytest.mark.parametrize("make", ["open", "closed"])
def test_gradients_match_central_differences(make):
    if make == "open":
        sc = scenes.small_open(205, n_curves=2, size=40, p=(2, 3), delta_c=0.7)
    else:
        sc = scenes.small_closed(206, n_curves=2, size=44, filled=False, degrees=(2, 3), width=(1.5, 3.0))
        sc = sc.with_sample(delta_c=0.7)
    sc = sc.with_sample(contour_mode=1)
    ref = op.loss_and_grads(sc)
    plans = ref["plans"]
    rng = np.random.default_rng(207)
    key = sc.key.reshape(-1)
    for idx in rng.integers(0, key.shape[0], 6):
        fd = op.finite_difference(sc, "key", int(idx), plans)
        g = ref["dkey"].reshape(-1)[idx]
        assert abs(fd - g) <= 1e-5 * max(1e-3, np.abs(ref["dkey"]).max()), (idx, fd, g)
    for idx in rng.integers(0, sc.tau.shape[0], 3):
        fd = op.finite_difference(sc, "tau", int(idx), plans)
        assert abs(fd - ref["dtau"][idx]) <= 1e-5 * max(1e-3, np.abs(ref["dtau"]).max())
