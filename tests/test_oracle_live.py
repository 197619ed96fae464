"""Pins of the layer-wise vectorisation oracle (distance-weighted loss,
self-crossing penalty, seeding) against hand-computed values and invariants."""
import math

import numpy as np
import torch

import scenes
from oracle import live as ol
from oracle import pipeline as op

DT = torch.float64


def _poly_scene(pts, closed):
    key = np.zeros((len(pts), 4))
    key[:, :2] = pts
    key[:, 2] = 2.0
    key[:, 3] = 1.0
    p = 1
    tau = [1.0] * (len(pts) if closed else len(pts) - p)
    return scenes.from_curves([dict(p=p, key=key, tau=tau, closed=closed, filled=False)], 16, 16)


def test_xing_convex_polygon_is_zero():
    sq = _poly_scene([(1, 1), (9, 1), (9, 9), (1, 9)], closed=True)
    k, _, _ = op.leaves(sq, False)
    assert float(ol.xing_loss(sq, k)) == 0.0


def test_xing_bow_tie_and_zig_zag():
    """Bow tie (0,0),(1,1),(1,0),(0,1): turn sines -1/sqrt2, -1/sqrt2, +1/sqrt2,
    +1/sqrt2, winding sum 0 so sigma = +1: penalty 2/sqrt2 = sqrt2.  Open zig-zag
    (0,0),(1,0),(1,1),(2,1): sines +1, -1, sigma = +1: penalty 1."""
    bt = _poly_scene([(0, 0), (1, 1), (1, 0), (0, 1)], closed=True)
    k, _, _ = op.leaves(bt, False)
    assert abs(float(ol.xing_loss(bt, k)) - math.sqrt(2.0)) <= 1e-14
    zz = _poly_scene([(0, 0), (1, 0), (1, 1), (2, 1)], closed=False)
    k, _, _ = op.leaves(zz, False)
    assert abs(float(ol.xing_loss(zz, k)) - 1.0) <= 1e-14


def test_xing_gradient_matches_central_differences():
    sc = scenes.small_closed(81, n_curves=3, size=48, filled=True, degrees=(3,))
    k, t, c = op.leaves(sc)
    # fold one key point across its neighbours so that some turns reverse
    with torch.no_grad():
        k0 = int(sc.key_offset[0])
        k[k0 + 1, :2] = 2 * k[k0 + 2, :2] - k[k0 + 1, :2]
    base = k.detach().clone()
    L = ol.xing_loss(sc, k)
    assert float(L.detach()) > 0
    L.backward()
    g = k.grad.numpy()
    for i in range(0, base.shape[0], 3):
        for j in (0, 1):
            h = 1e-6
            kp, km = base.clone(), base.clone()
            kp[i, j] += h
            km[i, j] -= h
            fd = (float(ol.xing_loss(sc, kp)) - float(ol.xing_loss(sc, km))) / (2 * h)
            assert abs(fd - g[i, j]) <= 1e-6 * max(1.0, abs(g).max())


def test_udf_loss_of_a_uniform_error_is_its_square():
    """With I - I* = delta everywhere the weighted mean is delta^2 whatever the
    weights; the gradient is 2 w delta / (C sum w S) and zero beyond tau."""
    sc = scenes.small_closed(82, n_curves=2, size=40, filled=True, h=2.0)
    plans = op.plan(sc)
    k, t, c = op.leaves(sc, False)
    tau = 6.0
    w = ol.udf_weights(sc, k, t, plans, [1], tau)
    img = torch.full((1, 40, 40, 3), 0.25, dtype=DT, requires_grad=True)
    tgt = torch.full((1, 40, 40, 3), 0.75, dtype=DT)
    L = ol.udf_mse(img, tgt, w, [True])
    assert abs(float(L) - 0.25) <= 1e-14
    L.backward()
    ref = 2 * w[0, :, :, None].expand(40, 40, 3) * (-0.5) / (3 * float(w.sum()))
    assert torch.allclose(img.grad[0], ref, rtol=0, atol=1e-15)
    assert float(w.max()) <= tau and float(w.min()) == 0.0


def test_udf_weights_of_an_exact_circle():
    """Boundary points of the exact rational circle lie on the circle and each
    chord stays within its sagitta R (1 - cos(gap/2)) inside it, so the
    distance from a pixel centre q to the polyline is | |q - c| - R | to within
    the largest sagitta."""
    b = scenes._Builder(1, 48, 48, 3)
    keys, tau = scenes.circle_keys(24.0, 24.0, 12.0), scenes.circle_tau()
    b.add(0, 2, keys, tau, (0.3, 0.3, 0.3, 1.0), True, True)
    sc = b.build("circle", np.ones((1, 48, 48, 3), np.float32), dict(scenes.SAMPLE_DEFAULTS, h=2.0),
                 dict(scenes.RASTER_PARITY))
    plans = op.plan(sc)
    k, t, c = op.leaves(sc, False)
    tau_w = 5.0
    w = ol.udf_weights(sc, k, t, plans, [0], tau_w)[0].numpy()
    poly = ol.boundary_polyline(sc, 0, k, t, plans[0]).numpy()
    assert np.abs(np.hypot(poly[:, 0] - 24.0, poly[:, 1] - 24.0) - 12.0).max() <= 1e-6   # float32 inputs
    gap = np.diff(np.unwrap(np.r_[np.arctan2(poly[:, 1] - 24.0, poly[:, 0] - 24.0),
                                  np.arctan2(poly[0, 1] - 24.0, poly[0, 0] - 24.0)])).max()
    sag = 12.0 * (1 - math.cos(gap / 2))
    yy, xx = np.mgrid[0:48, 0:48]
    r = np.hypot(xx + 0.5 - 24.0, yy + 0.5 - 24.0)
    dmin = np.abs(r - 12.0)
    assert np.all(w <= np.maximum(tau_w - dmin + sag, 0) + 1e-6)
    assert np.all(w >= np.maximum(tau_w - dmin - sag, 0) - 1e-6)


def test_seed_single_spike_and_two_blobs():
    """One nonzero error pixel at (x0, y0): every window within r of it holds
    the same sum, so the first in row-major order is (x0 - r, y0 - r).  Two
    blobs: the one with more mass wins, at its centre."""
    img = np.zeros((1, 20, 24, 3), np.float32)
    tgt = np.zeros_like(img)
    img[0, 9, 13, 1] = 2.0
    (x, y, v), = ol.seed_pixels(img, tgt, 3)
    assert (x, y) == (10, 6) and v == 4.0
    img = np.zeros((1, 30, 30, 1), np.float32)
    img[0, 4:7, 4:7, 0] = 1.0          # 9 px
    img[0, 19:24, 18:23, 0] = 1.0      # 25 px, centre (20, 21)
    (x, y, v), = ol.seed_pixels(img, np.zeros_like(img), 2)
    assert (x, y) == (20, 21) and v == 25.0
