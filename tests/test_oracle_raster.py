"""Pins of the oracle's compositing and binning (§3.4, Eq. 8-9)."""
import json
import math
import os

import numpy as np
import torch

import scenes
from oracle import raster as rs
from oracle import pipeline as pl

DT = torch.float64
R = dict(scenes.RASTER_DEFAULTS)


def _g(mu, sigma, o, curve=None, layer=None):
    G = len(sigma)
    return dict(mu=torch.tensor(mu, dtype=DT).reshape(G, 2), sigma=torch.tensor(sigma, dtype=DT),
                o=torch.tensor(o, dtype=DT),
                curve=torch.zeros(G, dtype=torch.long) if curve is None else torch.tensor(curve),
                sample=torch.arange(G), layer=torch.zeros(G, dtype=torch.long) if layer is None else torch.tensor(layer),
                scene=torch.zeros(G, dtype=torch.long))


def test_single_gaussian_closed_form():
    H = W = 20
    g = _g([[7.3, 11.6]], [2.2], [0.7])
    col = torch.tensor([[0.1, 0.5, 0.9, 1.0]], dtype=DT)
    r = dict(R, alpha_min=0.0, t_min=0.0, bg=(0.3, 0.2, 0.1))
    img = rs.render_brute(g, col, 1, H, W, 3, r)[0].numpy()
    yy, xx = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    a = 0.7 * np.exp(-((xx - 7.3) ** 2 + (yy - 11.6) ** 2) / (2 * 2.2 ** 2))
    ref = a[..., None] * np.array([0.1, 0.5, 0.9]) + (1 - a[..., None]) * np.array([0.3, 0.2, 0.1])
    assert np.abs(img - ref).max() < 1e-15


def test_same_colour_is_order_invariant():
    # One colour: I = c (1 - prod(1 - a)) + bg prod(1 - a), whatever the order.
    rng = np.random.default_rng(1)
    G = 30
    mu = rng.uniform(0, 16, (G, 2))
    sg = rng.uniform(0.8, 3, G)
    o = rng.uniform(0.2, 0.95, G)
    col = torch.tensor([[0.25, 0.5, 0.75, 1.0]], dtype=DT)
    r = dict(R, alpha_min=0.0, t_min=0.0, bg=(1.0, 1.0, 1.0))
    img1 = rs.render_brute(_g(mu, sg, o), col, 1, 16, 16, 3, r).numpy()
    perm = rng.permutation(G)
    img2 = rs.render_brute(_g(mu[perm], sg[perm], o[perm]), col, 1, 16, 16, 3, r).numpy()
    yy, xx = np.meshgrid(np.arange(16) + 0.5, np.arange(16) + 0.5, indexing="ij")
    a = np.minimum(0.99, o * np.exp(-((xx[..., None] - mu[:, 0]) ** 2 + (yy[..., None] - mu[:, 1]) ** 2)
                                   / (2 * sg ** 2)))
    T = np.prod(1 - a, axis=-1)
    ref = (1 - T)[..., None] * np.array([0.25, 0.5, 0.75]) + T[..., None]
    assert np.abs(img1[0] - ref).max() < 1e-13
    assert np.abs(img2[0] - ref).max() < 1e-13


def test_transparent_gives_background():
    g = _g([[5, 5], [9, 3]], [2, 3], [0.0, 0.0])
    col = torch.tensor([[0, 0, 0, 0.0]], dtype=DT)
    r = dict(R, bg=(0.2, 0.4, 0.6))
    img = rs.render_tiled(g, col, 1, 12, 12, 3, r).numpy()
    assert np.abs(img - np.array([0.2, 0.4, 0.6])).max() == 0.0


def test_sequential_equals_cumprod_with_thresholds():
    rng = np.random.default_rng(2)
    al = torch.tensor(rng.uniform(0, 0.99, (64, 50)) ** 2, dtype=DT)
    al[:, ::7] = 1e-3
    col = torch.tensor(rng.uniform(0, 1, (50, 3)), dtype=DT)
    for amin, tmin in [(1 / 255, 1e-4), (0.0, 1e-7), (0.05, 0.2)]:
        a1, T1, _ = rs.composite_sequential(al, col, (1, 1, 1), amin, tmin)
        a2, T2 = rs.composite_cumprod(al, col, (1, 1, 1), amin, tmin)
        assert float((a1 - a2).abs().max()) < 1e-14
        assert float((T1 - T2).abs().max()) < 1e-14
        assert bool((T1 >= tmin).all())


def test_termination_stops_before_crossing():
    al = torch.tensor([[0.9, 0.9, 0.9, 0.9, 0.9]], dtype=DT)
    col = torch.eye(5, 3, dtype=DT)
    out, T, n = rs.composite_sequential(al, col, (0, 0, 0), 0.0, 2e-3)
    # T: 1 -> 0.1 -> 0.01 -> (0.001 < 2e-3: stop before the third)
    assert abs(float(T[0]) - 0.01) < 1e-15 and int(n[0]) == 2


def test_bin_rect_covers_every_visible_pixel():
    # Production thresholds: k_sigma = 3.5 > sqrt(2 ln 255) so any pixel where
    # alpha >= alpha_min lies in a tile of the Gaussian's rectangle.
    rng = np.random.default_rng(3)
    G = 400
    H = W = 80
    mu = rng.uniform(-10, 90, (G, 2)).astype(np.float32)
    sg = rng.uniform(0.3, 6, G).astype(np.float32)
    o = rng.uniform(0, 1, G).astype(np.float32)
    T = 16
    tx = ty = 5
    xlo, xhi, ylo, yhi, valid = rs.tile_rects(mu, sg, o, T, 3.5, 1 / 255, tx, ty)
    yy, xx = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    for i in range(G):
        a = np.minimum(0.99, o[i] * np.exp(-((xx - mu[i, 0]) ** 2 + (yy - mu[i, 1]) ** 2) / (2.0 * sg[i] ** 2)))
        vis = a >= 1 / 255
        if not vis.any():
            continue
        assert valid[i]
        tys, txs = np.nonzero(vis)
        assert (txs // T).min() >= xlo[i] and (txs // T).max() <= xhi[i]
        assert (tys // T).min() >= ylo[i] and (tys // T).max() <= yhi[i]


def test_bin_rule_tile_boundaries():
    # Rectangles just right and just left of the tile edge at x = 16.
    mu = np.array([[np.float32(16.000002), 40.0]], np.float32)
    sg = np.array([np.float32(2.0 ** -21)], np.float32)
    xlo, xhi, *_ = rs.tile_rects(mu, sg, np.ones(1, np.float32), 16, 3.5, 0.0, 8, 8)
    assert xlo[0] == 1 and xhi[0] == 1
    mu2 = np.array([[np.float32(15.999999), 40.0]], np.float32)
    xlo, xhi, *_ = rs.tile_rects(mu2, sg, np.ones(1, np.float32), 16, 3.5, 0.0, 8, 8)
    assert xlo[0] == 0 and xhi[0] == 1


def test_sorted_pairs_order_and_ranges():
    sc = scenes.small_closed(5, n_curves=3, n_scenes=2, size=40)
    g = pl.gaussians_fp32(sc)
    import oracle.sampling as sm
    k, t, c = pl.leaves(sc, False)
    gg = sm.sample_scene(sc, k, t, c)
    tid, gid, ranges = rs.sorted_pairs(gg, sc.height, sc.width, 16, 6.0, 0.0, sc.n_scenes)
    assert np.all(np.diff(tid) >= 0)
    lay = gg["layer"].numpy()[gid]
    smp = gg["sample"].numpy()[gid]
    same = np.diff(tid) == 0
    key = lay * 10 ** 7 + smp
    assert np.all(np.diff(key)[same] > 0)       # strictly front to back, no repeats
    for tt in range(ranges.shape[0]):
        a, b = ranges[tt]
        assert np.all(tid[a:b] == tt)
    assert ranges[:, 1].max() == tid.shape[0]


def test_brute_equals_tiled():
    for sc in (scenes.small_open(4, n_curves=3, size=40), scenes.small_closed(6, n_curves=2, size=36)):
        k, t, c = pl.leaves(sc, False)
        plans = pl.plan(sc)
        with torch.no_grad():
            ib, _ = pl.render(sc, k, t, c, plans, mode="brute")
            it, _ = pl.render(sc, k, t, c, plans, mode="tiled")
        # parity thresholds: only alpha < exp(-18) lies outside the 6-sigma bins
        assert float((ib - it).abs().max()) < 1e-6
        sp = sc.with_raster(**{kk: v for kk, v in scenes.RASTER_DEFAULTS.items()})
        with torch.no_grad():
            ib, _ = pl.render(sp, k, t, c, plans, mode="brute")
            it, _ = pl.render(sp, k, t, c, plans, mode="tiled")
        assert float((ib - it).abs().max()) < 1e-12


def test_table_s1_defaults():
    here = os.path.dirname(__file__)
    gold = json.load(open(os.path.join(here, "golden", "table_s1_defaults.json")))
    for k in ("delta_c", "rho", "kappa", "nl_mult", "delta_b", "h", "eta", "gamma"):
        assert scenes.SAMPLE_DEFAULTS[k] == gold[k], k
