"""Pins of the oracle's Gaussian sampling (§3.2 Eq. 4-5, §3.3 Eq. 6-7, Eq. S1-S3)."""
import math

import numpy as np
import torch

import scenes
from oracle import sampling as sm
from oracle import nurbs as nb

DT = torch.float64


def _one_curve_scene(key, tau, p, closed=False, filled=False, size=64, **sample):
    b = scenes._Builder(1, size, size, 3)
    b.add(0, p, key, tau, [0.2, 0.4, 0.6, 0.8], closed, filled)
    return b.build("t", np.ones((1, size, size, 3), np.float32),
                   dict(scenes.SAMPLE_DEFAULTS, **sample), dict(scenes.RASTER_PARITY))


def _leaves(sc):
    return (torch.tensor(sc.key, dtype=DT), torch.tensor(sc.tau, dtype=DT), torch.tensor(sc.color, dtype=DT))


def test_segment_worked_example():
    # Degree 1 through (10,20) -> (40,60): L = 50, M = ceil(0.3 * 50) = 15,
    # centres equally spaced on the segment, sigma = s / rho, kappa replicas.
    key = [[10, 20, 3.0, 1.0], [40, 60, 3.0, 1.0]]
    sc = _one_curve_scene(key, [2.5], 1, delta_c=0.3)
    k, t, c = _leaves(sc)
    pl = sm.plan_curve(sc, 0, k, t)
    assert abs(pl.length - 50.0) < 1e-9
    assert pl.m_contour == 15 and pl.count == 15 + 8
    mu, sig, o, _ = sm.curve_gaussians(sc, 0, k, t, c, pl)
    j = np.arange(15) / 14.0
    ref = np.c_[10 + 30 * j, 20 + 40 * j]
    assert np.abs(mu[4:19].numpy() - ref).max() < 1e-12
    assert np.abs(mu[:4].numpy() - ref[0]).max() < 1e-12       # first centre x kappa
    assert np.abs(mu[19:].numpy() - ref[-1]).max() < 1e-12     # last centre x kappa
    assert np.abs(sig.numpy() - 1.5).max() < 1e-12
    assert np.abs(o.numpy() - 0.8).max() < 1e-7


def test_closed_stroke_does_not_repeat_start():
    key = scenes.circle_keys(32, 32, 10)
    sc = _one_curve_scene(key, scenes.circle_tau(), 2, closed=True, delta_c=1.0)
    k, t, c = _leaves(sc)
    pl = sm.plan_curve(sc, 0, k, t)
    assert pl.kind == "closed"
    assert abs(pl.length - 2 * math.pi * 10) < 2e-3   # midpoint rule, N_L = 192
    assert pl.m_contour == math.ceil(pl.length)
    mu, _, _, _ = sm.curve_gaussians(sc, 0, k, t, c, pl)
    r = (mu - torch.tensor([32.0, 32.0], dtype=DT)).norm(dim=1)
    assert float((r - 10).abs().max()) < 1e-5     # key points are stored in float32
    d = (mu - torch.roll(mu, -1, 0)).norm(dim=1)
    assert float(d.min()) > 0.5         # no duplicated start point


def _even_odd_inside(q, poly):
    """Independent point-in-polygon test (ray casting) for the pin."""
    x, y = q
    inside = False
    n = len(poly)
    for i in range(n):
        x1, y1 = poly[i]
        x2, y2 = poly[(i + 1) % n]
        if (y1 > y) != (y2 > y):
            xi = x1 + (y - y1) * (x2 - x1) / (y2 - y1)
            if x < xi:
                inside = not inside
    return inside


def test_sdf_square_closed_form():
    poly = torch.tensor([[0, 0], [10, 0], [10, 10], [0, 10]], dtype=DT)   # positive area
    rng = np.random.default_rng(0)
    q = torch.tensor(rng.uniform(-5, 15, (400, 2)), dtype=DT)
    d, _ = sm.unsigned_distance(q, poly)
    x, y = q[:, 0].numpy(), q[:, 1].numpy()
    dx = np.maximum(np.maximum(-x, x - 10), 0)
    dy = np.maximum(np.maximum(-y, y - 10), 0)
    outside = np.hypot(dx, dy)
    inside = np.minimum(np.minimum(x, 10 - x), np.minimum(y, 10 - y))
    ins = (x > 0) & (x < 10) & (y > 0) & (y < 10)
    ref = np.where(ins, inside, outside)
    assert np.abs(d.numpy() - ref).max() < 1e-12
    wn = sm.winding_number(q, poly).numpy()
    assert np.abs(wn - np.round(wn)).max() < 1e-9
    for i in range(q.shape[0]):
        assert (wn[i] > 0.5) == _even_odd_inside(q[i].numpy(), poly.numpy())
    # clockwise traversal flips the winding number's sign
    wn_cw = sm.winding_number(q, torch.flip(poly, [0])).numpy()
    assert np.abs(wn + wn_cw).max() < 1e-9


def test_fill_opacity_of_a_circle():
    # Filled exact circle: o_j = o sigmoid(gamma/h (r - |q - c|)) up to the
    # polyline's sagitta r (1 - cos(pi/B)) in the distance.
    key = scenes.circle_keys(32, 32, 12)
    sc = _one_curve_scene(key, scenes.circle_tau(), 2, closed=True, filled=True, h=1.0)
    k, t, c = _leaves(sc)
    pl = sm.plan_curve(sc, 0, k, t)
    B = pl.n_boundary
    assert B == math.ceil(0.5 * pl.length)
    # padded box: extent 24 +- 10 %, i.e. [17.6, 46.4] -> 29 columns from 17.6
    assert abs(pl.x0 - 17.6) < 1e-6 and pl.nx == math.ceil(28.8)
    mu, sig, oj, (arg, sgn) = sm.curve_gaussians(sc, 0, k, t, c, pl)
    assert mu.shape[0] == pl.nx * pl.ny
    assert abs(float(mu[0, 0]) - (pl.x0 + 0.5)) < 1e-12
    assert float((sig - 0.75).abs().max()) < 1e-15
    rr = (mu - torch.tensor([32.0, 32.0], dtype=DT)).norm(dim=1)
    # boundary points are uniform in u, not in angle; the rational quadratic
    # parametrisation stretches angles by < 25 %, so every chord subtends less
    # than 1.25 * 2 pi / B and lies within that sagitta of the circle
    sag = 12 * (1 - math.cos(1.25 * math.pi / B))
    f = (oj / float(sc.color[0, 3])).numpy()      # o is stored in float32
    ok = (f > 1e-6) & (f < 1 - 1e-6)
    sdf = np.log(f[ok] / (1 - f[ok])) / 5.0
    assert np.abs(sdf - (12 - rr.numpy()[ok])).max() <= sag + 1e-9
    assert bool((sgn[rr < 11.0] > 0).all()) and bool((sgn[rr > 12.5] < 0).all())


def test_grid_clipped_to_canvas():
    key = scenes.circle_keys(2, 2, 10)     # mostly outside the canvas
    sc = _one_curve_scene(key, scenes.circle_tau(), 2, closed=True, filled=True, h=2.0, size=32)
    k, t, c = _leaves(sc)
    pl = sm.plan_curve(sc, 0, k, t)
    assert pl.x0 == 0.0 and pl.y0 == 0.0
    # boundary spans [-8, 12] (edge midpoints are boundary samples), pad 2,
    # clipped box [0, 14] -> 7 columns of step 2
    assert pl.nx == 7 and pl.ny == pl.nx


def test_grid_outside_canvas_is_empty():
    key = scenes.circle_keys(-40, 20, 10)
    sc = _one_curve_scene(key, scenes.circle_tau(), 2, closed=True, filled=True, size=32)
    k, t, c = _leaves(sc)
    pl = sm.plan_curve(sc, 0, k, t)
    assert pl.nx == 0 and pl.count == 0


def test_layers_painter_order():
    sc = scenes.small_closed(3, n_curves=3, n_scenes=2)
    k, t, c = _leaves(sc)
    g = sm.sample_scene(sc, k, t, c)
    for cv in range(sc.n_curves):
        s = sc.curve_scene()[cv]
        lay = g["layer"][g["curve"] == cv]
        assert bool((lay == sc.scene_curve_offset[s + 1] - 1 - cv).all())


def test_sign_margin_flags_a_grid_point_on_the_polyline():
    """The fill plan's "sign" margin is the smallest distance of a grid point
    from the boundary polyline (Eq. S1): it must equal a brute-force minimum
    over every grid point and segment, and it flags a scene whose grid point
    lies within rounding of the polyline (there the winding sign of Eq. S3,
    and with it the sign of the sdf gradient, is not decided by the data)."""
    from oracle import pipeline as op
    sc = scenes.small_closed(311, n_curves=3, size=48, filled=True, h=2.0)
    k, t, c = op.leaves(sc, False)
    with torch.no_grad():
        g = sm.sample_scene(sc, k, t, c)
    pl = g["plans"][0]
    p, fl, cp, U = sm.curve_inputs(sc, 0, k, t)
    a, b = nb.domain(U, p)
    poly = nb.curve_point(cp, U, p, sm.boundary_parameters(a, b, pl.n_boundary))[:, :2].detach().numpy()
    best = np.inf
    for iy in range(pl.ny):
        for ix in range(pl.nx):
            q = np.array([pl.x0 + (ix + 0.5) * 2.0, pl.y0 + (iy + 0.5) * 2.0])
            for i in range(poly.shape[0]):
                b0, b1 = poly[i], poly[(i + 1) % poly.shape[0]]
                e = b1 - b0
                tt = min(max(np.dot(q - b0, e) / np.dot(e, e), 0.0), 1.0)
                best = min(best, np.linalg.norm(q - b0 - tt * e))
    assert abs(pl.margin["sign"] - best) <= 1e-12
    assert pl.margin["sign"] < 1e-4
