"""Pins of the regulariser oracle (Eq. 11 derivative loss, Eq. 12 box loss)
against what does not come from the oracle itself: derivatives of an
independent symbolic B-spline basis (sympy), the closed form of a cubic
Bezier's third derivative, the exact error of the midpoint rule on a quartic,
hand-computed box penalties of a straight segment, translation invariance, and
central differences of the losses."""
import math

import numpy as np
import pytest
import sympy as sy
import torch

import scenes
from oracle import geometry as og
from oracle import nurbs as nb
from oracle import pipeline as op

DT = torch.float64


def _knots_open(tau, p):
    """Clamped knot vector written out from its definition (§3.1): p zero
    intervals, the stored intervals, p zero intervals, cumulative sum from 0."""
    iv = [0] * p + list(tau) + [0] * p
    out = [sy.Integer(0)]
    for v in iv:
        out.append(out[-1] + v)
    return out


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_basis_derivatives_sum_to_zero(p):
    """Partition of unity: sum_i N_{i,p} = 1, so every derivative of the sum is 0."""
    rng = np.random.default_rng(10 + p)
    for closed in (False, True):
        nk = p + 4
        tau = torch.tensor(rng.uniform(0.3, 1.7, nk if closed else nk - p), dtype=DT)
        U = nb.knot_vector(tau, p, closed)
        a, b = nb.domain(U, p)
        u = og.quadrature_nodes(a, b, 37)
        for k in range(1, 5):
            N = og.basis_derivatives(U, p, u, k)
            scale = max(1.0, float(N.abs().max()))
            assert float(N.sum(1).abs().max()) <= 1e-11 * scale


@pytest.mark.parametrize("p", [2, 3, 4])
def test_curve_derivatives_match_symbolic_bspline(p):
    """C^(r)(u), r = 0..4, of a rational open curve against sympy's own B-spline
    basis (bspline_basis_set) differentiated symbolically."""
    rng = np.random.default_rng(20 + p)
    nk = p + 3
    key = np.zeros((nk, 4))
    key[:, :2] = np.round(rng.uniform(0, 50, (nk, 2)) * 4) / 4
    key[:, 2] = 1.0
    key[:, 3] = np.round(rng.uniform(0.5, 2.0, nk) * 8) / 8
    tau = [sy.Rational(int(v), 8) for v in rng.integers(4, 14, nk - p)]
    U = _knots_open(tau, p)
    x = sy.Symbol("x")
    basis = sy.bspline_basis_set(p, U, x)
    # evaluation points strictly inside spans
    us = []
    for lo, hi in zip(U[p:-p - 1], U[p + 1:-p]):
        if hi > lo:
            us += [lo + (hi - lo) * sy.Rational(1, 3), lo + (hi - lo) * sy.Rational(4, 5)]
    Ut = torch.tensor([float(v) for v in U], dtype=DT)
    cp = torch.tensor(key, dtype=DT)
    ut = torch.tensor([float(v) for v in us], dtype=DT)
    C = og.curve_derivatives(cp, Ut, p, ut, 4)

    def piece(f, uv):
        """The polynomial piece of a piecewise basis function active at uv."""
        if isinstance(f, sy.Piecewise):
            for expr, cond in f.args:
                if bool(cond.subs(x, uv)):
                    return expr
            return sy.Integer(0)
        return f

    for j, uv in enumerate(us):
        bj = [piece(b, uv) for b in basis]
        W = sum(bj[i] * sy.nsimplify(key[i, 3]) for i in range(nk))
        fx = sum(bj[i] * sy.nsimplify(key[i, 3] * key[i, 0]) for i in range(nk)) / W
        fy = sum(bj[i] * sy.nsimplify(key[i, 3] * key[i, 1]) for i in range(nk)) / W
        for r in range(5):
            ex = float(sy.diff(fx, x, r).subs(x, uv))
            ey = float(sy.diff(fy, x, r).subs(x, uv))
            ref = np.array([ex, ey])
            got = C[r][j].numpy()
            assert np.abs(got - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max()), (r, j, got, ref)


def _bezier_scene(p, pts, T, w=None, size=64):
    nk = p + 1
    key = np.zeros((nk, 4))
    key[:, :2] = pts
    key[:, 2] = 2.0
    key[:, 3] = 1.0 if w is None else w
    return scenes.from_curves([dict(p=p, key=key, tau=[T])], size, size)


def test_cubic_bezier_third_derivative_closed_form():
    """One cubic Bezier span over [0, T] with unit weights: C'''(u) is the
    constant 6 (P3 - 3 P2 + 3 P1 - P0) / T^3, so Eq. 11 is its squared norm
    whatever the number of nodes."""
    pts = np.array([[3.0, 40.0], [20.0, 5.0], [41.0, 60.0], [60.0, 22.0]])
    T = 1.375
    sc = _bezier_scene(3, pts, T)
    k, t, c = op.leaves(sc, False)
    d3 = 6 * (pts[3] - 3 * pts[2] + 3 * pts[1] - pts[0]) / T ** 3
    for n in (1, 7, 192):
        got = float(og.deriv_loss(sc, k, t, 3, n))
        assert abs(got - float(d3 @ d3)) <= 1e-10 * float(d3 @ d3)
    # a quadratic polynomial has no third derivative
    sc2 = _bezier_scene(2, pts[:3], T)
    k2, t2, _ = op.leaves(sc2, False)
    assert abs(float(og.deriv_loss(sc2, k2, t2, 3, 50))) <= 1e-18


def test_midpoint_rule_exact_error_on_a_quartic():
    """Quartic Bezier (unit weights) over [0, T]: C'''(u) = 24 ((1-t) A + t B) / T^3
    with t = u/T, A, B the third differences of the control points, so
    |C'''|^2 = g(t) is quadratic.  Its mean over [0, 1] is
    576 (|A|^2 + A.B + |B|^2) / (3 T^6), and the n-node midpoint rule is off by
    exactly g''/(24 n^2) = 2 * 576 |B - A|^2 / T^6 / (24 n^2)."""
    P = np.array([[2.0, 9.0], [17.0, 50.0], [33.0, 4.0], [47.0, 61.0], [62.0, 30.0]])
    T = 0.75   # exact in float32, as the scene stores it
    sc = _bezier_scene(4, P, T)
    k, t, c = op.leaves(sc, False)
    A = P[3] - 3 * P[2] + 3 * P[1] - P[0]
    Bv = P[4] - 3 * P[3] + 3 * P[2] - P[1]
    exact = 576 * (A @ A + A @ Bv + Bv @ Bv) / (3 * T ** 6)
    g2 = 2 * 576 * ((Bv - A) @ (Bv - A)) / T ** 6
    for n in (1, 4, 25, 300):
        got = float(og.deriv_loss(sc, k, t, 3, n))
        assert abs(got - (exact - g2 / (24 * n * n))) <= 1e-10 * exact


def _segment_scene(x0, x1, y, box_size=64, delta_c=10.0):
    key = np.array([[x0, y, 2.0, 1.0], [x1, y, 2.0, 1.0]])
    return scenes.from_curves([dict(p=1, key=key, tau=[1.0])], box_size, box_size,
                              sample=dict(delta_c=delta_c))


def test_bbox_relu_and_softplus_on_a_segment():
    """A straight degree-1 stroke from (-10.25, 5) to (10, 5): length 20.25,
    M = ceil(10 * 20.25) = 203 samples x_j = x0 + j (x1 - x0)/(M - 1) (open
    curves include both ends, no endpoint copies in Eq. 12)."""
    sc = _segment_scene(-10.25, 10.0, 5.0)
    plans = op.plan(sc)
    assert plans[0].m_contour == 203
    k, t, c = op.leaves(sc, False)
    xs = [-10.25 + j * 20.25 / 202 for j in range(203)]
    relu = sum(max(0.0, -x) for x in xs)
    got = float(og.bbox_loss(sc, k, t, plans, (0.0, 0.0, 64.0, 64.0), og.RELU))
    assert abs(got - relu) <= 1e-9 * relu

    def sp(v):
        return math.log1p(math.exp(v))
    soft = sum(sp(-x) + sp(x - 64.0) + sp(-5.0) + sp(5.0 - 64.0) for x in xs)
    got = float(og.bbox_loss(sc, k, t, plans, (0.0, 0.0, 64.0, 64.0), og.SOFTPLUS))
    assert abs(got - soft) <= 1e-9 * soft


@pytest.mark.parametrize("kind", ["open", "closed", "fill"])
def test_bbox_translation_counts_the_sampled_points(kind):
    """With every sampled point beyond the right edge, the ReLU box loss is
    sum_j (x_j - x_max): moving all key points by d in x moves every curve point
    by d (the rational basis sums to 1), so sum_i dL/dx_i = number of points:
    M for a stroke (no endpoint copies), B boundary points for a fill."""
    if kind == "open":
        sc = scenes.small_open(31, n_curves=1, size=40)
    else:
        sc = scenes.small_closed(32, n_curves=1, size=48, filled=kind == "fill", h=2.0)
    plans = op.plan(sc)
    k, t, c = op.leaves(sc)
    L = og.bbox_loss(sc, k, t, plans, (-1000.0, -1000.0, 0.5, 1000.0), og.RELU)
    L.backward()
    pl = plans[0]
    npts = pl.n_boundary if kind == "fill" else pl.m_contour
    assert abs(float(k.grad[:, 0].sum()) - npts) <= 1e-9 * npts
    assert float(k.grad[:, 1].abs().max()) <= 1e-12


def _geo_value(sc, plans, key, tau, order, n, box, kind):
    k = torch.as_tensor(key, dtype=DT)
    t = torch.as_tensor(tau, dtype=DT)
    with torch.no_grad():
        return float(og.deriv_loss(sc, k, t, order, n) + og.bbox_loss(sc, k, t, plans, box, kind))


@pytest.mark.parametrize("kind", [og.RELU, og.SOFTPLUS])
@pytest.mark.parametrize("make", ["open", "closed", "fill"])
def test_geometry_grads_match_central_differences(make, kind):
    if make == "open":
        sc = scenes.small_open(33, n_curves=2, size=40, p=(2, 3, 5))
    else:
        sc = scenes.small_closed(34, n_curves=2, size=48, filled=make == "fill", h=2.0)
    plans = op.plan(sc)
    box = (10.0, 9.0, sc.width - 11.0, sc.height - 8.0)
    n = 96
    ref = og.geometry_loss_and_grads(sc, plans, order=3, nodes=n, box=box, kind=kind)
    rng = np.random.default_rng(35)
    key0 = sc.key.astype(np.float64)
    tau0 = sc.tau.astype(np.float64)
    picks = [("key", int(i), int(j)) for i, j in zip(rng.integers(0, key0.shape[0], 6), [0, 1, 3, 0, 1, 3])]
    picks += [("tau", int(i), 0) for i in rng.integers(0, tau0.shape[0], 3)]
    for which, i, j in picks:
        key, tau = key0.copy(), tau0.copy()
        arr = key if which == "key" else tau
        idx = (i, j) if which == "key" else (i,)
        h = 1e-6 * max(1.0, abs(arr[idx]))
        arr[idx] += h
        fp = _geo_value(sc, plans, key, tau, 3, n, box, kind)
        arr[idx] -= 2 * h
        fm = _geo_value(sc, plans, key, tau, 3, n, box, kind)
        fd = (fp - fm) / (2 * h)
        g = ref["dkey"][i, j] if which == "key" else ref["dtau"][i]
        scale = max(1.0, np.abs(ref["dkey"]).max(), np.abs(ref["dtau"]).max())
        assert abs(fd - g) <= 1e-5 * scale, (which, i, j, fd, g)
