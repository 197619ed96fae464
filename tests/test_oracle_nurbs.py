"""Pins of the oracle's NURBS evaluation (§3.1, Eq. 1-3) against closed forms
and identities that do not reuse its code."""
import math

import numpy as np
import pytest
import torch

from oracle import nurbs as nb

DT = torch.float64


def _rand_tau(rng, n, zeros=0):
    t = rng.uniform(0.3, 1.5, n)
    if zeros:
        t[rng.choice(n, zeros, replace=False)] = 0.0
    return torch.tensor(t, dtype=DT)


def test_open_knot_vector_worked_example():
    # §3.1: p zero intervals prepended and appended, then a cumulative sum.
    # tau = [1,0,1,0,1,0,1], p = 2 -> [0,0,0,1,1,2,2,3,3,4,4,4] (by hand).
    U = nb.knot_vector(torch.tensor([1, 0, 1, 0, 1, 0, 1], dtype=DT), 2, False)
    assert U.tolist() == [0, 0, 0, 1, 1, 2, 2, 3, 3, 4, 4, 4]


def test_closed_knot_vector_worked_example():
    # §3.1: last p core intervals wrapped before, first p after, cumulative sum.
    # tau = [a, b, c], p = 2 -> intervals [b, c, a, b, c, a, b].
    U = nb.knot_vector(torch.tensor([1.0, 2.0, 4.0], dtype=DT), 2, True)
    assert U.tolist() == [0, 2, 6, 7, 9, 13, 14, 16]
    a, b = nb.domain(U, 2)
    assert float(b - a) == 7.0      # one period = sum of the core intervals


@pytest.mark.parametrize("closed", [False, True])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_partition_of_unity(p, closed):
    rng = np.random.default_rng(p + 10 * closed)
    nk = 9
    tau = _rand_tau(rng, nk if closed else nk - p, zeros=2)
    U = nb.knot_vector(tau, p, closed)
    a, b = nb.domain(U, p)
    u = torch.linspace(float(a), float(b), 257, dtype=DT)
    N = nb.basis(U, p, u)
    assert N.shape[1] == (nk + p if closed else nk)
    assert torch.all(N >= -1e-15)
    assert float((N.sum(1) - 1).abs().max()) < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_bezier_reduction(p):
    # Clamped knots with no interior knot: the NURBS is the rational Bezier
    # curve with Bernstein basis (closed form), for unit and random weights.
    rng = np.random.default_rng(p)
    key = torch.tensor(np.c_[rng.uniform(0, 50, (p + 1, 3)), rng.uniform(0.5, 2, p + 1)], dtype=DT)
    U = nb.knot_vector(torch.tensor([1.7], dtype=DT), p, False)
    u = torch.linspace(0, 1.7, 101, dtype=DT)
    for k in (torch.cat([key[:, :3], torch.ones(p + 1, 1, dtype=DT)], 1), key):
        C = nb.curve_point(k, U, p, u)
        ref = nb.bernstein_curve(k, u / 1.7)
        assert float((C - ref).abs().max()) < 1e-12


def _nine_point_circle(r):
    pts = []
    for q in range(4):
        a = q * math.pi / 2
        pts.append([r * math.cos(a), r * math.sin(a), 1.0, 1.0])
        pts.append([r * math.sqrt(2) * math.cos(a + math.pi / 4), r * math.sqrt(2) * math.sin(a + math.pi / 4),
                    1.0, math.sqrt(2) / 2])
    return pts


def test_open_quadratic_circle_is_exact():
    # Conics are exact NURBS: nine-point circle, weights (1, sqrt2/2, ...).
    pts = _nine_point_circle(7.0)
    pts.append(pts[0])
    U = nb.knot_vector(torch.tensor([1, 0, 1, 0, 1, 0, 1], dtype=DT), 2, False)
    u = torch.linspace(0, 4, 1001, dtype=DT)
    C = nb.curve_point(torch.tensor(pts, dtype=DT), U, 2, u)
    assert float((C[:, :2].norm(dim=1) - 7.0).abs().max()) < 1e-12


def test_closed_quadratic_circle_is_exact_and_periodic():
    key = torch.tensor(_nine_point_circle(5.0), dtype=DT)
    tau = torch.tensor([0, 1, 0, 1, 0, 1, 0, 1], dtype=DT) * 0.8
    cp = nb.control_net(key, 2, True)
    assert cp.shape[0] == 10
    U = nb.knot_vector(tau, 2, True)
    a, b = nb.domain(U, 2)
    u = torch.linspace(float(a), float(b), 777, dtype=DT)
    C = nb.curve_point(cp, U, 2, u)
    assert float((C[:, :2].norm(dim=1) - 5.0).abs().max()) < 1e-12
    assert float((C[0] - C[-1]).abs().max()) < 1e-12
    # quarter turn per pair of intervals: u = a + 0.8 lands on the next midpoint
    c1 = nb.curve_point(cp, U, 2, torch.tensor([float(a) + 0.8], dtype=DT))[0]
    assert abs(float(c1[0])) < 1e-12 and abs(float(c1[1]) - 5.0) < 1e-12


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_closed_curves_close(p):
    rng = np.random.default_rng(100 + p)
    nk = 8
    key = torch.tensor(np.c_[rng.uniform(0, 30, (nk, 3)), rng.uniform(0.5, 2, nk)], dtype=DT)
    cp = nb.control_net(key, p, True)
    assert cp.shape[0] == nk + p
    U = nb.knot_vector(_rand_tau(rng, nk), p, True)
    assert U.shape[0] == nk + 2 * p + 1
    a, b = nb.domain(U, p)
    C = nb.curve_point(cp, U, p, torch.stack([a, b]))
    assert float((C[0] - C[1]).abs().max()) < 1e-11
    # the derivative closes too (C^{p-1} continuity across the seam)
    d = nb.curve_derivative(cp, U, p, torch.stack([a + 1e-12, b - 1e-12]))
    assert float((d[0] - d[1]).abs().max()) < 1e-6 * float(d.abs().max())


def test_affine_invariance():
    rng = np.random.default_rng(3)
    key = torch.tensor(np.c_[rng.uniform(0, 30, (7, 3)), rng.uniform(0.5, 2, 7)], dtype=DT)
    U = nb.knot_vector(_rand_tau(rng, 4), 3, False)
    u = torch.linspace(0, float(U[-1]), 50, dtype=DT)
    A = torch.tensor([[1.3, -0.4], [0.2, 0.7]], dtype=DT)
    t = torch.tensor([3.0, -2.0], dtype=DT)
    k2 = key.clone()
    k2[:, :2] = key[:, :2] @ A.T + t
    C1 = nb.curve_point(key, U, 3, u)[:, :2] @ A.T + t
    C2 = nb.curve_point(k2, U, 3, u)[:, :2]
    assert float((C1 - C2).abs().max()) < 1e-11


@pytest.mark.parametrize("closed", [False, True])
def test_derivative_matches_difference_quotient(closed):
    # Eq. 2 against the definition of the derivative (central difference).
    rng = np.random.default_rng(11)
    p, nk = 3, 9
    key = torch.tensor(np.c_[rng.uniform(0, 30, (nk, 3)), rng.uniform(0.5, 2, nk)], dtype=DT)
    cp = nb.control_net(key, p, closed)
    U = nb.knot_vector(_rand_tau(rng, nk if closed else nk - p), p, closed)
    a, b = nb.domain(U, p)
    u = a + (b - a) * torch.tensor(rng.uniform(0.02, 0.98, 40), dtype=DT)
    h = 1e-6
    fd = (nb.curve_point(cp, U, p, u + h) - nb.curve_point(cp, U, p, u - h)) / (2 * h)
    d = nb.curve_derivative(cp, U, p, u)
    assert float((fd - d).abs().max()) < 1e-6 * float(d.abs().max())


def test_arc_length_segment_exact_and_circle_converges():
    # Degree 1 through two points: |C'| is constant, the rule is exact.
    key = torch.tensor([[1.0, 2.0, 1, 1], [4.0, 6.0, 1, 1]], dtype=DT)
    U = nb.knot_vector(torch.tensor([0.6], dtype=DT), 1, False)
    assert abs(float(nb.arc_length(key, U, 1, 7)) - 5.0) < 1e-13
    # Circle: midpoint rule error falls as N_L^-2 towards 2 pi r.
    cp = nb.control_net(torch.tensor(_nine_point_circle(3.0), dtype=DT), 2, True)
    Uc = nb.knot_vector(torch.tensor([0, 1, 0, 1, 0, 1, 0, 1], dtype=DT), 2, True)
    errs = [abs(float(nb.arc_length(cp, Uc, 2, n)) - 2 * math.pi * 3.0) for n in (64, 128, 256)]
    assert errs[2] < 1e-3
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_zero_last_interval_uses_nonempty_span():
    # tau may reach 0 (clamp [0, 2]); the right end must still evaluate.
    key = torch.tensor([[0, 0, 1, 1], [1, 2, 1, 1], [3, 2, 1, 1], [4, 0, 1, 1], [6, 1, 1, 1]], dtype=DT)
    U = nb.knot_vector(torch.tensor([1.0, 0.0], dtype=DT), 3, False)
    a, b = nb.domain(U, 3)
    C = nb.curve_point(key, U, 3, torch.stack([a, b, b - 1e-9]))
    assert torch.isfinite(C).all()
    assert float((C[0] - key[0, :3]).abs().max()) < 1e-14
    # the end point is the limit from inside the domain (left-continuous)
    assert float((C[1] - C[2]).abs().max()) < 1e-7
    # knot 1 has multiplicity p + 2: the last control point has empty support
    assert float((C[1] - key[3, :3]).abs().max()) < 1e-14
