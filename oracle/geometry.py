"""FP64 oracle, part 6: the geometric regularisers of the total loss (Eq. 10):
the derivative loss (Eq. 11) and the bounding-box loss (Eq. 12).

Test infrastructure only: the tests, the smoke check and the bench's CPU
baseline use this module.  Gradients come from `torch.autograd` through these
definitions, with the knot span of every quadrature node and the number of
sample points held fixed (as in the rest of the oracle).

Readings (the paper leaves these open):
  - Eq. 11's integral over [u_min, u_max] = [u_p, u_{m-p}] is taken with the
    same N-node midpoint rule as the arc length (Eq. 3): u_j = a + (j - 1/2)(b - a)/N,
    so (1/(b - a)) * integral ~= (1/N) sum_j |C^(r)(u_j)|^2.  The norm is over
    the planar (x, y) part of the curve, as for the arc length; the width
    coordinate is not smoothed.
  - "Averages over all curves": the mean over every curve of the batch.
  - The r-th derivative comes from differentiating the quotient C = S/W of
    Eq. 1 r times (Eq. 2 is the case r = 1):
        S^(k) = sum_{i=0..k} binom(k, i) W^(i) C^(k-i),
    solved for C^(k).  The basis derivatives follow from differentiating the
    Cox-de Boor recursion (Piegl & Tiller, The NURBS Book, Eq. 2.9):
        N^(k)_{i,d} = d (N^(k-1)_{i,d-1} / (u_{i+d} - u_i)
                         - N^(k-1)_{i+1,d-1} / (u_{i+d+1} - u_{i+1})),  0/0 := 0.
  - Eq. 12's "sampled curve positions" are the curve points the sampler
    evaluates: the M contour samples of a stroke (without the kappa endpoint
    copies) and the boundary polyline points of a filled curve.  The penalty
    is applied per axis, summed over x and y; ReLU has derivative 0 at 0;
    softplus is log(1 + e^x) in pixel units.
"""
from __future__ import annotations

import math

import torch

from . import nurbs as nb
from . import sampling as sm

DT = torch.float64
RELU, SOFTPLUS = 0, 1


def basis_derivatives(U: torch.Tensor, p: int, u: torch.Tensor, k: int) -> torch.Tensor:
    """N^(k)_{i,p}(u) for i = 0..n, shape [len(u), n+1] (k-times differentiated
    Cox-de Boor recursion; zero for k > p)."""
    m = U.shape[0] - 1
    levels = nb.basis_levels(U, p, u)

    def deriv(d: int, kk: int) -> torch.Tensor:
        if kk == 0:
            return levels[d]
        if kk > d:
            return torch.zeros(u.shape[0], m - d, dtype=DT)
        prev = deriv(d - 1, kk - 1)            # m - d + 1 functions of degree d - 1
        i = torch.arange(m - d)
        t1 = nb._ratio(d * prev[:, i], (U[i + d] - U[i])[None, :])
        t2 = nb._ratio(d * prev[:, i + 1], (U[i + d + 1] - U[i + 1])[None, :])
        return t1 - t2

    return deriv(p, k)


def curve_derivatives(cp: torch.Tensor, U: torch.Tensor, p: int, u: torch.Tensor, r: int):
    """[C, C', ..., C^(r)] of the planar part (x, y) at every u, each [len(u), 2]."""
    w = cp[:, 3][None, :]
    S, W = [], []
    for k in range(r + 1):
        Nk = basis_derivatives(U, p, u, k) * w
        S.append(Nk @ cp[:, :2])
        W.append(Nk.sum(1)[:, None])
    C = []
    for k in range(r + 1):
        acc = S[k]
        for i in range(1, k + 1):
            acc = acc - math.comb(k, i) * W[i] * C[k - i]
        C.append(acc / W[0])
    return C


def quadrature_nodes(a, b, n: int) -> torch.Tensor:
    """Midpoint nodes u_j = a + (j - 1/2)(b - a)/n, j = 1..n (the Eq. 3 rule)."""
    return a + (torch.arange(n, dtype=DT) + 0.5) * ((b - a) / n)


def curve_deriv_energy(cp, U, p: int, r: int, n: int) -> torch.Tensor:
    """Eq. 11 for one curve: (1/(b-a)) int |C^(r)_xy|^2 du by the n-node midpoint rule."""
    a, b = nb.domain(U, p)
    Cr = curve_derivatives(cp, U, p, quadrature_nodes(a, b, n), r)[r]
    return (Cr * Cr).sum(1).mean()


def deriv_loss(scene, key_t, tau_t, r: int, n: int) -> torch.Tensor:
    """Eq. 11 averaged over all curves of the batch."""
    tot = torch.zeros((), dtype=DT)
    for c in range(scene.n_curves):
        p, fl, cp, U = sm.curve_inputs(scene, c, key_t, tau_t)
        tot = tot + curve_deriv_energy(cp, U, p, r, n)
    return tot / scene.n_curves


def sample_positions(scene, c, key_t, tau_t, pl) -> torch.Tensor:
    """The curve points the sampler evaluates (Eq. 12's P_i): contour samples
    u_1..u_M of a stroke (§3.2 placement, no endpoint copies) or the boundary
    points of a filled curve (§3.3); [count, 2]."""
    p, fl, cp, U = sm.curve_inputs(scene, c, key_t, tau_t)
    a, b = nb.domain(U, p)
    if pl.kind == "fill":
        u = sm.boundary_parameters(a, b, pl.n_boundary)
    else:
        u = sm.contour_parameters(a, b, pl.m_contour, 0, pl.kind == "closed")
    return nb.curve_point(cp, U, p, u)[:, :2]


def penalty(x: torch.Tensor, kind: int) -> torch.Tensor:
    if kind == RELU:
        return torch.relu(x)
    if kind == SOFTPLUS:
        return torch.logaddexp(x, torch.zeros_like(x))
    raise ValueError("penalty must be RELU or SOFTPLUS")


def bbox_loss(scene, key_t, tau_t, plans, box, kind: int) -> torch.Tensor:
    """Eq. 12: sum over sampled positions of phi(b_min - P) + phi(P - b_max),
    per axis; box = (x_min, y_min, x_max, y_max)."""
    lo = torch.tensor(box[:2], dtype=DT)
    hi = torch.tensor(box[2:], dtype=DT)
    tot = torch.zeros((), dtype=DT)
    for c in range(scene.n_curves):
        P = sample_positions(scene, c, key_t, tau_t, plans[c])
        tot = tot + penalty(lo[None, :] - P, kind).sum() + penalty(P - hi[None, :], kind).sum()
    return tot


def geometry_loss_and_grads(scene, plans, order=3, nodes=None, lambda_deriv=1.0, lambda_bbox=1.0,
                            box=None, kind=RELU):
    """lambda_deriv * L_deriv^r + lambda_bbox * L_bbox and their exact gradients.
    nodes: quadrature nodes per curve (default N_L = nl_mult * max(W, H));
    box: default the canvas (0, 0, W, H).  Returns numpy values."""
    from .pipeline import leaves
    k, t, c = leaves(scene)
    n = nodes or int(scene.sample["nl_mult"]) * max(scene.width, scene.height)
    box = box or (0.0, 0.0, float(scene.width), float(scene.height))
    ld = lambda_deriv * deriv_loss(scene, k, t, order, n)
    lb = lambda_bbox * bbox_loss(scene, k, t, plans, box, kind)
    (ld + lb).backward()
    return dict(deriv=float(ld.detach()), bbox=float(lb.detach()), dkey=k.grad.numpy().copy(),
                dtau=t.grad.numpy().copy())
