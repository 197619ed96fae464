"""FP64 oracle, part 1: NURBS curves (paper §3.1, Eq. 1-3).

Test infrastructure: only the tests, the smoke check and the bench's CPU
baseline use this module.  Written for plain readability against the paper:
the basis functions come from the textbook Cox-de Boor recursion over *all*
n+1 functions (not the span-local triangle), with 0/0 taken as 0.
"""
from __future__ import annotations

import math

import torch

DT = torch.float64


def knot_vector(tau: torch.Tensor, p: int, closed: bool) -> torch.Tensor:
    """Knot vector from knot intervals (§3.1).

    Open: prepend and append p zero intervals, then a cumulative sum starting at
    0; the result is clamped with multiplicity p+1 at both ends.
    Closed: wrap the last p core intervals before and the first p after (indices
    taken cyclically), then the cumulative sum.
    """
    n = tau.shape[0]
    if closed:
        before = [(n - p + q) % n for q in range(p)]
        after = [q % n for q in range(p)]
        intervals = torch.cat([tau[before], tau, tau[after]])
    else:
        z = tau.new_zeros(p)
        intervals = torch.cat([z, tau, z])
    return torch.cat([tau.new_zeros(1), torch.cumsum(intervals, 0)])


def control_net(key: torch.Tensor, p: int, closed: bool) -> torch.Tensor:
    """Control points (x, y, s) and weights from key points (§3.1).

    Open curves use the key points directly.  Closed curves wrap the last
    ceil(p/2) and the first floor(p/2) key points around the polygon, giving
    n_k + p control points; weights and widths travel with their key point.
    Returns the [n+1, 4] rows {x, y, s, w}.
    """
    if not closed:
        return key
    nk = key.shape[0]
    nb, na = (p + 1) // 2, p // 2
    before = [(nk - nb + q) % nk for q in range(nb)]
    after = [q % nk for q in range(na)]
    return torch.cat([key[before], key, key[after]])


def domain(U: torch.Tensor, p: int):
    """Valid parameter range [u_p, u_{m-p}] (Eq. 3 limits)."""
    m = U.shape[0] - 1
    return U[p], U[m - p]


def span_index(U: torch.Tensor, p: int, u: torch.Tensor) -> torch.Tensor:
    """Knot span i with u_i <= u < u_{i+1} (Eq. 4), restricted to the curve's
    spans p..n.  At the right end of the domain, and wherever knots repeat, the
    largest i with u_i <= u among the non-empty spans (u_i < u_{i+1}) is taken,
    so the degree-0 function used is never the empty one."""
    m = U.shape[0] - 1
    n = m - p - 1
    Ud = U.detach()
    i = torch.arange(p, n + 1)
    ok = (Ud[i] < Ud[i + 1])[None, :] & (Ud[i][None, :] <= u.detach()[:, None])
    cand = torch.where(ok, i[None, :], torch.full_like(i[None, :], -1))
    s = cand.max(dim=1).values
    if bool((s < 0).any()):
        raise ValueError("parameter below the curve's domain")
    return s


def _ratio(num: torch.Tensor, den: torch.Tensor) -> torch.Tensor:
    """num/den with 0/0 (a zero-length knot span) taken as 0."""
    nz = den != 0
    return torch.where(nz, num / torch.where(nz, den, torch.ones_like(den)), torch.zeros_like(num))


def basis_levels(U: torch.Tensor, p: int, u: torch.Tensor):
    """Cox-de Boor recursion: returns [N_{.,0}, N_{.,1}, ..., N_{.,p}] evaluated at
    every u; level d holds the m-d functions N_{i,d}, i = 0..m-d-1.

        N_{i,0}(u) = 1 on the span of u, else 0
        N_{i,d}(u) = (u - u_i)/(u_{i+d} - u_i) N_{i,d-1}(u)
                   + (u_{i+d+1} - u)/(u_{i+d+1} - u_{i+1}) N_{i+1,d-1}(u)
    """
    m = U.shape[0] - 1
    s = span_index(U, p, u)
    N = (torch.arange(m)[None, :] == s[:, None]).to(DT)
    levels = [N]
    for d in range(1, p + 1):
        i = torch.arange(m - d)
        a = _ratio(u[:, None] - U[i][None, :], (U[i + d] - U[i])[None, :])
        b = _ratio(U[i + d + 1][None, :] - u[:, None], (U[i + d + 1] - U[i + 1])[None, :])
        N = a * N[:, : m - d] + b * N[:, 1 : m - d + 1]
        levels.append(N)
    return levels


def basis(U, p, u):
    """N_{i,p}(u) for i = 0..n, shape [len(u), n+1]."""
    return basis_levels(U, p, u)[p]


def basis_derivative(U, p, u):
    """N'_{i,p}(u) = p N_{i,p-1}/(u_{i+p} - u_i) - p N_{i+1,p-1}/(u_{i+p+1} - u_{i+1})."""
    m = U.shape[0] - 1
    n = m - p - 1
    Nm = basis_levels(U, p, u)[p - 1]
    i = torch.arange(n + 1)
    t1 = _ratio(p * Nm[:, i], (U[i + p] - U[i])[None, :])
    t2 = _ratio(p * Nm[:, i + 1], (U[i + p + 1] - U[i + 1])[None, :])
    return t1 - t2


def curve_point(cp: torch.Tensor, U: torch.Tensor, p: int, u: torch.Tensor) -> torch.Tensor:
    """C(u) = sum N_i w_i P_i / sum N_i w_i (Eq. 1) for P = (x, y, s): [len(u), 3]."""
    N = basis(U, p, u)
    Nw = N * cp[:, 3][None, :]
    S = Nw @ cp[:, :3]
    W = Nw.sum(1)
    return S / W[:, None]


def curve_derivative(cp: torch.Tensor, U: torch.Tensor, p: int, u: torch.Tensor) -> torch.Tensor:
    """C'(u) by the quotient rule (Eq. 2): (W S' - S W') / W^2, for (x, y, s)."""
    N = basis(U, p, u)
    dN = basis_derivative(U, p, u)
    w = cp[:, 3][None, :]
    S = (N * w) @ cp[:, :3]
    W = (N * w).sum(1)
    dS = (dN * w) @ cp[:, :3]
    dW = (dN * w).sum(1)
    return (W[:, None] * dS - S * dW[:, None]) / (W * W)[:, None]


def arc_length(cp: torch.Tensor, U: torch.Tensor, p: int, n_l: int) -> torch.Tensor:
    """Eq. 3 with N_L midpoint nodes u_j = a + (j - 1/2)(b - a)/N_L on the domain
    [u_p, u_{m-p}]; the norm is over the planar (x, y) part of C'."""
    a, b = domain(U, p)
    du = (b - a) / n_l
    u = a + (torch.arange(n_l, dtype=DT) + 0.5) * du
    d = curve_derivative(cp, U, p, u)[:, :2]
    return (torch.sqrt((d * d).sum(1)) * du).sum()


def bernstein_curve(cp: torch.Tensor, t: torch.Tensor) -> torch.Tensor:
    """Closed-form rational Bezier curve sum_i B_i^p(t) w_i P_i / sum_i B_i^p(t) w_i,
    with B_i^p(t) = binom(p, i) t^i (1-t)^(p-i); used to pin the recursion."""
    p = cp.shape[0] - 1
    B = torch.stack([math.comb(p, i) * t ** i * (1 - t) ** (p - i) for i in range(p + 1)], 1)
    Bw = B * cp[:, 3][None, :]
    return (Bw @ cp[:, :3]) / Bw.sum(1)[:, None]
