"""FP64 oracle, part 2: Gaussian sampling (paper §3.2 contours, §3.3 regions,
supplementary "Signed Distance Field Evaluation", Eq. S1-S3).

Test infrastructure only.  Every discrete choice (sample counts, grid size and
origin, winding sign, nearest segment) is computed here in FP64 and treated as
piecewise constant for the gradient; the continuous quantities stay on the
autograd tape so that `torch.autograd` yields the exact derivative.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

from . import nurbs as nb

DT = torch.float64
FLAG_CLOSED = 1
FLAG_FILLED = 2


@dataclass
class CurvePlan:
    """Discrete structure of one curve's Gaussians (frozen for finite differences)."""
    length: float = 0.0           # arc length L (Eq. 3)
    kind: str = "open"            # "open", "closed" (stroke) or "fill"
    m_contour: int = 0            # M = ceil(delta_c L)
    n_boundary: int = 0           # ceil(delta_b L)
    x0: float = 0.0               # grid origin (padded, clipped box corner)
    y0: float = 0.0
    nx: int = 0
    ny: int = 0
    count: int = 0                # Gaussians this curve emits
    # distance of each discrete decision from a tie: count decisions in counts
    # (ceil() of Eq. 3-based sizes); for fills, once their Gaussians are
    # sampled, "sign": the smallest distance (px) of a grid point from the
    # boundary polyline.  At such a point the winding sign of Eq. S3 can flip
    # under rounding of the polyline, which leaves sdf ~ 0 unchanged but
    # reverses the sign of its gradient with respect to the polyline.
    margin: dict = field(default_factory=dict)

    def well_separated(self, count_bar: float = 1e-3, sign_bar_px: float = 1e-4) -> bool:
        """True when every discrete decision is far from a tie: each count at
        least count_bar from an integer, and every fill grid point at least
        sign_bar_px from the polyline (about ten times the rounding of a
        float32 boundary point at these canvas sizes)."""
        return all(v > (sign_bar_px if k == "sign" else count_bar) for k, v in self.margin.items())


def curve_inputs(scene, c, key_t, tau_t):
    """Per-curve tensors: degree, flags, control net rows {x, y, s, w}, knot vector."""
    p = int(scene.degree[c])
    fl = int(scene.flags[c])
    closed = bool(fl & FLAG_CLOSED)
    k0, k1 = int(scene.key_offset[c]), int(scene.key_offset[c + 1])
    t0, t1 = int(scene.tau_offset[c]), int(scene.tau_offset[c + 1])
    cp = nb.control_net(key_t[k0:k1], p, closed)
    U = nb.knot_vector(tau_t[t0:t1], p, closed)
    return p, fl, cp, U


def contour_parameters(a, b, M: int, kappa: int, closed: bool):
    """Sample parameters along the domain (§3.2).

    Open: M values uniformly from a to b inclusive, u_j = a + (j-1)(b-a)/(M-1),
    plus kappa extra copies of the first and of the last centre (ordered
    [first x kappa, u_1..u_M, last x kappa]).  Closed: u_j = a + (j-1)(b-a)/M,
    which does not repeat the start point.
    """
    if closed:
        t = torch.arange(M, dtype=DT) / M
        return a + t * (b - a)
    t = torch.arange(M, dtype=DT) / (M - 1)
    u = a + t * (b - a)
    first = u[:1].expand(kappa)
    last = u[-1:].expand(kappa)
    return torch.cat([first, u, last])


def boundary_parameters(a, b, B: int):
    """Boundary polyline parameters: B values a + i(b-a)/B, i = 0..B-1 (§3.3)."""
    return a + torch.arange(B, dtype=DT) / B * (b - a)


def unsigned_distance(q: torch.Tensor, poly: torch.Tensor):
    """Eq. S1: min over closed-polyline segments of |q - proj(q)|, the projection
    parameter clamped to [0, 1].  Returns (d, index of the nearest segment)."""
    b0 = poly
    b1 = torch.roll(poly, -1, 0)
    e = b1 - b0                                                   # [B, 2]
    rel = q[:, None, :] - b0[None, :, :]                          # [Q, B, 2]
    ee = (e * e).sum(1)
    t = _safe_div((rel * e[None]).sum(2), ee[None, :]).clamp(0.0, 1.0)
    diff = rel - t[..., None] * e[None]
    d2 = (diff * diff).sum(2)
    d2min, arg = d2.min(1)
    return torch.sqrt(d2min), arg


def _safe_div(a, b):
    nz = b != 0
    return torch.where(nz, a / torch.where(nz, b, torch.ones_like(b)), torch.zeros_like(a))


def winding_number(q: torch.Tensor, poly: torch.Tensor) -> torch.Tensor:
    """Eq. S2: (1/2pi) sum of signed angles between b_i - q and b_{i+1} - q,
    angle(a, b) = atan2(a x b, a . b).  Detached: it only provides the sign."""
    q = q.detach()
    b0 = poly.detach()[None] - q[:, None]
    b1 = torch.roll(poly.detach(), -1, 0)[None] - q[:, None]
    cross = b0[..., 0] * b1[..., 1] - b0[..., 1] * b1[..., 0]
    dot = (b0 * b1).sum(2)
    return torch.atan2(cross, dot).sum(1) / (2 * math.pi)


def inside_sign(wn: torch.Tensor, fill_rule: int) -> torch.Tensor:
    """Eq. S3 sign: +1 inside, -1 outside.  Rule 0 (the paper): inside iff
    wn > 0.5; rule 1 (nonzero): inside iff |wn| > 0.5."""
    w = wn if fill_rule == 0 else wn.abs()
    return torch.where(w > 0.5, torch.ones_like(w), -torch.ones_like(w))


def sigmoid(z):
    return 1.0 / (1.0 + torch.exp(-z))


def plan_curve(scene, c, key_t, tau_t) -> CurvePlan:
    """Counts and grid of one curve (§3.2, §3.3), decided in FP64."""
    sp = scene.sample
    p, fl, cp, U = curve_inputs(scene, c, key_t, tau_t)
    closed = bool(fl & FLAG_CLOSED)
    filled = bool(fl & FLAG_FILLED)
    n_l = int(sp["nl_mult"]) * max(scene.width, scene.height)
    with torch.no_grad():
        L = float(nb.arc_length(cp.detach(), U.detach(), p, n_l))
    pl = CurvePlan(length=L)
    if filled:
        pl.kind = "fill"
        xB = sp["delta_b"] * L
        pl.n_boundary = max(3, math.ceil(xB))
        pl.margin["boundary"] = abs(xB - round(xB))
        with torch.no_grad():
            a, b = nb.domain(U.detach(), p)
            poly = nb.curve_point(cp.detach(), U.detach(), p,
                                  boundary_parameters(a, b, pl.n_boundary))[:, :2]
        h = float(sp["h"])
        lo = poly.min(0).values
        hi = poly.max(0).values
        ext = hi - lo
        pad = sp["pad_frac"] * ext
        x0 = max(0.0, float(lo[0] - pad[0]))
        x1 = min(float(scene.width), float(hi[0] + pad[0]))
        y0 = max(0.0, float(lo[1] - pad[1]))
        y1 = min(float(scene.height), float(hi[1] + pad[1]))
        pl.x0, pl.y0 = x0, y0
        pl.nx = math.ceil((x1 - x0) / h) if x1 > x0 else 0
        pl.ny = math.ceil((y1 - y0) / h) if y1 > y0 else 0
        for nm, lo_, hi_ in (("nx", x0, x1), ("ny", y0, y1)):
            v = (hi_ - lo_) / h
            pl.margin[nm] = abs(v - round(v)) if hi_ > lo_ else 1.0
        pl.count = pl.nx * pl.ny
    else:
        xM = sp["delta_c"] * L
        M = math.ceil(xM)
        pl.margin["contour"] = abs(xM - round(xM))
        if closed:
            pl.kind = "closed"
            pl.m_contour = max(1, M)
            pl.count = pl.m_contour
        else:
            pl.kind = "open"
            pl.m_contour = max(2, M)
            pl.count = pl.m_contour + 2 * int(sp["kappa"])
    return pl


def curve_gaussians(scene, c, key_t, tau_t, color_t, pl: CurvePlan):
    """Gaussians of one curve in sample order: (mu [G,2], sigma [G], o [G], aux).

    Contour (§3.2, Eq. 4-5): mu_j = C_xy(u_j), sigma_j = C_s(u_j)/rho, o_j = o.
    Fill (§3.3, Eq. 6-7): mu_j = grid point q_j (row-major over the padded box,
    q = origin + (i + 1/2) h), sigma = eta h / rho,
    o_j = o * sigmoid(gamma/h * sdf(q_j)) with sdf from Eq. S1-S3 against the
    boundary polyline b_i = C_xy(a + i(b-a)/B).
    aux holds, for fills, (nearest segment, inside sign); None for contours.
    """
    sp = scene.sample
    p, fl, cp, U = curve_inputs(scene, c, key_t, tau_t)
    o = color_t[c, 3]
    a, b = nb.domain(U, p)
    if pl.kind == "fill":
        h = float(sp["h"])
        if pl.count == 0:
            z = torch.zeros(0, dtype=DT)
            return torch.zeros(0, 2, dtype=DT), z, z, (torch.zeros(0, dtype=torch.long), z)
        poly = nb.curve_point(cp, U, p, boundary_parameters(a, b, pl.n_boundary))[:, :2]
        iy, ix = torch.meshgrid(torch.arange(pl.ny, dtype=DT), torch.arange(pl.nx, dtype=DT),
                                indexing="ij")
        q = torch.stack([pl.x0 + (ix.reshape(-1) + 0.5) * h, pl.y0 + (iy.reshape(-1) + 0.5) * h], 1)
        d, arg = unsigned_distance(q, poly)
        pl.margin["sign"] = float(d.detach().min())
        sgn = inside_sign(winding_number(q, poly), int(sp["fill_rule"]))
        sdf = sgn * d
        oj = o * sigmoid(sp["gamma"] / h * sdf)
        sigma = torch.full((q.shape[0],), sp["eta"] * h / sp["rho"], dtype=DT)
        return q, sigma, oj, (arg, sgn)   # fills stay isotropic in every contour mode
    closed = pl.kind == "closed"
    u = contour_parameters(a, b, pl.m_contour, int(sp["kappa"]), closed)
    C = nb.curve_point(cp, U, p, u)
    sigma = C[:, 2] / sp["rho"]
    if int(sp.get("contour_mode", 0)) == 1:
        return C[:, :2], sigma, o.expand(u.shape[0]), tangent_shape(cp, U, p, u, a, b, pl, sp, sigma)
    return C[:, :2], sigma, o.expand(u.shape[0]), None


def tangent_shape(cp, U, p, u, a, b, pl, sp, sigma_n):
    """Tangent-aligned contour Gaussians (the anisotropic prototype): the unit
    tangent (cos, sin) = C'_xy/|C'_xy| (Eq. 2) and sigma_t = |C'_xy| du / rho,
    du the parameter step between consecutive samples ((b - a)/(M - 1) open,
    (b - a)/M closed): the arc length between samples over the same ratio rho
    as the width.  Where C' vanishes: tangent (1, 0) and sigma_t = sigma_n.
    Returns [G, 3] = (sigma_t, cos, sin)."""
    d = nb.curve_derivative(cp, U, p, u)
    v = d[:, :2]
    n = torch.sqrt((v * v).sum(1))
    step = (b - a) / (pl.m_contour - 1 if pl.kind == "open" else pl.m_contour)
    ok = n > 0
    nn = torch.where(ok, n, torch.ones_like(n))
    cs = torch.where(ok, v[:, 0] / nn, torch.ones_like(n))
    sn = torch.where(ok, v[:, 1] / nn, torch.zeros_like(n))
    st = torch.where(ok, n * step / sp["rho"], sigma_n)
    return torch.stack([st, cs, sn], 1)


def sample_scene(scene, key_t, tau_t, color_t, plans=None):
    """All Gaussians of a batch.  Returns a dict of per-Gaussian tensors, with
    layer (0 = front; the last curve of a scene is in front) and sample index,
    plus the plans used.  Pass `plans` to freeze the discrete structure."""
    if plans is None:
        plans = [plan_curve(scene, c, key_t, tau_t) for c in range(scene.n_curves)]
    mus, sigmas, ops, curves, samples, layers, scenes_, shapes = [], [], [], [], [], [], [], []
    cs = scene.curve_scene()
    aniso = int(scene.sample.get("contour_mode", 0)) == 1
    for c in range(scene.n_curves):
        mu, sg, oj, extra = curve_gaussians(scene, c, key_t, tau_t, color_t, plans[c])
        G = mu.shape[0]
        s = int(cs[c])
        mus.append(mu)
        sigmas.append(sg)
        if aniso:
            if plans[c].kind == "fill" or extra is None:
                ones = torch.ones(G, dtype=DT)
                shapes.append(torch.stack([sg, ones, torch.zeros(G, dtype=DT)], 1))
            else:
                shapes.append(extra)
        ops.append(oj)
        curves.append(torch.full((G,), c, dtype=torch.long))
        samples.append(torch.arange(G))
        layers.append(torch.full((G,), int(scene.scene_curve_offset[s + 1]) - 1 - c, dtype=torch.long))
        scenes_.append(torch.full((G,), s, dtype=torch.long))
    cat = lambda xs, shape: torch.cat(xs) if xs else torch.zeros(shape)
    out = dict(mu=cat(mus, (0, 2)), sigma=cat(sigmas, (0,)), o=cat(ops, (0,)),
               curve=cat(curves, (0,)).long(), sample=cat(samples, (0,)).long(),
               layer=cat(layers, (0,)).long(), scene=cat(scenes_, (0,)).long(), plans=plans)
    if aniso:
        out["shape"] = cat(shapes, (0, 3))
    return out
