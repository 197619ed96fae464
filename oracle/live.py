"""FP64 oracle, part 7: the losses and the seeding of the layer-wise
vectorisation loop (§4.2, "Layer-wise Image Vectorization", adapted from LIVE):
the distance-weighted image loss, the self-crossing penalty and the choice of
where a new path starts.

Test infrastructure only: the tests, the smoke check and the bench's CPU
baseline use this module.

Readings (the paper names these terms but does not define them):
  - Distance-weighted loss: per pixel i of a scene that received a new path,
    d_i is the distance from the pixel centre to that path's closed boundary
    polyline (§3.3's boundary points) and w_i = max(0, tau - d_i).  The scene's
    loss is sum_i w_i sum_c (I_ic - I*_ic)^2 / (C sum_i w_i); a scene without a
    new path (or with no pixel within tau) takes the plain mean square error.
    The batch loss is the mean over scenes.  The weights are constants: no
    gradient flows through d_i.
  - Self-crossing penalty: for every curve, the legs a_i = K_{i+1} - K_i of its
    key-point polygon (cyclic for closed curves), the sine of each turn
    sin_i = (a_i x a_{i+1}) / (|a_i| |a_{i+1}|), and the curve's winding sign
    sigma = sign(sum_i a_i x a_{i+1}) (held fixed): L_xing = sum over curves and
    turns of max(0, -sigma sin_i), i.e. turns against the curve's own winding.
  - Seeding: per scene, the squared error e_i = sum_c (I_ic - I*_ic)^2, its sum
    over the (2r+1) x (2r+1) window centred on each pixel (clipped to the
    image), and the pixel with the largest window sum (ties: the first in
    row-major order).
"""
from __future__ import annotations

import numpy as np
import torch

from . import nurbs as nb
from . import sampling as sm

DT = torch.float64


def segment_distance(q: torch.Tensor, poly: torch.Tensor) -> torch.Tensor:
    """Distance from points q [n, 2] to the closed polyline poly [B, 2] (segments
    b_k -> b_{k+1}, the last one closing the loop)."""
    d, _ = sm.unsigned_distance(q, poly)
    return d


def boundary_polyline(scene, c, key_t, tau_t, pl) -> torch.Tensor:
    """The boundary points of filled curve c (§3.3), [B, 2]."""
    p, fl, cp, U = sm.curve_inputs(scene, c, key_t, tau_t)
    a, b = nb.domain(U, p)
    return nb.curve_point(cp, U, p, sm.boundary_parameters(a, b, pl.n_boundary))[:, :2]


def udf_weights(scene, key_t, tau_t, plans, new_curve, tau):
    """w [S, H, W] for the distance-weighted loss; new_curve[s] is the curve
    index of scene s's new path or -1."""
    S, H, W = scene.n_scenes, scene.height, scene.width
    iy, ix = torch.meshgrid(torch.arange(H, dtype=DT), torch.arange(W, dtype=DT), indexing="ij")
    q = torch.stack([ix.reshape(-1) + 0.5, iy.reshape(-1) + 0.5], 1)
    out = torch.zeros(S, H, W, dtype=DT)
    for s in range(S):
        c = int(new_curve[s])
        if c < 0:
            continue
        with torch.no_grad():
            poly = boundary_polyline(scene, c, key_t.detach(), tau_t.detach(), plans[c])
            d = segment_distance(q, poly)
        out[s] = torch.clamp(tau - d, min=0.0).reshape(H, W)
    return out


def udf_mse(image, target, weights, has_path):
    """Mean over scenes of the distance-weighted (or plain) squared error."""
    S, H, W, C = image.shape
    e = ((image - target) ** 2).sum(-1)          # [S, H, W]
    terms = []
    for s in range(S):
        wsum = weights[s].sum()
        if has_path[s] and float(wsum) > 0.0:
            terms.append((weights[s] * e[s]).sum() / (C * wsum))
        else:
            terms.append(e[s].mean() / C)
    return torch.stack(terms).mean()


def xing_loss(scene, key_t) -> torch.Tensor:
    """Self-crossing penalty over every curve's key-point polygon."""
    tot = torch.zeros((), dtype=DT)
    for c in range(scene.n_curves):
        k0, k1 = int(scene.key_offset[c]), int(scene.key_offset[c + 1])
        P = key_t[k0:k1, :2]
        closed = bool(int(scene.flags[c]) & sm.FLAG_CLOSED)
        if closed:
            a = torch.roll(P, -1, 0) - P                 # a_i = K_{i+1} - K_i, cyclic
            b = torch.roll(a, -1, 0)
        else:
            if P.shape[0] < 3:
                continue
            a = P[1:-1] - P[:-2]
            b = P[2:] - P[1:-1]
        cross = a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]
        norm = torch.sqrt((a * a).sum(1)) * torch.sqrt((b * b).sum(1))
        sgn = 1.0 if float(cross.detach().sum()) >= 0.0 else -1.0
        ok = norm > 0
        sin = torch.where(ok, cross / torch.where(ok, norm, torch.ones_like(norm)), torch.zeros_like(cross))
        tot = tot + torch.relu(-sgn * sin).sum()
    return tot


def seed_pixels(image: np.ndarray, target: np.ndarray, r: int):
    """Per scene, (x, y, window sum) of the pixel whose (2r+1)^2 window of
    squared error is largest (first in row-major order on ties)."""
    e = ((image.astype(np.float64) - target.astype(np.float64)) ** 2).sum(-1)   # [S, H, W]
    S, H, W = e.shape
    out = []
    for s in range(S):
        best, arg = -1.0, (0, 0)
        for y in range(H):
            y0, y1 = max(0, y - r), min(H, y + r + 1)
            for x in range(W):
                x0, x1 = max(0, x - r), min(W, x + r + 1)
                v = float(e[s, y0:y1, x0:x1].sum())
                if v > best:
                    best, arg = v, (x, y)
        out.append((arg[0], arg[1], best))
    return out
