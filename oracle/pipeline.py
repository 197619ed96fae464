"""FP64 oracle, part 4: the whole step (sample -> render -> L2 loss) and its
exact gradient (paper §3.5: image loss back to control points, weights, knot
intervals, widths, colours and opacities).

Test infrastructure only.  Gradients come from `torch.autograd` through the
FP64 definition, with the discrete structure (counts, grid, spans, nearest
segment, winding sign) held fixed; `finite_difference` checks them.
"""
from __future__ import annotations

import numpy as np
import torch

from . import raster as rs
from . import sampling as sm

DT = torch.float64


def leaves(scene, requires_grad=True):
    """FP64 leaf tensors for the learnable inputs (key, tau, color)."""
    k = torch.tensor(scene.key, dtype=DT, requires_grad=requires_grad)
    t = torch.tensor(scene.tau, dtype=DT, requires_grad=requires_grad)
    c = torch.tensor(scene.color, dtype=DT, requires_grad=requires_grad)
    return k, t, c


def plan(scene):
    k, t, c = leaves(scene, False)
    return [sm.plan_curve(scene, i, k, t) for i in range(scene.n_curves)]


def render(scene, key_t, tau_t, color_t, plans=None, mode="tiled", return_flags=False):
    """Image [S, H, W, C] (FP64) of a batch and the Gaussians it was built from."""
    g = sm.sample_scene(scene, key_t, tau_t, color_t, plans)
    args = (g, color_t, scene.n_scenes, scene.height, scene.width, scene.channels, scene.raster)
    if mode == "brute":
        return rs.render_brute(*args), g
    if return_flags:
        img, fl = rs.render_tiled(*args, return_flags=True)
        return img, g, fl
    return rs.render_tiled(*args), g


def mse(image, target):
    """L2 image loss: mean of squared differences over S*H*W*C."""
    d = image - target
    return (d * d).mean()


def loss_and_grads(scene, plans=None, target=None, mode="tiled"):
    """Forward and exact backward.  Returns dict(image, loss, dkey [nk,4],
    dtau [nt], dcolor [nc,4], gaussians, plans) as numpy FP64."""
    k, t, c = leaves(scene)
    if plans is None:
        plans = plan(scene)
    img, g = render(scene, k, t, c, plans, mode)
    tgt = torch.as_tensor(scene.target if target is None else target, dtype=DT)
    L = mse(img, tgt)
    L.backward()
    return dict(image=img.detach().numpy(), loss=float(L.detach()), dkey=k.grad.numpy().copy(),
                dtau=t.grad.numpy().copy(), dcolor=c.grad.numpy().copy(),
                gaussians={kk: (v.detach().numpy() if torch.is_tensor(v) else v) for kk, v in g.items()},
                plans=plans)


def loss_value(scene, key, tau, color, plans, target=None, mode="tiled"):
    k = torch.as_tensor(key, dtype=DT)
    t = torch.as_tensor(tau, dtype=DT)
    c = torch.as_tensor(color, dtype=DT)
    with torch.no_grad():
        img, _ = render(scene, k, t, c, plans, mode)
        tgt = torch.as_tensor(scene.target if target is None else target, dtype=DT)
        return float(mse(img, tgt))


def finite_difference(scene, which, index, plans, eps_rel=1e-6, mode="tiled"):
    """Central difference of the loss with respect to one input entry, with the
    discrete structure frozen to `plans`."""
    arrs = dict(key=scene.key.astype(np.float64).copy(), tau=scene.tau.astype(np.float64).copy(),
                color=scene.color.astype(np.float64).copy())
    a = arrs[which].reshape(-1)
    x0 = a[index]
    eps = eps_rel * max(1.0, abs(x0))
    a[index] = x0 + eps
    lp = loss_value(scene, arrs["key"], arrs["tau"], arrs["color"], plans, mode=mode)
    a[index] = x0 - eps
    lm = loss_value(scene, arrs["key"], arrs["tau"], arrs["color"], plans, mode=mode)
    a[index] = x0
    return (lp - lm) / (2 * eps)


def gaussians_fp32(scene, plans=None):
    """The batch's Gaussians as FP32 arrays in front-to-back order per scene
    (scene ascending, layer ascending, sample ascending): the order a renderer
    consumes them in.  Returns dict(rec [G,4] {mu_x, mu_y, sigma, o},
    curve [G] int32, layer, sample, scene, order)."""
    k, t, c = leaves(scene, False)
    with torch.no_grad():
        g = sm.sample_scene(scene, k, t, c, plans)
    key = (g["scene"].numpy().astype(np.int64) << 40) + (g["layer"].numpy().astype(np.int64) << 24) \
        + g["sample"].numpy().astype(np.int64)
    order = np.argsort(key, kind="stable")
    rec = np.zeros((order.shape[0], 4), np.float32)
    rec[:, 0:2] = g["mu"].numpy()[order]
    rec[:, 2] = g["sigma"].numpy()[order]
    rec[:, 3] = g["o"].numpy()[order]
    out = dict(rec=rec, curve=g["curve"].numpy()[order].astype(np.int32),
               layer=g["layer"].numpy()[order], sample=g["sample"].numpy()[order],
               scene=g["scene"].numpy()[order], order=order, plans=g["plans"])
    if "shape" in g:
        shape = np.zeros((order.shape[0], 4), np.float32)   # {sigma_t, cos, sin, 0}
        shape[:, 0:3] = g["shape"].numpy()[order]
        out["shape"] = shape
    return out


def render_records(scene, rec, curve, mode="tiled", return_flags=False, shape=None):
    """Render a given FP32 Gaussian set (front to back per scene, as produced
    by `gaussians_fp32`) in FP64.  Layer and sample are re-derived from the
    position in that order, so the sort key is the same one the set came in.
    shape: [G, 4] {sigma_t, cos, sin, 0} for tangent-aligned records."""
    cs = scene.curve_scene()
    rec64 = torch.as_tensor(rec.astype(np.float64))
    curve_t = torch.as_tensor(curve.astype(np.int64))
    scene_of = torch.as_tensor(cs[curve].astype(np.int64))
    off = scene.scene_curve_offset
    layer = torch.as_tensor((off[cs[curve] + 1] - 1 - curve).astype(np.int64))
    G = rec.shape[0]
    sample = torch.arange(G)   # position order inside each (scene, layer) group
    g = dict(mu=rec64[:, 0:2], sigma=rec64[:, 2], o=rec64[:, 3], curve=curve_t, sample=sample,
             layer=layer, scene=scene_of)
    if shape is not None:
        g["shape"] = torch.as_tensor(np.asarray(shape)[:, :3].astype(np.float64))
    color_t = torch.as_tensor(scene.color, dtype=DT)
    args = (g, color_t, scene.n_scenes, scene.height, scene.width, scene.channels, scene.raster)
    if mode == "brute":
        return rs.render_brute(*args).numpy()
    if return_flags:
        img, fl = rs.render_tiled(*args, return_flags=True)
        return img.numpy(), fl.numpy()
    return rs.render_tiled(*args).numpy()


def _records_g(scene, rec, curve, requires_grad=False, shape=None):
    cs = scene.curve_scene()
    rec64 = torch.tensor(rec.astype(np.float64), requires_grad=requires_grad)
    off = scene.scene_curve_offset
    g = dict(mu=rec64[:, 0:2], sigma=rec64[:, 2], o=rec64[:, 3],
             curve=torch.as_tensor(curve.astype(np.int64)), sample=torch.arange(rec.shape[0]),
             layer=torch.as_tensor((off[cs[curve] + 1] - 1 - curve).astype(np.int64)),
             scene=torch.as_tensor(cs[curve].astype(np.int64)))
    shape64 = None
    if shape is not None:
        shape64 = torch.tensor(np.asarray(shape)[:, :3].astype(np.float64), requires_grad=requires_grad)
        g["shape"] = shape64
    return rec64, g, shape64


def pairs_records(scene, rec, curve, shape=None):
    """Sorted (tile, Gaussian) pairs of a given FP32 Gaussian set in the
    documented order; Gaussian ids are positions in that set."""
    _, g, _ = _records_g(scene, rec, curve, shape=shape)
    r = scene.raster
    return rs.sorted_pairs(g, scene.height, scene.width, int(r["tile"]), r["k_sigma"], r["alpha_min"],
                           scene.n_scenes)


def record_grads(scene, rec, curve, dimage, shape=None):
    """Gradient of sum(image * dimage) with respect to each record's
    (mu_x, mu_y, sigma, o) and each curve's colour, for a given FP32 set;
    with tangent-aligned records also with respect to (sigma_t, cos, sin),
    returned as a third array."""
    rec64, g, shape64 = _records_g(scene, rec, curve, requires_grad=True, shape=shape)
    color_t = torch.tensor(scene.color.astype(np.float64), requires_grad=True)
    img = rs.render_tiled(g, color_t, scene.n_scenes, scene.height, scene.width, scene.channels, scene.raster)
    (img * torch.as_tensor(dimage, dtype=DT)).sum().backward()
    if shape64 is not None:
        return rec64.grad.numpy(), color_t.grad.numpy(), shape64.grad.numpy()
    return rec64.grad.numpy(), color_t.grad.numpy()
