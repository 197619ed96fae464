"""FP64 oracle, part 3: tile binning and alpha compositing (paper §3.4, Eq. 8-9).

Test infrastructure only.  The image is computed from the definition:
    alpha_i(x) = min(alpha_max, o_i exp(-|x - mu_i|^2 / (2 sigma_i^2)))      (Eq. 9)
    I(x) = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j) + T_final bg            (Eq. 8)
over the Gaussians in depth order (front first).  Pixel (x, y) is sampled at
(x + 1/2, y + 1/2).  Thresholds the paper leaves to its rasterizer: a Gaussian
with alpha < alpha_min is skipped, and compositing stops before a Gaussian
that would take the transmittance below t_min.

The tangent-aligned variant (the paper's anisotropic prototype, §3.2 and the
supplement's comparison with Bezier Splatting) replaces the isotropic exponent
by -(along^2 / sigma_t^2 + across^2 / sigma_n^2) / 2 in the tangent frame.

Two renders are provided: brute force over every Gaussian of a scene, and the
tiled render over per-tile lists built with the FP32 bin rule.  The bin rule
and the sort order are computed in IEEE float32 (numpy, one rounding per
operation) so that a GPU implementation can be compared bit for bit.
"""
from __future__ import annotations

import numpy as np
import torch

DT = torch.float64


def alpha(px, py, mu, sigma, o, alpha_max, shape=None):
    """Eq. 9 with the cap alpha_max: [P] pixels x [G] Gaussians.

    shape [G, 3] = (sigma_t, cos theta, sin theta) gives the tangent-aligned
    (anisotropic) variant: the offset is written in the frame of the unit
    tangent (cos, sin) and its normal, with deviations sigma_t along the
    tangent and sigma (= sigma_n) across it."""
    dx = px[:, None] - mu[None, :, 0]
    dy = py[:, None] - mu[None, :, 1]
    if shape is None:
        a = o[None, :] * torch.exp(-(dx * dx + dy * dy) / (2.0 * sigma * sigma)[None, :])
    else:
        st, c, s = shape[:, 0][None, :], shape[:, 1][None, :], shape[:, 2][None, :]
        along = dx * c + dy * s
        across = -dx * s + dy * c
        a = o[None, :] * torch.exp(-0.5 * (along * along / (st * st) + across * across / (sigma * sigma)[None, :]))
    return torch.clamp(a, max=alpha_max)


def composite_sequential(al, color, bg, alpha_min, t_min):
    """Eq. 8 front to back, one Gaussian at a time, for every pixel at once.
    al [P, G] in depth order, color [G, C].  Returns (image [P, C], T_final [P],
    n_used [P]) where n_used counts the list entries the pixel walked through."""
    P, G = al.shape
    C = color.shape[1]
    out = torch.zeros(P, C, dtype=DT)
    T = torch.ones(P, dtype=DT)
    live = torch.ones(P, dtype=torch.bool)
    n_used = torch.zeros(P, dtype=torch.long)
    for i in range(G):
        a = al[:, i]
        use = live & (a >= alpha_min)
        test = T * (1.0 - a)
        stop = use & (test < t_min)
        live = live & ~stop
        use = use & ~stop
        out = out + torch.where(use[:, None], color[i][None, :] * (a * T)[:, None], torch.zeros_like(out))
        T = torch.where(use, test, T)
        n_used = torch.where(live, torch.full_like(n_used, i + 1), n_used)
    out = out + T[:, None] * torch.as_tensor(bg, dtype=DT)[None, :]
    return out, T, n_used


def composite_cumprod(al, color, bg, alpha_min, t_min):
    """The same result as `composite_sequential`, written with a cumulative
    product: skipped entries have alpha 0, a pixel is live up to (not including)
    the first entry whose inclusive transmittance falls below t_min."""
    P, G = al.shape
    if G == 0:
        T = torch.ones(P, dtype=DT)
        return T[:, None] * torch.as_tensor(bg, dtype=DT)[None, :], T
    a = torch.where(al >= alpha_min, al, torch.zeros_like(al))
    T_incl = torch.cumprod(1.0 - a, dim=1)
    live = T_incl >= t_min
    T_excl = torch.cat([torch.ones(P, 1, dtype=DT), T_incl[:, :-1]], 1)
    w = torch.where(live, a * T_excl, torch.zeros_like(a))
    T_final = torch.where(live, 1.0 - a, torch.ones_like(a)).prod(1)
    out = w @ color + T_final[:, None] * torch.as_tensor(bg, dtype=DT)[None, :]
    return out, T_final


def near_threshold(al, alpha_min, t_min, rel=1e-4):
    """Pixels whose result depends on a threshold decision within `rel` of a
    tie (alpha near alpha_min, or inclusive transmittance near t_min); FP32
    and FP64 may decide these differently."""
    with torch.no_grad():
        if al.shape[1] == 0:
            return torch.zeros(al.shape[0], dtype=torch.bool)
        a = torch.where(al >= alpha_min, al, torch.zeros_like(al))
        T_incl = torch.cumprod(1.0 - a, dim=1)
        f1 = ((al - alpha_min).abs() <= rel * max(alpha_min, 1e-30)).any(1) if alpha_min > 0 else \
            torch.zeros(al.shape[0], dtype=torch.bool)
        f2 = ((T_incl - t_min).abs() <= rel * t_min).any(1)
        return f1 | f2


# ----------------------------------------------------------------------------
# binning (FP32, bit-exact rule)

def tile_rects(mu, sigma, o, tile, k_sigma, alpha_min, tiles_x, tiles_y, shape=None):
    """Per-Gaussian inclusive tile rectangle [x_lo, x_hi] x [y_lo, y_hi], or an
    empty one.  Every step is one IEEE float32 operation rounded to nearest:
        ks = k_sigma * sigma;  x_lo = floor((mu_x - ks) * (1/tile));
        x_hi = floor((mu_x + ks) * (1/tile)); the same in y; clipped to the grid.
    With a tangent-aligned shape (sigma_t, c, s) the half widths are those of
    the k_sigma ellipse's bounding box,
        kx = k_sigma * sqrt(sigma_t^2 c^2 + sigma^2 s^2),
        ky = k_sigma * sqrt(sigma_t^2 s^2 + sigma^2 c^2),
    each square, product, sum and the (correctly rounded) square root one
    float32 operation, in that order.
    A Gaussian with sigma <= 0, o <= 0 or o < alpha_min covers no tile (it
    cannot reach alpha_min anywhere)."""
    mu = np.asarray(mu, np.float32)
    s = np.asarray(sigma, np.float32)
    o = np.asarray(o, np.float32)
    inv = np.float32(1.0 / tile)
    k = np.float32(k_sigma)
    if shape is None:
        kx = ky = k * s
        ok = s > 0
    else:
        sh = np.asarray(shape, np.float32)
        st, cs, sn = sh[:, 0], sh[:, 1], sh[:, 2]
        st2, cs2, sn2, sg2 = st * st, cs * cs, sn * sn, s * s
        kx = k * np.sqrt(st2 * cs2 + sg2 * sn2)
        ky = k * np.sqrt(st2 * sn2 + sg2 * cs2)
        ok = (s > 0) & (st > 0)
    xlo = np.floor((mu[:, 0] - kx) * inv)
    xhi = np.floor((mu[:, 0] + kx) * inv)
    ylo = np.floor((mu[:, 1] - ky) * inv)
    yhi = np.floor((mu[:, 1] + ky) * inv)
    valid = ok & (o > 0) & (o >= np.float32(alpha_min))
    valid &= (xhi >= 0) & (yhi >= 0) & (xlo <= tiles_x - 1) & (ylo <= tiles_y - 1)
    xlo = np.clip(xlo, 0, tiles_x - 1).astype(np.int64)
    xhi = np.clip(xhi, 0, tiles_x - 1).astype(np.int64)
    ylo = np.clip(ylo, 0, tiles_y - 1).astype(np.int64)
    yhi = np.clip(yhi, 0, tiles_y - 1).astype(np.int64)
    return xlo, xhi, ylo, yhi, valid


def sorted_pairs(g, H, W, tile, k_sigma, alpha_min, n_scenes):
    """(global tile, Gaussian) pairs sorted by the key (tile, layer, sample)
    ascending, i.e. front to back inside each tile.  Returns (tile_ids,
    gaussian_ids) as int64 arrays and the per-tile [start, end) ranges."""
    tx = (W + tile - 1) // tile
    ty = (H + tile - 1) // tile
    mu = g["mu"].detach().numpy()
    sg = g["sigma"].detach().numpy()
    o = g["o"].detach().numpy()
    shape = g.get("shape")
    shape = None if shape is None else shape.detach().numpy()
    xlo, xhi, ylo, yhi, valid = tile_rects(mu, sg, o, tile, k_sigma, alpha_min, tx, ty, shape)
    layer = g["layer"].numpy()
    sample = g["sample"].numpy()
    scene = g["scene"].numpy()
    idx = np.nonzero(valid)[0]
    nx = (xhi - xlo + 1)[idx]
    ny = (yhi - ylo + 1)[idx]
    cnt = nx * ny
    gi = np.repeat(idx, cnt)                                  # Gaussian of each pair
    k = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)   # pair number within it
    nxr = np.repeat(nx, cnt)
    tyy = ylo[gi] + k // nxr
    txx = xlo[gi] + k % nxr
    rows = np.stack([scene[gi] * tx * ty + tyy * tx + txx, layer[gi], sample[gi], gi], 1)
    n_tiles = n_scenes * tx * ty
    if rows.shape[0] == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros((n_tiles, 2), np.int64)
    arr = rows.astype(np.int64)
    order = np.lexsort((arr[:, 2], arr[:, 1], arr[:, 0]))
    arr = arr[order]
    ranges = np.zeros((n_tiles, 2), np.int64)
    starts = np.searchsorted(arr[:, 0], np.arange(n_tiles), "left")
    ends = np.searchsorted(arr[:, 0], np.arange(n_tiles), "right")
    ranges[:, 0] = starts
    ranges[:, 1] = ends
    ranges[starts == ends] = 0
    return arr[:, 0], arr[:, 3], ranges


# ----------------------------------------------------------------------------
# renders

def _colors(g, color_t, C):
    return color_t[g["curve"], :C]


def render_brute(g, color_t, n_scenes, H, W, C, r):
    """Every pixel against every Gaussian of its scene, in depth order."""
    imgs = []
    yy, xx = torch.meshgrid(torch.arange(H, dtype=DT) + 0.5, torch.arange(W, dtype=DT) + 0.5, indexing="ij")
    px, py = xx.reshape(-1), yy.reshape(-1)
    col = _colors(g, color_t, C)
    for s in range(n_scenes):
        sel = torch.nonzero(g["scene"] == s).reshape(-1)
        key = g["layer"][sel] * (1 << 32) + g["sample"][sel]
        sel = sel[torch.argsort(key)]
        shp = g.get("shape")
        al = alpha(px, py, g["mu"][sel], g["sigma"][sel], g["o"][sel], r["alpha_max"],
                   None if shp is None else shp[sel])
        out, _, _ = composite_sequential(al, col[sel], r["bg"][:C], r["alpha_min"], r["t_min"])
        imgs.append(out.reshape(H, W, C))
    return torch.stack(imgs)


def render_tiled(g, color_t, n_scenes, H, W, C, r, return_flags=False, only_tiles=None, flag_rel=1e-4):
    """Per-tile lists from the FP32 bin rule, composited with Eq. 8 per pixel.
    `only_tiles` (global tile ids) restricts the work to those tiles; the
    other pixels are left at 0."""
    T = int(r["tile"])
    tx = (W + T - 1) // T
    ty = (H + T - 1) // T
    _, gid, ranges = sorted_pairs(g, H, W, T, r["k_sigma"], r["alpha_min"], n_scenes)
    col = _colors(g, color_t, C)
    N = n_scenes * H * W
    vals, idxs, flags = [], [], []
    wanted = None if only_tiles is None else set(int(x) for x in only_tiles)
    for s in range(n_scenes):
        for t in range(tx * ty):
            gt = s * tx * ty + t
            if wanted is not None and gt not in wanted:
                continue
            x0, y0 = (t % tx) * T, (t // tx) * T
            ys = torch.arange(y0, min(y0 + T, H))
            xs = torch.arange(x0, min(x0 + T, W))
            yy, xx = torch.meshgrid(ys, xs, indexing="ij")
            yy, xx = yy.reshape(-1), xx.reshape(-1)
            lst = torch.as_tensor(gid[ranges[gt, 0]:ranges[gt, 1]], dtype=torch.long)
            shp = g.get("shape")
            al = alpha(xx.to(DT) + 0.5, yy.to(DT) + 0.5, g["mu"][lst], g["sigma"][lst], g["o"][lst],
                       r["alpha_max"], None if shp is None else shp[lst])
            out, _ = composite_cumprod(al, col[lst], r["bg"][:C], r["alpha_min"], r["t_min"])
            vals.append(out)
            idxs.append(s * H * W + yy * W + xx)
            if return_flags:
                flags.append(near_threshold(al, r["alpha_min"], r["t_min"], flag_rel))
    idx = torch.cat(idxs)
    img = torch.zeros(N, C, dtype=DT).index_add(0, idx, torch.cat(vals)).reshape(n_scenes, H, W, C)
    if return_flags:
        fl = torch.zeros(N, dtype=torch.bool)
        fl[idx] = torch.cat(flags)
        return img, fl.reshape(n_scenes, H, W)
    return img
