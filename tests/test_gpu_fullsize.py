"""The large workloads at full size, run exactly as bench.py runs its step
(same Step class, capacities and kernels), checked on samples the oracle can
compute one by one: the plans of sampled curves, their Gaussians, the image
on sampled tiles (rendered by the oracle from the curves that can reach those
tiles) and, for the configuration bench.py times, the gradients of sampled
curves.  Fill points that provably stay below alpha_min carry opacity 0
(fill_cull); they bin to no tile, exactly as their tiny exact opacity would.

The timed configuration (tile 8, fill layers) forms every pixel-to-grid-point
offset in grid-local coordinates from the FP64 grid origin, so its image must
meet the 1e-5 gate against the FP64 oracle: everywhere at the parity
thresholds, and outside pixels whose threshold decision lies within 1e-4 of
its tie at the production thresholds.  Sampled gradients: 1e-3 relative.

The per-Gaussian path (the scene defaults below) reads absolute FP32 centres
from the records: a centre placed by a few FP32 operations at coordinate x
carries up to 32 eps32 (W + L) px (a few ulps of the coordinate and of the
parameter u = a + t(b - a), times |C'|), and an isotropic Gaussian's alpha has
slope at most 1/(sigma sqrt(e)) per px, so the image tolerance there is
32 eps32 (W + L_max) / (sigma_min sqrt(e)) + 1e-5, except at pixels where a
production threshold decision lies within 5 % of its tie (an alpha error of
2e-5 is 0.5 % of alpha_min = 1/255)."""
import math

import numpy as np
import pytest
import torch

import bench
import scenes
from oracle import pipeline as op
from oracle import raster as rs
from oracle import sampling as sm

from gpu_util import plans

pytestmark = pytest.mark.gpu
EPS32 = float(np.finfo(np.float32).eps)

WORKLOADS = [
    ("vectorize-2048-1024", lambda: scenes.config5(), (10_000_000, 20_000_000, 400_000)),
    ("long-spline-512", lambda: scenes.config3(), (3_000_000, 12_000_000, 16)),
    ("batched-64x256", lambda: scenes.config4(), (4_000_000, 8_000_000, 200_000)),
]


def _curve_reach_box(sc, cv, k_sigma):
    """A box that contains every pixel a curve's Gaussians can reach, from the
    key points alone: the curve lies in the convex hull of its control points
    (positive weights), a fill grid lies in the hull's box padded by pad_frac of
    its extent plus one grid step, and a Gaussian reaches k_sigma sigma."""
    sp = sc.sample
    k0, k1 = sc.key_offset[cv], sc.key_offset[cv + 1]
    key = sc.key[k0:k1].astype(np.float64)
    x0, x1, y0, y1 = key[:, 0].min(), key[:, 0].max(), key[:, 1].min(), key[:, 1].max()
    if sc.flags[cv] & scenes.FLAG_FILLED:
        h = sp["h"]
        px = sp["pad_frac"] * (x1 - x0) + h
        py = sp["pad_frac"] * (y1 - y0) + h
        r = k_sigma * sp["eta"] * h / sp["rho"] + 1e-3
        return x0 - px - r, x1 + px + r, y0 - py - r, y1 + py + r
    r = k_sigma * key[:, 2].max() / sp["rho"] + 1e-3
    return x0 - r, x1 + r, y0 - r, y1 + r


@pytest.mark.parametrize("name,make,cap", WORKLOADS, ids=[w[0] for w in WORKLOADS])
def test_fullsize_samples(name, make, cap):
    sc = make()
    step = bench.Step(sc, capacity=cap)
    step()
    torch.cuda.synchronize()
    rep = step.sp.report()
    assert rep.status == 0
    G = step.gaussians()
    f, ii = plans(step.sp, (step.key, step.tau, step.color), sc.n_curves)
    rec = step.sp.rec[:G].cpu().numpy().astype(np.float64)
    img = step.image.cpu().numpy().astype(np.float64)
    k, t, c = op.leaves(sc, False)
    rng = np.random.default_rng(2024)
    sample = rng.choice(sc.n_curves, min(24, sc.n_curves), replace=False)
    all_plans = {}
    skipped = 0
    for cv in sample:
        pl = sm.plan_curve(sc, int(cv), k, t)
        all_plans[int(cv)] = pl
        assert abs(f[cv, 0] - pl.length) <= 1e-5 * pl.length + 1e-3, (cv, f[cv, 0], pl.length)
        if not pl.well_separated():
            skipped += 1                # a count within 1e-3 of a ceil() tie: FP32 may round either way
            continue
        assert ii[cv, 2] == pl.count, (cv, ii[cv, 2], pl.count)
        mu, sig, oj, _ = sm.curve_gaussians(sc, int(cv), k, t, c, pl)
        g0 = ii[cv, 5]
        got = rec[g0:g0 + pl.count]
        tol = 32 * EPS32 * (max(sc.width, sc.height) + pl.length)
        assert np.abs(got[:, :2] - mu.numpy()).max() <= tol
        assert np.abs(got[:, 2] - sig.numpy()).max() <= tol
        tol_o = tol * sc.sample["gamma"] / sc.sample["h"] if pl.kind == "fill" else 1e-7
        go, ro = got[:, 3], oj.numpy()
        # fill points proven to stay below alpha_min are written with opacity 0
        # (they bin to no tile either way); every other record matches
        amin = sc.raster["alpha_min"]
        culled = (go == 0.0) & (ro < amin)
        assert np.all(ro[go == 0.0] < amin + tol_o)
        assert np.abs(go - ro)[~culled].max(initial=0.0) <= tol_o
    # the seeded sample holds at most a few curves with a count near a tie
    assert skipped <= len(sample) // 6, (skipped, len(sample))

    # image on sampled tiles of sampled scenes
    T = 16
    tx, ty = (sc.width + T - 1) // T, (sc.height + T - 1) // T
    cs = sc.curve_scene()
    for s in rng.choice(sc.n_scenes, min(2, sc.n_scenes), replace=False):
        tiles = rng.choice(tx * ty, 3, replace=False)
        curves = []
        c0, c1 = sc.scene_curve_offset[s], sc.scene_curve_offset[s + 1]
        for cv in range(c0, c1):
            x0, x1, y0, y1 = _curve_reach_box(sc, cv, sc.raster["k_sigma"])
            for tt in tiles:
                bx, by = (tt % tx) * T, (tt // tx) * T
                if x1 >= bx and x0 <= bx + T and y1 >= by and y0 <= by + T:
                    curves.append(cv)
                    if cv not in all_plans:
                        all_plans[cv] = sm.plan_curve(sc, cv, k, t)
                    break
        if not curves:
            continue
        sub = sc.subset([int(s)])
        # keep only the selected curves (same relative order, so the same depth order)
        keep = [cv - c0 for cv in curves]
        sub = _keep_curves(sub, keep)
        sub_plans = [all_plans[cv] for cv in curves]
        with torch.no_grad():
            kk, tt_, cc = op.leaves(sub, False)
            g = sm.sample_scene(sub, kk, tt_, cc, sub_plans)
            ref, flags = rs.render_tiled(g, cc, 1, sub.height, sub.width, sub.channels, sub.raster,
                                         return_flags=True, only_tiles=tiles, flag_rel=0.05)
        ref = ref.numpy()[0]
        flags = flags.numpy()[0]
        Lmax = max(p.length for p in sub_plans)
        smin = float(g["sigma"].min())
        tol = 32 * EPS32 * (max(sc.width, sc.height) + Lmax) / (smin * math.sqrt(math.e)) + 1e-5
        for tt in tiles:
            bx, by = (tt % tx) * T, (tt // tx) * T
            a = img[s, by:by + T, bx:bx + T]
            b = ref[by:by + T, bx:bx + T]
            ok = ~flags[by:by + T, bx:bx + T]
            if ok.any():
                assert np.abs(a - b)[ok].max() <= tol, (name, s, tt, np.abs(a - b)[ok].max(), tol)


def _tiles_reached(sc, boxes, s, tiles, T):
    """Curves of scene s whose reach boxes meet one of the tiles (edge T)."""
    tx = (sc.width + T - 1) // T
    out = []
    for cv in range(sc.scene_curve_offset[s], sc.scene_curve_offset[s + 1]):
        x0, x1, y0, y1 = boxes[cv]
        for tt in tiles:
            bx, by = (tt % tx) * T, (tt // tx) * T
            if x1 >= bx and x0 <= bx + T and y1 >= by and y0 <= by + T:
                out.append(cv)
                break
    return out


def _oracle_tiles(sc, curves, plans, tiles, flag_rel):
    """Oracle image and threshold flags of the listed curves on the tiles."""
    sub = _keep_curves(sc.subset([0]), curves)
    with torch.no_grad():
        kk, tt, cc = op.leaves(sub, False)
        g = sm.sample_scene(sub, kk, tt, cc, [plans[cv] for cv in curves])
        ref, flags = rs.render_tiled(g, cc, 1, sub.height, sub.width, sub.channels, sub.raster,
                                     return_flags=True, only_tiles=tiles, flag_rel=flag_rel)
    return ref.numpy()[0], flags.numpy()[0]


TIMED = dict(tile=8, fill_layers=1)   # the configuration bench.py's autotuner keeps


@pytest.mark.parametrize("ppt", [1, 2])
def test_fullsize_timed_config_image(ppt):
    """1024x1024 vectorisation workload, tile 8 with fill layers: the image on
    sampled tiles within 1e-5 of the oracle at both threshold settings."""
    base = scenes.config5()
    k, t, _ = op.leaves(base, False)
    rng = np.random.default_rng(2025 + ppt)
    T = TIMED["tile"]   # tile ids in the numbering of the oracle's tiled render
    tx, ty = (base.width + T - 1) // T, (base.height + T - 1) // T
    boxes = [_curve_reach_box(base, cv, scenes.RASTER_PARITY["k_sigma"]) for cv in range(base.n_curves)]
    plans_cache = {}
    for thr, raster, flag_rel in (("parity", scenes.RASTER_PARITY, None),
                                  ("production", scenes.RASTER_DEFAULTS, 1e-4)):
        sc = base.with_raster(**dict(raster, **TIMED, ppt_fwd=ppt, ppt_bwd=ppt))
        step = bench.Step(sc, capacity=(10_000_000, 20_000_000, 400_000), raster=sc.raster)
        step()
        torch.cuda.synchronize()
        assert step.sp.report().status == 0
        img = step.image.cpu().numpy().astype(np.float64)[0]
        # tiles reached only by curves whose counts are clear of a ceil() tie
        tiles = []
        for tt in rng.permutation(tx * ty):
            reach = _tiles_reached(base, boxes, 0, [tt], T)
            for cv in reach:
                if cv not in plans_cache:
                    plans_cache[cv] = sm.plan_curve(base, cv, k, t)
            if all(plans_cache[cv].well_separated(sign_bar_px=0.0) for cv in reach):
                tiles.append(int(tt))
            if len(tiles) == 12:
                break
        curves = _tiles_reached(base, boxes, 0, tiles, T)
        ref, flags = _oracle_tiles(sc, curves, plans_cache, tiles, flag_rel or 1e-4)
        for tt in tiles:
            bx, by = (tt % tx) * T, (tt // tx) * T
            d = np.abs(img[by:by + T, bx:bx + T] - ref[by:by + T, bx:bx + T])
            ok = np.ones(d.shape[:2], bool) if flag_rel is None else ~flags[by:by + T, bx:bx + T]
            assert d[ok].max(initial=0.0) <= 1e-5, (thr, int(tt), float(d[ok].max(initial=0.0)))


def test_fullsize_timed_config_gradients():
    """The gradients of sampled curves of the 1024x1024 workload, as the timed
    step computes them (tile 8, fill layers, production thresholds), against
    the oracle's exact gradient of the same loss.  A curve's parameters only
    move pixels inside its reach box, and only curves whose reach boxes meet
    that box touch those pixels; so the oracle renders that neighbourhood on
    the tiles covering the box, and the loss over those pixels (normalised by
    the whole image's size) has the same gradient with respect to the curve."""
    sc = scenes.config5().with_raster(**TIMED)
    step = bench.Step(sc, capacity=(10_000_000, 20_000_000, 400_000), raster=sc.raster)
    step()
    torch.cuda.synchronize()
    assert step.sp.report().status == 0
    dk, dt, dc = (g.cpu().numpy().astype(np.float64) for g in step.grads)
    dk = dk.reshape(-1, 4)
    dc = dc.reshape(-1, 4)
    k, t, _ = op.leaves(sc, False)
    T = int(sc.raster["tile"])
    tx, ty = (sc.width + T - 1) // T, (sc.height + T - 1) // T
    boxes = [_curve_reach_box(sc, cv, sc.raster["k_sigma"]) for cv in range(sc.n_curves)]
    rng = np.random.default_rng(2026)
    sample = [int(c) for c in rng.choice(sc.n_curves, 16, replace=False)]
    got, want = {"dkey": [], "dtau": [], "dcolor": []}, {"dkey": [], "dtau": [], "dcolor": []}
    used = 0
    n_total = sc.n_scenes * sc.height * sc.width * sc.channels
    for cv in sample:
        x0, x1, y0, y1 = boxes[cv]
        nb = [c for c in range(sc.n_curves)
              if boxes[c][1] >= x0 and boxes[c][0] <= x1 and boxes[c][3] >= y0 and boxes[c][2] <= y1]
        plans = [sm.plan_curve(sc, c, k, t) for c in nb]
        if not all(p.well_separated() for p in plans):   # counts near a ceil() tie
            continue
        ix0, ix1 = max(0, int(x0) // T), min(tx - 1, int(x1) // T)
        iy0, iy1 = max(0, int(y0) // T), min(ty - 1, int(y1) // T)
        tiles = [yy * tx + xx for yy in range(iy0, iy1 + 1) for xx in range(ix0, ix1 + 1)]
        sub = _keep_curves(sc.subset([0]), nb)
        kk, tt_, cc = op.leaves(sub, True)
        g = sm.sample_scene(sub, kk, tt_, cc, plans)
        # a grid point of this curve within 1e-4 px of its polyline (a winding
        # sign FP32 may take either way; the neighbours' signs leave sdf ~ 0)
        if not plans[nb.index(cv)].well_separated():
            continue
        img = rs.render_tiled(g, cc, 1, sub.height, sub.width, sub.channels, sub.raster, only_tiles=tiles)
        mask = torch.zeros(1, sub.height, sub.width, 1, dtype=torch.float64)
        for tl in tiles:
            bx, by = (tl % tx) * T, (tl // tx) * T
            mask[0, by:by + T, bx:bx + T] = 1.0
        tgt = torch.as_tensor(sub.target, dtype=torch.float64)
        loss = (((img - tgt) ** 2) * mask).sum() / n_total
        loss.backward()
        j = nb.index(cv)
        k0, k1 = sub.key_offset[j], sub.key_offset[j + 1]
        t0, t1 = sub.tau_offset[j], sub.tau_offset[j + 1]
        K0, K1 = sc.key_offset[cv], sc.key_offset[cv + 1]
        T0, T1 = sc.tau_offset[cv], sc.tau_offset[cv + 1]
        want["dkey"].append(kk.grad.numpy()[k0:k1].reshape(-1))
        want["dtau"].append(tt_.grad.numpy()[t0:t1])
        want["dcolor"].append(cc.grad.numpy()[j])
        got["dkey"].append(dk[K0:K1].reshape(-1))
        got["dtau"].append(dt[T0:T1])
        got["dcolor"].append(dc[cv])
        used += 1
    assert used >= 10, used
    for nm in ("dkey", "dtau", "dcolor"):
        a, b = np.concatenate(got[nm]), np.concatenate(want[nm])
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b), (nm, np.linalg.norm(a - b) / np.linalg.norm(b))


def _keep_curves(sc, keep):
    b = scenes._Builder(1, sc.height, sc.width, sc.channels)
    for cv in keep:
        k0, k1 = sc.key_offset[cv], sc.key_offset[cv + 1]
        t0, t1 = sc.tau_offset[cv], sc.tau_offset[cv + 1]
        b.add(0, int(sc.degree[cv]), sc.key[k0:k1], sc.tau[t0:t1], sc.color[cv],
              bool(sc.flags[cv] & scenes.FLAG_CLOSED), bool(sc.flags[cv] & scenes.FLAG_FILLED))
    return b.build(sc.name, sc.target, dict(sc.sample), dict(sc.raster))
