"""The three large workloads at full size, run exactly as bench.py runs its
step (same Step class, capacities and kernels), checked on samples the oracle
can compute one by one: the plans of sampled curves, their Gaussians, and the
image on sampled tiles (rendered by the oracle from the curves that can reach
those tiles).  Fill points that provably stay below alpha_min carry opacity 0
(fill_cull); they bin to no tile, exactly as their tiny exact opacity would.

Tolerances: records within 32 eps32 (W + L) px (FP32 parameter placement and
evaluation); image within 32 eps32 (W + L_max) / (sigma_min sqrt(e)) + 1e-5,
except at pixels where a production threshold decision (alpha near alpha_min,
transmittance near t_min) lies within 5 % of its tie, where FP32 records may
legitimately decide the other way."""
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
    for cv in sample:
        pl = sm.plan_curve(sc, int(cv), k, t)
        all_plans[int(cv)] = pl
        assert abs(f[cv, 0] - pl.length) <= 1e-5 * pl.length + 1e-3, (cv, f[cv, 0], pl.length)
        if not pl.well_separated():
            continue                    # a count within 1e-3 of a ceil() tie: FP32 may round either way
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


def _keep_curves(sc, keep):
    b = scenes._Builder(1, sc.height, sc.width, sc.channels)
    for cv in keep:
        k0, k1 = sc.key_offset[cv], sc.key_offset[cv + 1]
        t0, t1 = sc.tau_offset[cv], sc.tau_offset[cv + 1]
        b.add(0, int(sc.degree[cv]), sc.key[k0:k1], sc.tau[t0:t1], sc.color[cv],
              bool(sc.flags[cv] & scenes.FLAG_CLOSED), bool(sc.flags[cv] & scenes.FLAG_FILLED))
    return b.build(sc.name, sc.target, dict(sc.sample), dict(sc.raster))
