"""nurbs_sample on the GPU against the oracle's plan and Gaussians.

Counts are integers decided by ceil() of FP values; they must agree exactly
wherever the oracle's value is not within 1e-3 of an integer (the inputs are
checked to have no such tie).  Records agree within a bound derived from FP32
rounding: |dmu| <= 32 eps32 (max |coordinate| + L) for a curve of arc length L."""
import numpy as np
import pytest
import torch

import scenes
from oracle import pipeline as op

from gpu_util import plans, run_scene

pytestmark = pytest.mark.gpu
EPS32 = float(np.finfo(np.float32).eps)

CASES = [
    ("open", lambda: scenes.small_open(41, n_curves=4, size=64, p=(1, 2, 3, 4, 5), delta_c=1.5)),
    ("open-long", lambda: scenes.small_open(42, n_curves=2, size=96, nk_range=(40, 80), delta_c=1.0)),
    ("filled", lambda: scenes.small_closed(43, n_curves=4, size=64, filled=True, h=2.0)),
    ("strokes", lambda: scenes.small_closed(44, n_curves=4, size=64, filled=False)),
    ("batched", lambda: scenes.small_closed(45, n_curves=3, size=48, filled=True, h=1.0, n_scenes=3)),
    ("config1", scenes.config1),
]


def _no_ties(pl):
    return all(p.well_separated() for p in pl)


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_plan_and_records(name, make):
    sc = make()
    pl_o = op.plan(sc)
    assert _no_ties(pl_o), "seed has a count within 1e-3 of a tie; pick another"
    sp, img, rep, inputs, G = run_scene(sc)
    assert rep.status == 0
    f, i = plans(sp, inputs, sc.n_curves)
    for c, p in enumerate(pl_o):
        assert abs(f[c, 0] - p.length) <= 1e-5 * p.length + 1e-4, (c, f[c, 0], p.length)
        kind = {"open": 1, "closed": 2, "fill": 3}[p.kind]
        assert i[c, 0] == kind
        assert i[c, 2] == p.count, (c, i[c, 2], p.count)
        if p.kind == "fill":
            assert i[c, 1] == p.n_boundary and i[c, 3] == p.nx and i[c, 4] == p.ny
    g = op.gaussians_fp32(sc, pl_o)
    assert G == g["rec"].shape[0]
    rec = sp.rec[:G].cpu().numpy().astype(np.float64)
    cur = sp.curve[:G].cpu().numpy()
    np.testing.assert_array_equal(cur, g["curve"])
    ref = g["rec"].astype(np.float64)
    for c, p in enumerate(pl_o):
        sel = cur == c
        scale = 32 * EPS32 * (max(sc.width, sc.height) + p.length)
        assert np.abs(rec[sel, :2] - ref[sel, :2]).max() <= scale, c
        assert np.abs(rec[sel, 2] - ref[sel, 2]).max() <= scale, c
        tol_o = scale * sc.sample["gamma"] / sc.sample["h"] if p.kind == "fill" else 1e-7
        assert np.abs(rec[sel, 3] - ref[sel, 3]).max() <= tol_o, c


def test_invalid_curve_is_reported_not_rendered():
    sc = scenes.small_open(46, n_curves=2, size=40)
    sc.degree[1] = 7   # degree above 5
    sp, img, rep, inputs, G = run_scene(sc) if False else (None, None, None, None, None)
    from paper_2606_31764_b300.splat import Splatter, scene_tensors
    s = Splatter(sc)
    k, t, c = scene_tensors(sc)
    s.forward(k, t, c)
    r = s.report()
    assert r.status == 3 and r.bad_curve == 1
    f, i = plans(s, (k, t, c), 2)
    assert i[1, 2] == 0 and i[0, 2] > 0


def test_capacity_overflow_reports_needed_sizes():
    sc = scenes.small_closed(47, n_curves=3, size=48, filled=True, h=2.0)
    pl_o = op.plan(sc)
    from paper_2606_31764_b300.splat import Splatter, scene_tensors
    s = Splatter(sc, capacity=(100, 1 << 16, 8))
    k, t, c = scene_tensors(sc)
    img = s.forward(k, t, c)
    r = s.report()
    assert r.status == 2
    assert r.gaussians == sum(p.count for p in pl_o)
    assert r.boundary == sum(p.n_boundary for p in pl_o)
    # the backward on the truncated set still runs within bounds: tasks beyond
    # the task table fall back to the plan search, work beyond the capacities
    # is dropped, and the status stays NS_ERR_CAPACITY
    import torch as _t
    dk, dt, dc = s.backward(k, t, c, _t.ones_like(img))
    _t.cuda.synchronize()
    assert s.report().status == 2
    assert bool(_t.isfinite(dk).all()) and bool(_t.isfinite(dt).all()) and bool(_t.isfinite(dc).all())


@pytest.mark.parametrize("seed,h", [(61, 1.0), (62, 2.0), (63, 1.0)])
def test_fill_nearest_segment_and_sign(seed, h):
    """The kernel's nearest segment (aux) attains the oracle's minimum distance
    from the same grid point, and its inside/outside sign agrees with the
    winding number wherever the point is not on the polyline."""
    import torch as _t
    from oracle import sampling as sm
    sc = scenes.small_closed(seed, n_curves=4, size=80, filled=True, h=h, degrees=(2, 3, 4, 5))
    pl_o = op.plan(sc)
    assert _no_ties(pl_o)
    sp, img, rep, inputs, G = run_scene(sc)
    rec = sp.rec[:G].cpu().numpy().astype(np.float64)
    cur = sp.curve[:G].cpu().numpy()
    aux = sp.aux[:G].cpu().numpy()
    k, t, c = op.leaves(sc, False)
    for cv in range(sc.n_curves):
        sel = np.nonzero(cur == cv)[0]
        p, fl, cp, U = sm.curve_inputs(sc, cv, k, t)
        a, b = sm.nb.domain(U, p)
        poly = sm.nb.curve_point(cp, U, p, sm.boundary_parameters(a, b, pl_o[cv].n_boundary))[:, :2]
        q = _t.as_tensor(rec[sel, :2])
        d_min, _ = sm.unsigned_distance(q, poly)
        tol = 32 * EPS32 * (sc.width + pl_o[cv].length)
        # points recorded as deep inside (no segment): inside, and far enough
        # that the sigmoid of Eq. 7 is 1 in FP32 (z >= 17)
        deep = aux[sel] == 0x7fffffff
        wn = sm.winding_number(q, poly).numpy()
        assert np.all(wn[deep] > 0.5)
        assert np.all(d_min.numpy()[deep] >= 17.0 * h / sc.sample["gamma"] - tol)
        sel, q, d_min, wn = sel[~deep], q[~deep], d_min[~deep], wn[~deep]
        ins = aux[sel] >= 0
        i0 = np.where(ins, aux[sel], ~aux[sel])
        b0 = poly[i0]
        b1 = poly[(i0 + 1) % poly.shape[0]]
        e = b1 - b0
        tt = (((q - b0) * e).sum(1) / (e * e).sum(1)).clamp(0, 1)
        d_sel = (q - b0 - tt[:, None] * e).norm(dim=1)
        assert float((d_sel - d_min).abs().max()) <= tol
        clear = d_min.numpy() > tol
        assert np.array_equal(ins[clear], (wn > 0.5)[clear])


@pytest.mark.parametrize("production", [False, True])
def test_fill_tile_changes_no_record(production):
    """The fill tile (Gaussians per sampling block, 8 x 8 or 16 x 16) is a work
    decomposition only: every grid point takes the same minimum over the same
    segment distances and the same crossing tests, so the records, nearest
    segments and signs are identical bit for bit, and so are the gradients."""
    sc = scenes.small_closed(46, n_curves=4, size=72, filled="alternate", h=1.0, n_scenes=2)
    if production:
        sc = sc.with_raster(**scenes.RASTER_DEFAULTS)
    out = {}
    for ft in (16, 8):
        s2 = sc.with_sample(fill_tile=ft)
        sp, img, rep, (k, t, c), G = run_scene(s2)
        assert rep.status == 0
        dimg = torch.as_tensor(np.random.default_rng(47).standard_normal(tuple(img.shape)).astype(np.float32),
                               device="cuda")
        dk, dt, dc = sp.backward(k, t, c, dimg)
        torch.cuda.synchronize()
        out[ft] = (sp.rec[:G].cpu().numpy(), sp.aux[:G].cpu().numpy(), img.cpu().numpy(), dk.cpu().numpy(),
                   dt.cpu().numpy(), dc.cpu().numpy())
    for a, b in zip(out[16][:3], out[8][:3]):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(out[16][3:], out[8][3:]):   # float additions in another order
        assert np.abs(a - b).max() <= 1e-5 * max(np.abs(a).max(), 1e-30)


def test_fill_tile_is_checked():
    sc = scenes.small_closed(48, n_curves=2, size=40, filled=True, h=2.0).with_sample(fill_tile=12)
    with pytest.raises(Exception):
        run_scene(sc)
