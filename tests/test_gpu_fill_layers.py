"""Fill layers (ns_raster_params.fill_layers = 1): the Gaussians of a filled
curve are binned as one tile pair per tile of the whole grid, and the blend
kernels find the grid points that reach each pixel by index arithmetic.

Every pixel composites the same Gaussians in the same order as with one pair
per Gaussian.  The two paths differ in rounding only: per-Gaussian pairs read
the records' absolute FP32 centres, while fill layers form the offset of a
pixel from a grid point in grid-local coordinates, exact to about 1e-7 px,
take the exponential as a power of 2 with a prescaled coefficient and add a
layer's colour once from its summed weights.
So the fill-layer image is checked against the FP64 oracle at the 1e-5 gate
(outside pixels where a production threshold decision lies within 1e-4 of its
tie), and against the per-Gaussian image within the rounding of the records'
centres, 32 eps32 max(W, H) / (sigma_min sqrt(e)) + 1e-5.  Gradients of the
two paths agree within 1e-4 of their norm, and the whole step is checked
against the oracle (1e-3)."""
import math

import numpy as np
import pytest
import torch

import scenes
from oracle import pipeline as op

from gpu_util import run_scene, run_step

pytestmark = pytest.mark.gpu
EPS32 = float(np.finfo(np.float32).eps)

SCENES = [
    ("filled-h1-production", lambda: scenes.small_closed(331, n_curves=3, size=70, filled=True, h=1.0, height=53)
     .with_raster(**scenes.RASTER_DEFAULTS)),
    ("filled-h2-parity", lambda: scenes.small_closed(332, n_curves=3, size=64, filled=True, h=2.0)),
    ("fills-and-strokes-production", lambda: scenes.small_closed(333, n_curves=4, size=60, filled="alternate",
                                                                 h=1.0).with_raster(**scenes.RASTER_DEFAULTS)),
    ("fills-and-strokes-parity", lambda: scenes.small_closed(334, n_curves=4, size=52, filled="alternate", h=1.5)),
    ("batched-h1", lambda: scenes.small_closed(335, n_curves=3, size=44, filled=True, h=1.0, n_scenes=3)
     .with_raster(**scenes.RASTER_DEFAULTS)),
    ("coarse-grid-h6", lambda: scenes.small_closed(336, n_curves=2, size=72, filled=True, h=6.0)
     .with_raster(**scenes.RASTER_DEFAULTS)),
    ("open-strokes-only", lambda: scenes.small_open(337, n_curves=3, size=48, p=(2, 3, 5))),
]
DECOMP = [(8, 1), (8, 2), (16, 1), (16, 2), (16, 4), (32, 4), (32, 1)]


def _rel(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("name,make", SCENES, ids=[s[0] for s in SCENES])
def test_layers_match_oracle_and_per_gaussian_pairs(name, make):
    sc = make()
    k, t, c = op.leaves(sc, False)
    with torch.no_grad():
        ref, g, flags = op.render(sc, k, t, c, return_flags=True)
    ref = ref.numpy()
    ok = np.broadcast_to(~flags.numpy()[..., None], ref.shape)
    smin = float(g["sigma"].min()) if g["sigma"].numel() else 1.0
    tol_rec = 32 * EPS32 * max(sc.width, sc.height) / (smin * math.sqrt(math.e)) + 1e-5
    for tile, ppt in DECOMP:
        base = run_step(sc.with_raster(tile=tile, ppt_fwd=ppt, ppt_bwd=ppt, fill_layers=0))
        lay = run_step(sc.with_raster(tile=tile, ppt_fwd=ppt, ppt_bwd=ppt, fill_layers=1))
        assert base["report"].status == 0 and lay["report"].status == 0
        assert np.abs(lay["image"] - ref)[ok].max() <= 1e-5, (tile, ppt)
        assert np.abs(lay["image"] - base["image"])[ok].max() <= tol_rec, (tile, ppt)
        nb, nl = base["report"].blend_contribs, lay["report"].blend_contribs
        assert abs(nl - nb) <= 1e-3 * nb + 2, (tile, ppt, nb, nl)
        assert lay["report"].pairs <= base["report"].pairs
        for nm in ("dkey", "dtau", "dcolor"):
            assert _rel(lay[nm], base[nm]) <= 1e-4, (tile, ppt, nm)


@pytest.mark.parametrize("name,make", SCENES[:4], ids=[s[0] for s in SCENES[:4]])
def test_layers_per_gaussian_rows(name, make):
    """Without the chain the adjoint returns every per-Gaussian row."""
    sc = make()
    rows = {}
    for fl in (0, 1):
        s2 = sc.with_raster(tile=8, fill_layers=fl)
        sp, img, rep, (k, t, c), G = run_scene(s2)
        dimg = np.random.default_rng(338).standard_normal(tuple(img.shape)).astype(np.float32)
        sp.backward(k, t, c, torch.as_tensor(dimg, device="cuda"), chain=False)
        torch.cuda.synchronize()
        rows[fl] = sp.dgauss[:G].cpu().numpy().astype(np.float64)
    scale = max(np.abs(rows[0]).max(), 1e-30)
    assert np.abs(rows[1] - rows[0]).max() <= 1e-5 * scale


@pytest.mark.parametrize("tile", [8, 16])
def test_layers_step_matches_oracle(tile):
    sc = scenes.small_closed(321, n_curves=3, size=48, filled=True, h=2.0).with_raster(tile=tile, fill_layers=1)
    ref = op.loss_and_grads(sc)
    assert all(p.well_separated() for p in ref["plans"])
    out = run_step(sc)
    assert out["report"].status == 0
    assert abs(out["loss"] - ref["loss"]) <= 1e-4 * ref["loss"] + 1e-7
    for nm in ("dcolor", "dtau"):
        assert _rel(out[nm], ref[nm]) <= 1e-3, nm
    for j in range(4):
        assert _rel(out["dkey"][:, j], ref["dkey"][:, j]) <= 1e-3


def test_tangent_aligned_sets_keep_per_gaussian_pairs():
    """Tangent-aligned sets are binned per Gaussian whatever fill_layers says."""
    sc = scenes.small_closed(339, n_curves=4, size=52, filled="alternate", h=2.0).with_sample(contour_mode=1)
    a = run_step(sc.with_raster(tile=8, fill_layers=0))
    b = run_step(sc.with_raster(tile=8, fill_layers=1))
    assert np.array_equal(a["image"], b["image"])
    assert a["report"].pairs == b["report"].pairs


def test_layers_need_far_fewer_pairs():
    sc = scenes.small_closed(331, n_curves=3, size=70, filled=True, h=1.0).with_raster(**scenes.RASTER_DEFAULTS)
    a = run_step(sc.with_raster(tile=8, fill_layers=0))
    b = run_step(sc.with_raster(tile=8, fill_layers=1))
    assert b["report"].pairs * 20 < a["report"].pairs


def test_compact_opacity_gradients_match_rows():
    """With fill layers and the per-Gaussian rows left to the workspace, the
    step keeps the fill Gaussians' opacity gradients in one float per Gaussian
    and clears only the contour Gaussians' rows.  The curve gradients equal
    those of the same backward writing every per-Gaussian row (within the
    rounding of atomic sums), and a second call gives them again (nothing of
    the first is left in the workspace)."""
    sc = scenes.small_closed(352, n_curves=4, size=64, filled="alternate", h=1.0).with_raster(
        **dict(scenes.RASTER_DEFAULTS, tile=8, fill_layers=1))
    sp, img, rep, (k, t, c), G = run_scene(sc)
    dimg = torch.as_tensor(np.random.default_rng(353).standard_normal(tuple(img.shape)).astype(np.float32),
                           device="cuda")
    a = [x.cpu().numpy() for x in sp.backward(k, t, c, dimg)]
    b = [x.cpu().numpy() for x in sp.backward(k, t, c, dimg, rows=True)]
    a2 = [x.cpu().numpy() for x in sp.backward(k, t, c, dimg)]
    torch.cuda.synchronize()
    for nm, x, y, z in zip(("dkey", "dtau", "dcolor"), a, b, a2):
        assert np.isfinite(x).all(), nm
        assert _rel(x, y) <= 1e-5, nm
        assert _rel(z, x) <= 1e-5, nm


def _corner_scene(r):
    """A filled circle past the bottom right corner, behind a filled star in
    the middle.  The Gaussians are laid out front to back, so the circle's grid
    comes last in the batch; the canvas clips it, so its last grid points lie
    inside the shape and are live."""
    rng = np.random.default_rng(354)
    H, W = 40, 48
    b = scenes._Builder(1, H, W, 3)
    b.add(0, 2, scenes.circle_keys(W - 3.0, H - 2.0, r), scenes.circle_tau(), (0.9, 0.3, 0.1, 0.85), True, True)
    b.add(0, 3, scenes.star_keys(rng, 18.0, 17.0, 9.0, 9, 1.0, 2.0), rng.uniform(0.5, 1.5, 9),
          (0.2, 0.5, 0.8, 0.9), True, True)
    tgt = scenes.blob_target(rng, 1, H, W, 3, 6)
    return b.build("corner-circle", tgt, dict(scenes.SAMPLE_DEFAULTS, h=1.0),
                   dict(scenes.RASTER_DEFAULTS, tile=8, fill_layers=1))


def test_opacity_gradients_at_the_capacity_end():
    """The adjoint adds a staged region's opacity gradients four consecutive
    Gaussians at a time (one vector reduction); a quad that would run past the
    Gaussian capacity is added point by point instead.  With the capacity
    exactly the Gaussian count, not a multiple of 4, and the batch's last
    Gaussians live, the curve gradients equal those of the backward writing
    every per-Gaussian row (no quads) at the same capacity, and those of a run
    with room to spare."""
    for r in (12.0, 12.5, 13.0, 13.5, 14.0, 14.5, 15.0):
        sc = _corner_scene(r)
        sp, img, rep, (k, t, c), G = run_scene(sc)
        if G % 4:
            break
    else:
        pytest.fail("no corner scene with a Gaussian count that is not a multiple of 4")
    dimg = torch.as_tensor(np.random.default_rng(355).standard_normal(tuple(img.shape)).astype(np.float32),
                           device="cuda")
    room = [x.cpu().numpy() for x in sp.backward(k, t, c, dimg)]
    sp2, img2, rep2, _, G2 = run_scene(sc, capacity=(G, 1 << 16, 1 << 12))
    assert G2 == G and sp2.cap.gaussians == G
    assert np.array_equal(img2.cpu().numpy(), img.cpu().numpy())
    # the circle's last grid point is a live Gaussian: opacity above the cull threshold
    rec = sp2.rec[G - 1].cpu().numpy()
    assert rec[3] >= sc.raster["alpha_min"]
    exact = [x.cpu().numpy() for x in sp2.backward(k, t, c, dimg)]
    rows = [x.cpu().numpy() for x in sp2.backward(k, t, c, dimg, rows=True)]
    torch.cuda.synchronize()
    for nm, x, y, z in zip(("dkey", "dtau", "dcolor"), exact, rows, room):
        assert np.isfinite(x).all(), nm
        assert _rel(x, y) <= 1e-5, nm
        assert _rel(x, z) <= 1e-5, nm
