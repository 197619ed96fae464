"""The lane-group blend decomposition (each warp split into four 8-lane groups
of two pixel columns, each walking its own hits) against the whole-warp
kernels and the oracle.

Every pixel composites the same tile list in the same order whatever the
decomposition, so the image must be bit-identical to the whole-warp kernels'.
The per-Gaussian adjoint differs only in the order of its float atomics:
within 1e-5 of the largest entry.  The whole step through the curves is
checked against the oracle's exact gradients (1e-3 relative), at production
thresholds too, where the groups cull different entries."""
import numpy as np
import pytest
import torch

import scenes
from oracle import pipeline as op
from paper_2606_31764_b300 import binding as B

from gpu_util import run_records, run_step

pytestmark = pytest.mark.gpu
GRP = B.BLEND_LANE_GROUPS

SCENES = [
    ("filled-h1-production", lambda: scenes.small_closed(301, n_curves=3, size=70, filled=True, h=1.0, height=53)
     .with_raster(**scenes.RASTER_DEFAULTS), False),
    ("filled-h2-parity", lambda: scenes.small_closed(302, n_curves=3, size=70, filled=True, h=2.0, height=53),
     False),
    ("open-production", lambda: scenes.small_open(303, n_curves=4, size=61, p=(2, 3, 5))
     .with_raster(**scenes.RASTER_DEFAULTS), False),
    ("closed-strokes", lambda: scenes.small_closed(304, n_curves=3, size=45, filled=False, degrees=(2, 3, 4))
     .with_raster(**scenes.RASTER_DEFAULTS), False),
    ("open-gray", lambda: scenes.small_open(307, n_curves=3, size=45, channels=1)
     .with_raster(**scenes.RASTER_DEFAULTS), False),
    ("tangent-aligned", lambda: scenes.small_open(305, n_curves=3, size=48, p=(2, 3, 5), delta_c=0.8)
     .with_sample(contour_mode=1).with_raster(**scenes.RASTER_DEFAULTS), True),
]
DECOMP = [(8, 1), (8, 2), (16, 1), (16, 2), (32, 1), (32, 2)]


def _splat(sc, g, tile, pf, pb, dimg):
    sc = sc.with_raster(tile=tile, ppt_fwd=pf, ppt_bwd=pb)
    G = g["rec"].shape[0]
    sp, img, rep, (k, t, c) = run_records(sc, g["rec"], g["curve"], shape=g.get("shape"))
    assert rep.status == 0
    sp.backward(k, t, c, torch.as_tensor(dimg, device="cuda"), chain=False)
    torch.cuda.synchronize()
    return img.cpu().numpy(), sp.dgauss[:G].cpu().numpy().astype(np.float64), rep


@pytest.mark.parametrize("name,make,aniso", SCENES, ids=[s[0] for s in SCENES])
def test_groups_match_whole_warp(name, make, aniso):
    sc = make()
    g = op.gaussians_fp32(sc)
    if not aniso:
        g.pop("shape", None)
    assert g["rec"].shape[0] > 0
    dimg = np.random.default_rng(306).standard_normal(
        (sc.n_scenes, sc.height, sc.width, sc.channels)).astype(np.float32)
    for tile, ppt in DECOMP:
        img0, rows0, rep0 = _splat(sc, g, tile, ppt, ppt, dimg)
        img1, rows1, rep1 = _splat(sc, g, tile, ppt | GRP, ppt | GRP, dimg)
        assert np.array_equal(img0, img1), (tile, ppt)
        assert rep1.blend_contribs == rep0.blend_contribs
        assert rep1.blend_evals <= rep0.blend_evals
        scale = max(np.abs(rows0).max(), 1e-30)
        assert np.abs(rows1 - rows0).max() <= 1e-5 * scale, (tile, ppt)


def _rel_ok(gpu, ref, tol=1e-3):
    gpu = np.asarray(gpu, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    nr = np.linalg.norm(ref)
    if nr == 0:
        return np.abs(gpu).max() <= 1e-9
    return (np.linalg.norm(gpu - ref) <= tol * nr) and (np.abs(gpu - ref).max() <= tol * np.abs(ref).max())


STEPS = [
    ("filled", lambda: scenes.small_closed(321, n_curves=3, size=48, filled=True, h=2.0)),
    ("open", lambda: scenes.small_open(312, n_curves=3, size=48, p=(2, 3, 5))),
    ("filled-h1-batched", lambda: scenes.small_closed(55, n_curves=2, size=40, filled=True, h=1.0, n_scenes=2)),
    ("fills-and-strokes", lambda: scenes.small_closed(322, n_curves=4, size=52, filled="alternate", h=1.0)),
    ("tangent-aligned-mixed", lambda: scenes.small_closed(323, n_curves=4, size=52, filled="alternate", h=2.0)
     .with_sample(contour_mode=1, delta_c=0.8)),
]


@pytest.mark.parametrize("name,make", STEPS, ids=[s[0] for s in STEPS])
@pytest.mark.parametrize("tile,ppt", [(8, 1), (16, 2)])
def test_step_with_groups_matches_oracle(name, make, tile, ppt):
    sc = make().with_raster(tile=tile, ppt_fwd=ppt | GRP, ppt_bwd=ppt | GRP)
    ref = op.loss_and_grads(sc)
    assert all(p.well_separated() for p in ref["plans"])
    out = run_step(sc)
    assert out["report"].status == 0
    base = run_step(sc.with_raster(ppt_fwd=ppt, ppt_bwd=ppt))
    assert np.array_equal(out["image"], base["image"])
    # against the whole-warp kernels: only the order of the float atomics differs
    for nm in ("dkey", "dtau", "dcolor"):
        a = np.asarray(out[nm], np.float64)
        b = np.asarray(base[nm], np.float64)
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b) + 1e-12, nm
    assert abs(out["loss"] - ref["loss"]) <= 1e-4 * ref["loss"] + 1e-7
    assert _rel_ok(out["dcolor"], ref["dcolor"]), "dcolor"
    assert _rel_ok(out["dtau"], ref["dtau"]), "dtau"
    for j, nm in enumerate("xysw"):
        assert _rel_ok(out["dkey"][:, j], ref["dkey"][:, j]), "dkey." + nm


def test_invalid_group_decompositions_are_rejected():
    sc = scenes.small_closed(314, n_curves=2, size=40, filled=True, h=2.0)
    g = op.gaussians_fp32(sc)
    for bad in (4 | GRP, 3 | GRP, 32):
        with pytest.raises(B.NsError):
            run_records(sc.with_raster(tile=16, ppt_fwd=bad), g["rec"], g["curve"])
