"""The tangent-aligned (anisotropic) contour variant on the GPU against the
oracle: records and shapes, bins and sort order bit for bit from the same FP32
set, the image within 1e-5, the blend adjoint per record, and the whole step's
gradients within 1e-3."""
import math

import numpy as np
import pytest
import torch

import scenes
from oracle import pipeline as op

from gpu_util import run_records, run_step, run_scene, sorted_pairs, tile_ranges

pytestmark = pytest.mark.gpu
EPS32 = float(np.finfo(np.float32).eps)


def _aniso(sc):
    return sc.with_sample(contour_mode=1)


CASES = [
    ("open", lambda: _aniso(scenes.small_open(211, n_curves=3, size=48, p=(2, 3, 5), delta_c=0.8))),
    ("closed-strokes", lambda: _aniso(scenes.small_closed(212, n_curves=3, size=48, filled=False,
                                                          degrees=(2, 3, 4)).with_sample(delta_c=0.8))),
    ("mixed-with-fill", lambda: _aniso(scenes.small_closed(213, n_curves=2, size=44, filled=True, h=2.0))),
    ("open-gray", lambda: _aniso(scenes.small_open(214, n_curves=3, size=40, channels=1, delta_c=0.6))),
]


def _rel_ok(gpu, ref, tol=1e-3, floor=0.0):
    """Per tensor within tol of the reference in norm and elementwise against
    its largest entry; `floor` is an absolute scale below which a reference
    counts as zero (FP64 rounding noise of an exactly vanishing gradient)."""
    gpu = np.asarray(gpu, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    nr = np.linalg.norm(ref)
    if nr <= floor:
        return np.abs(gpu).max() <= max(1e-9, tol * floor)
    return (np.linalg.norm(gpu - ref) <= tol * nr) and (np.abs(gpu - ref).max() <= tol * np.abs(ref).max())


@pytest.mark.parametrize("name,make", CASES[:2], ids=[c[0] for c in CASES[:2]])
def test_records_and_shapes_match_oracle(name, make):
    sc = make()
    ref = op.gaussians_fp32(sc)
    sp, img, rep, inputs, G = run_scene(sc)
    assert rep.status == 0 and G == ref["rec"].shape[0]
    rec = sp.rec[:G].cpu().numpy()
    shp = sp.shape[:G].cpu().numpy()
    Lmax = max(p.length for p in ref["plans"])
    tol = 32 * EPS32 * (max(sc.width, sc.height) + Lmax)
    assert np.abs(rec[:, :2] - ref["rec"][:, :2]).max() <= tol
    assert np.abs(rec[:, 2:] - ref["rec"][:, 2:]).max() <= 1e-5
    assert np.allclose(shp[:, 0], ref["shape"][:, 0], rtol=1e-4, atol=1e-5)
    assert np.abs(shp[:, 1:3] - ref["shape"][:, 1:3]).max() <= 1e-4


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_bins_image_and_adjoint_from_the_same_records(name, make):
    sc = make()
    g = op.gaussians_fp32(sc)
    G = g["rec"].shape[0]
    sp, img, rep, inputs = run_records(sc, g["rec"], g["curve"], shape=g["shape"])
    assert rep.status == 0
    tid_o, gid_o, ranges_o = op.pairs_records(sc, g["rec"], g["curve"], shape=g["shape"])
    tid, gid = sorted_pairs(sp, inputs, tid_o.shape[0])
    assert np.array_equal(tid, tid_o) and np.array_equal(gid, gid_o)
    assert np.array_equal(tile_ranges(sp, inputs, ranges_o.shape[0]), ranges_o)
    ref = op.render_records(sc, g["rec"], g["curve"], shape=g["shape"])
    assert np.abs(img.cpu().numpy() - ref).max() <= 1e-5
    # blend adjoint per record: rows {dmu_x, dmu_y, dA, dB2, do, dr, dg, db, dC}
    rng = np.random.default_rng(215)
    dimg = rng.standard_normal(ref.shape).astype(np.float32)
    k, t, c = inputs
    sp.backward(k, t, c, torch.as_tensor(dimg, device="cuda"), chain=False)
    torch.cuda.synchronize()
    rows = sp.dgauss[:G].cpu().numpy().astype(np.float64)
    drec, dcol, dshape = op.record_grads(sc, g["rec"], g["curve"], dimg, shape=g["shape"])
    st, cs, sn = (g["shape"][:, j].astype(np.float64) for j in range(3))
    sg = g["rec"][:, 2].astype(np.float64)
    dA, dB2, dC = rows[:, 2], rows[:, 3], rows[:, 8]
    # exponent conic A = -(c^2/st^2 + s^2/sg^2)/2, B2 = -c s (1/st^2 - 1/sg^2), C = -(s^2/st^2 + c^2/sg^2)/2
    it, inn = 1 / st ** 2, 1 / sg ** 2
    d_st = (dA * cs ** 2 + 2 * dB2 * cs * sn + dC * sn ** 2) / st ** 3
    d_sg = (dA * sn ** 2 - 2 * dB2 * cs * sn + dC * cs ** 2) / sg ** 3
    d_c = -dA * cs * it - dB2 * sn * (it - inn) - dC * cs * inn
    d_s = -dA * sn * inn - dB2 * cs * (it - inn) - dC * sn * it
    assert _rel_ok(rows[:, 0], drec[:, 0]) and _rel_ok(rows[:, 1], drec[:, 1])
    assert _rel_ok(rows[:, 4], drec[:, 3])
    assert _rel_ok(d_st, dshape[:, 0]) and _rel_ok(d_sg, drec[:, 2])
    # all-isotropic sets (fills) have exactly vanishing tangent gradients
    floor = 1e-9 * max(np.abs(drec[:, :2]).max(), 1e-30)
    assert _rel_ok(d_c, dshape[:, 1], floor=floor) and _rel_ok(d_s, dshape[:, 2], floor=floor)


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_step_matches_oracle(name, make):
    sc = make()
    ref = op.loss_and_grads(sc)
    assert all(p.well_separated() for p in ref["plans"])
    out = run_step(sc)
    assert out["report"].status == 0
    Lmax = max(p.length for p in ref["plans"])
    smin = float(np.min(ref["gaussians"]["sigma"]))
    tol_img = 32 * EPS32 * (max(sc.width, sc.height) + Lmax) / (smin * math.sqrt(math.e)) + 1e-5
    assert np.abs(out["image"] - ref["image"]).max() <= 4 * tol_img
    assert abs(out["loss"] - ref["loss"]) <= 1e-4 * ref["loss"] + 1e-7
    assert _rel_ok(out["dcolor"], ref["dcolor"]), "dcolor"
    assert _rel_ok(out["dtau"], ref["dtau"]), "dtau"
    for j, nm in enumerate("xysw"):
        assert _rel_ok(out["dkey"][:, j], ref["dkey"][:, j]), "dkey." + nm
