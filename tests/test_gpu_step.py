"""The whole step on the GPU (sample -> splat -> L2 loss -> backward through
the curves) against the oracle's FP64 values and exact gradients.

Gradients: per tensor ||g_gpu - g_ref|| <= 1e-3 ||g_ref|| and elementwise
|g_gpu - g_ref| <= 1e-3 max|g_ref|.  The end-to-end image tolerance follows
from the record bound of the sampling test: records move by up to
32 eps32 (W + L) px, and an isotropic Gaussian's alpha has slope at most
1/(sigma sqrt(e)) per px, so |dI| <= 32 eps32 (W + L) / sigma_min + 1e-5."""
import math

import numpy as np
import pytest

import scenes
from oracle import pipeline as op

from gpu_util import run_step

pytestmark = pytest.mark.gpu
EPS32 = float(np.finfo(np.float32).eps)

CASES = [
    ("open", lambda: scenes.small_open(51, n_curves=3, size=48, p=(2, 3, 5))),
    ("open-gray", lambda: scenes.small_open(52, n_curves=3, size=40, channels=1)),
    ("closed-strokes", lambda: scenes.small_closed(53, n_curves=3, size=48, filled=False, degrees=(2, 3, 4))),
    ("filled", lambda: scenes.small_closed(54, n_curves=3, size=48, filled=True, h=2.0)),
    # large interiors at h = 1: the sigmoid's slope several px inside must keep its digits (Eq. 7)
    ("filled-deep-h1", lambda: scenes.small_closed(315, n_curves=2, size=56, filled=True, h=1.0)),
    ("filled-h1-batched", lambda: scenes.small_closed(55, n_curves=2, size=40, filled=True, h=1.0, n_scenes=2)),
    ("config1", lambda: scenes.config1().with_raster(**scenes.RASTER_PARITY)),
    # 64 fill Gaussians per sampling block instead of 256
    ("filled-h1-fill-tile-8", lambda: scenes.small_closed(55, n_curves=2, size=40, filled=True, h=1.0, n_scenes=2)
     .with_sample(fill_tile=8)),
]


def _rel_ok(gpu, ref, tol=1e-3):
    gpu = np.asarray(gpu, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    nr = np.linalg.norm(ref)
    if nr == 0:
        return np.abs(gpu).max() <= 1e-9
    return (np.linalg.norm(gpu - ref) <= tol * nr) and (np.abs(gpu - ref).max() <= tol * np.abs(ref).max())


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_step_matches_oracle(name, make):
    sc = make()
    ref = op.loss_and_grads(sc)
    assert all(p.well_separated() for p in ref["plans"])
    out = run_step(sc)
    assert out["report"].status == 0
    Lmax = max(p.length for p in ref["plans"])
    smin = float(np.min(ref["gaussians"]["sigma"])) if ref["gaussians"]["sigma"].size else 1.0
    tol_img = 32 * EPS32 * (max(sc.width, sc.height) + Lmax) / (smin * math.sqrt(math.e)) + 1e-5
    assert np.abs(out["image"] - ref["image"]).max() <= tol_img
    assert abs(out["loss"] - ref["loss"]) <= 1e-4 * ref["loss"] + 1e-7
    assert _rel_ok(out["dcolor"], ref["dcolor"]), "dcolor"
    assert _rel_ok(out["dtau"], ref["dtau"]), "dtau"
    for j, nm in enumerate("xysw"):
        assert _rel_ok(out["dkey"][:, j], ref["dkey"][:, j]), "dkey." + nm


@pytest.mark.parametrize("tile", [8, 32])
def test_step_other_tile_sizes(tile):
    sc = scenes.small_closed(56, n_curves=3, size=48, filled=True, h=2.0).with_raster(tile=tile)
    ref = op.loss_and_grads(sc)
    out = run_step(sc)
    assert out["report"].status == 0
    assert _rel_ok(out["dcolor"], ref["dcolor"]) and _rel_ok(out["dtau"], ref["dtau"])
    for j in range(4):
        assert _rel_ok(out["dkey"][:, j], ref["dkey"][:, j])


def test_autograd_function_matches_oracle():
    """NurbsSplatFunction: torch autograd drives splat_backward; the gradient of
    a torch-side L2 loss matches the oracle's exact gradient."""
    import torch
    from paper_2606_31764_b300.splat import NurbsSplatFunction, Splatter, scene_tensors
    sc = scenes.small_open(57, n_curves=2, size=40)
    ref = op.loss_and_grads(sc)
    sp = Splatter(sc)
    k, t, c = scene_tensors(sc)
    sp.fit(k, t, c)
    k.requires_grad_(True)
    t.requires_grad_(True)
    c.requires_grad_(True)
    img = NurbsSplatFunction.apply(k, t, c, sp)
    tgt = torch.as_tensor(sc.target, device="cuda")
    loss = ((img - tgt) ** 2).mean()
    loss.backward()
    assert abs(loss.item() - ref["loss"]) <= 1e-4 * ref["loss"]
    assert _rel_ok(c.grad.cpu().numpy(), ref["dcolor"])
    assert _rel_ok(t.grad.cpu().numpy(), ref["dtau"])
    dk = k.grad.cpu().numpy().reshape(-1, 4)
    for j in range(4):
        assert _rel_ok(dk[:, j], ref["dkey"][:, j])


def test_empty_scenes_and_empty_batch():
    """A batch whose middle scene has no curves renders that scene as the
    background and gets the other scenes right; a batch with no curves at all
    renders only background and gives empty gradients."""
    import torch
    from paper_2606_31764_b300.splat import Splatter, scene_tensors
    base = scenes.small_closed(58, n_curves=2, size=40, filled=True, h=2.0, n_scenes=3)
    b = scenes._Builder(3, base.height, base.width, base.channels)
    for s in (0, 2):
        for cv in range(base.scene_curve_offset[s], base.scene_curve_offset[s + 1]):
            k0, k1 = base.key_offset[cv], base.key_offset[cv + 1]
            t0, t1 = base.tau_offset[cv], base.tau_offset[cv + 1]
            b.add(s, int(base.degree[cv]), base.key[k0:k1], base.tau[t0:t1], base.color[cv], True, True)
    sc = b.build("gap", base.target, dict(base.sample), dict(base.raster))
    assert sc.scene_curve_offset[1] == sc.scene_curve_offset[2]
    ref = op.loss_and_grads(sc)
    out = run_step(sc)
    assert out["report"].status == 0
    bg = np.asarray(sc.raster["bg"], np.float32)
    assert np.array_equal(out["image"][1], np.broadcast_to(bg, out["image"][1].shape))
    assert np.abs(out["image"] - ref["image"]).max() <= 1e-3
    assert _rel_ok(out["dkey"][:, 0], ref["dkey"][:, 0]) and _rel_ok(out["dcolor"], ref["dcolor"])
    # no curves at all
    e = scenes._Builder(1, 24, 24, 3).build("empty", np.ones((1, 24, 24, 3), np.float32), dict(base.sample),
                                             dict(base.raster))
    sp = Splatter(e)
    k, t, c = (torch.zeros(0, device="cuda"),) * 3
    img = sp.forward(k, t, c)
    torch.cuda.synchronize()
    assert sp.report().status == 0 and int(sp.count.item()) == 0
    assert torch.equal(img, torch.ones_like(img))
