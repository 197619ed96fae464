"""Frozen-parameter variants of the backward (the paper's "w/o weights",
"w/o knots", "w/o w & k" rows of Table 1): the remaining gradients match the
oracle's exact gradients, the frozen ones are not formed, and Adam leaves the
frozen parameters where they started."""
import numpy as np
import pytest
import torch

import scenes
from oracle import geometry as og
from oracle import pipeline as op
from paper_2606_31764_b300.splat import Splatter, scene_tensors

from gpu_util import run_scene

pytestmark = pytest.mark.gpu

CASES = [
    ("open", lambda: scenes.small_open(71, n_curves=3, size=48, p=(2, 3, 5))),
    ("closed-strokes", lambda: scenes.small_closed(72, n_curves=3, size=48, filled=False, degrees=(2, 3, 4))),
    ("filled", lambda: scenes.small_closed(73, n_curves=3, size=48, filled=True, h=2.0)),
]
VARIANTS = [("weights",), ("knots",), ("weights", "knots")]


def _rel_ok(gpu, ref, tol=1e-3):
    gpu = np.asarray(gpu, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    nr = np.linalg.norm(ref)
    if nr == 0:
        return np.abs(gpu).max() <= 1e-9
    return (np.linalg.norm(gpu - ref) <= tol * nr) and (np.abs(gpu - ref).max() <= tol * np.abs(ref).max())


def _backward(sc, frozen):
    sp, img, rep, (k, t, c), G = run_scene(sc)
    tgt = torch.as_tensor(sc.target, device="cuda").contiguous()
    dimg = torch.empty_like(img)
    loss = torch.zeros(1, device="cuda")
    sp.mse(img, tgt, dimg, loss)
    grads = (torch.full_like(k, 7.0), torch.full_like(t, 7.0), torch.full_like(c, 7.0))
    sp.backward(k, t, c, dimg, grads=grads, frozen=frozen)
    torch.cuda.synchronize()
    return sp, [g.cpu().numpy() for g in grads]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("frozen", VARIANTS, ids=["-".join(v) for v in VARIANTS])
def test_frozen_backward_matches_oracle(name, make, frozen):
    sc = make()
    ref = op.loss_and_grads(sc)
    _, (dk, dt, dc) = _backward(sc, frozen)
    dk = dk.reshape(-1, 4)
    assert _rel_ok(dc, ref["dcolor"]), "dcolor"
    for j in (0, 1, 2):
        assert _rel_ok(dk[:, j], ref["dkey"][:, j]), j
    if "weights" in frozen:
        assert np.all(dk[:, 3] == 0.0)
    else:
        assert _rel_ok(dk[:, 3], ref["dkey"][:, 3])
    if "knots" in frozen:
        assert np.all(dt == 7.0)   # not touched
    else:
        assert _rel_ok(dt, ref["dtau"])


@pytest.mark.parametrize("frozen", VARIANTS, ids=["-".join(v) for v in VARIANTS])
def test_frozen_geometry_matches_oracle(frozen):
    sc = scenes.small_open(74, n_curves=3, size=40, p=(2, 3, 4, 5))
    plans = op.plan(sc)
    box = (6.0, 5.0, sc.width - 7.0, sc.height - 6.0)
    ref = og.geometry_loss_and_grads(sc, plans, order=3, lambda_bbox=2.0, box=box)
    sp = Splatter(sc)
    k, t, c = scene_tensors(sc)
    sp.fit(k, t, c)
    loss = torch.zeros(2, device="cuda")
    g = (torch.zeros_like(k), torch.full_like(t, 7.0))
    sp.geometry(k, t, c, loss, g, lambda_bbox=2.0, box=box, frozen=frozen)
    dk = g[0].cpu().numpy().reshape(-1, 4)
    dt = g[1].cpu().numpy()
    for j in (0, 1):
        assert _rel_ok(dk[:, j], ref["dkey"][:, j]), j
    if "weights" in frozen:
        assert np.all(dk[:, 3] == 0.0)
    else:
        assert _rel_ok(dk[:, 3], ref["dkey"][:, 3])
    if "knots" in frozen:
        assert np.all(dt == 7.0)
    else:
        assert _rel_ok(dt - 7.0, ref["dtau"])


def test_adam_keeps_frozen_parameters():
    """Three optimisation steps with weights and knots frozen: w and tau stay
    bit-for-bit where they started while positions move."""
    sc = scenes.small_open(75, n_curves=3, size=40)
    sp = Splatter(sc)
    k, t, c = scene_tensors(sc)
    sp.fit(k, t, c)
    k0, t0 = k.clone(), t.clone()
    tgt = torch.as_tensor(sc.target, device="cuda").contiguous()
    state = {}
    frozen = ("weights", "knots")
    for step in range(1, 4):
        img = sp.forward(k, t, c)
        dimg = torch.empty_like(img)
        loss = torch.zeros(1, device="cuda")
        sp.mse(img, tgt, dimg, loss)
        grads = sp.backward(k, t, c, dimg, frozen=frozen)
        sp.adam(k, t, c, grads, state, step, frozen=frozen)
    torch.cuda.synchronize()
    kk, kk0 = k.view(-1, 4).cpu().numpy(), k0.view(-1, 4).cpu().numpy()
    assert np.array_equal(kk[:, 3], kk0[:, 3])
    assert np.array_equal(t.cpu().numpy(), t0.cpu().numpy())
    assert np.abs(kk[:, :2] - kk0[:, :2]).max() > 0
