"""The layer-wise vectorisation terms on the GPU against the oracle: the
distance-weighted image loss and its gradient, the self-crossing penalty and
its gradient, and the error-window seeding; then a short run of the loop."""
import dataclasses

import numpy as np
import pytest
import torch

import scenes
from oracle import live as ol
from oracle import pipeline as op
from paper_2606_31764_b300.live import LayerwiseVectorizer
from paper_2606_31764_b300.splat import Splatter, scene_tensors, seed_windows

pytestmark = pytest.mark.gpu
DT = torch.float64


@pytest.mark.parametrize("new", [[1, -1], [0, 3], [-1, -1]], ids=["one-new", "both-new", "none"])
def test_udf_loss_and_gradient_match_oracle(new):
    sc = scenes.small_closed(91, n_curves=2, size=40, filled=True, h=2.0, n_scenes=2)
    plans = op.plan(sc)
    rng = np.random.default_rng(92)
    img = rng.uniform(0, 1, (2, 40, 40, 3)).astype(np.float32)
    tgt = sc.target.astype(np.float32)
    sp = Splatter(sc)
    k, t, c = scene_tensors(sc)
    sp.fit(k, t, c)
    ti, tt = torch.as_tensor(img, device="cuda"), torch.as_tensor(tgt, device="cuda")
    newc = torch.as_tensor(new, dtype=torch.int32, device="cuda")
    dimg = torch.empty_like(ti)
    loss = torch.zeros(1, device="cuda")
    sp.udf_mse(k, t, c, ti, tt, newc, 6.0, dimg, loss)
    torch.cuda.synchronize()
    kk, tau_t, _ = op.leaves(sc, False)
    w = ol.udf_weights(sc, kk, tau_t, plans, new, 6.0)
    x = torch.tensor(img, dtype=DT, requires_grad=True)
    L = ol.udf_mse(x, torch.tensor(tgt, dtype=DT), w, [n >= 0 for n in new])
    L.backward()
    assert abs(float(loss.item()) - float(L.detach())) <= 1e-5 * float(L.detach())
    g = dimg.cpu().numpy()
    ref = x.grad.numpy()
    assert np.abs(g - ref).max() <= 1e-4 * np.abs(ref).max()


def test_xing_loss_and_gradient_match_oracle():
    sc = scenes.small_closed(93, n_curves=3, size=48, filled=True, degrees=(3,))
    key = sc.key.copy()
    k0 = int(sc.key_offset[1])
    key[k0 + 2, :2] = 2 * key[k0 + 3, :2] - key[k0 + 2, :2]   # fold one key point: reversed turns
    sc = dataclasses.replace(sc, key=key)
    kt, _, _ = op.leaves(sc)
    L = 0.5 * ol.xing_loss(sc, kt)
    L.backward()
    sp = Splatter(sc)
    k, t, c = scene_tensors(sc)
    loss = torch.zeros(1, device="cuda")
    dk = torch.zeros_like(k)
    sp.xing(k, t, c, loss, dk, 0.5)
    torch.cuda.synchronize()
    assert float(L.detach()) > 0
    assert abs(float(loss.item()) - float(L.detach())) <= 1e-5 * float(L.detach())
    g = dk.cpu().numpy().reshape(-1, 4)
    ref = kt.grad.numpy()
    assert np.abs(g[:, :2] - ref[:, :2]).max() <= 1e-4 * np.abs(ref).max()
    assert np.all(g[:, 2:] == 0)


@pytest.mark.parametrize("r", [0, 3, 9])
def test_seed_matches_oracle(r):
    rng = np.random.default_rng(94 + r)
    S, H, W, Cc = 2, 23, 31, 3
    img = rng.uniform(0, 1, (S, H, W, Cc)).astype(np.float32)
    tgt = rng.uniform(0, 1, (S, H, W, Cc)).astype(np.float32)
    img[1, 15:20, 3:9] += 2.0   # a clear maximum in scene 1
    xy, val = seed_windows(torch.as_tensor(img, device="cuda"), torch.as_tensor(tgt, device="cuda"), r)
    torch.cuda.synchronize()
    ref = ol.seed_pixels(img, tgt, r)
    e = ((img.astype(np.float64) - tgt) ** 2).sum(-1)
    for s in range(S):
        x, y = (int(v) for v in xy[s].cpu())
        win = e[s, max(0, y - r):y + r + 1, max(0, x - r):x + r + 1].sum()
        # the chosen window is a maximum (FP32 window sums may break near-ties differently)
        assert win >= ref[s][2] * (1 - 1e-5)
        assert abs(float(val[s]) - ref[s][2]) <= 1e-5 * ref[s][2]
    assert tuple(int(v) for v in xy[1].cpu()) == ref[1][:2]


def test_layerwise_loop_reduces_the_loss():
    """Two rounds of the loop on a two-blob target: each round adds one path
    per scene and the image moves towards the target."""
    rng = np.random.default_rng(95)
    tgt = scenes.blob_target(rng, 2, 48, 48, 3, 3)
    lv = LayerwiseVectorizer(tgt, scenes.SAMPLE_DEFAULTS, scenes.RASTER_DEFAULTS, rounds=2, iters=60, tau_udf=8.0)
    img = lv.run()
    torch.cuda.synchronize()
    assert lv.sp.report().status == 0
    assert lv.batch.n_curves == 4
    err0 = float(((torch.ones_like(lv.target) - lv.target) ** 2).mean())
    err1 = float(((img - lv.target) ** 2).mean())
    assert err1 < err0
