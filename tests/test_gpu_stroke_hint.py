"""The stroke-degree launch hint of ns_curves (stroke_degrees): with it,
splat_backward launches the contour-chain kernels of the strokes' degrees
only, and none for a batch of fills.  It changes which kernels are launched,
not what is computed: a step with the hint and one without it (0: not given)
give the same records and image bit for bit, and the same gradients within
the rounding of atomic sums in another order.  A stroke whose degree the hint
leaves out is reported as an invalid curve."""
import numpy as np
import pytest
import torch

import scenes
from paper_2606_31764_b300 import binding as B
from paper_2606_31764_b300.splat import Splatter, scene_tensors

pytestmark = pytest.mark.gpu


def _step(scene, hint=None):
    sp = Splatter(scene, capacity=(1 << 14, 1 << 16, 1 << 12))
    if hint is not None:
        sp.dev.stroke_degrees = hint
    k, t, c = scene_tensors(scene)
    rep = sp.fit(k, t, c)
    img = sp.forward(k, t, c).clone()
    tgt = torch.as_tensor(scene.target, device="cuda").contiguous()
    dimg = torch.empty_like(img)
    loss = torch.zeros(1, device="cuda")
    sp.mse(img, tgt, dimg, loss)
    dk, dt, dc = sp.backward(k, t, c, dimg)
    torch.cuda.synchronize()
    G = int(sp.count.item())
    return dict(sp=sp, rep=sp.report(), img=img.cpu().numpy(), rec=sp.rec[:G].cpu().numpy(),
                grads=[x.cpu().numpy() for x in (dk, dt, dc)])


def _rel(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("name,make", [
    ("fills-and-strokes", lambda: scenes.small_closed(361, n_curves=4, size=56, filled="alternate", h=1.0)
     .with_raster(**dict(scenes.RASTER_DEFAULTS, tile=8, fill_layers=1))),
    ("fills-only", lambda: scenes.small_closed(362, n_curves=3, size=48, filled=True, h=1.0)
     .with_raster(**dict(scenes.RASTER_DEFAULTS, tile=8, fill_layers=1))),
    ("open-strokes", lambda: scenes.small_open(363, n_curves=3, size=40)),
])
def test_hint_changes_launches_not_results(name, make):
    sc = make()
    with_hint = _step(sc)
    hint = with_hint["sp"].dev.stroke_degrees
    strokes = [int(p) for p, f in zip(sc.degree, sc.flags) if not (int(f) & B.NS_FILLED)]
    assert hint == 1 | sum(1 << p for p in set(strokes))
    without = _step(sc, hint=0)
    assert with_hint["rep"].status == B.NS_OK and without["rep"].status == B.NS_OK
    assert np.array_equal(with_hint["rec"], without["rec"])
    assert np.array_equal(with_hint["img"], without["img"])
    for nm, x, y in zip(("dkey", "dtau", "dcolor"), with_hint["grads"], without["grads"]):
        assert np.isfinite(x).all(), nm
        assert _rel(x, y) <= 1e-6, nm


def test_hint_leaving_out_a_stroke_degree_is_reported():
    sc = scenes.small_closed(364, n_curves=4, size=56, filled="alternate", h=1.0)
    strokes = [(c, int(p)) for c, (p, f) in enumerate(zip(sc.degree, sc.flags)) if not (int(f) & B.NS_FILLED)]
    assert strokes
    c0, p0 = strokes[0]
    degrees = {p for _, p in strokes}
    hint = 1 | sum(1 << p for p in degrees if p != p0)
    sp = Splatter(sc, capacity=(1 << 14, 1 << 16, 1 << 12))
    sp.dev.stroke_degrees = hint
    k, t, c = scene_tensors(sc)
    sp.sample(k, t, c)
    r = sp.report()
    assert r.status == B.NS_ERR_INVALID_CURVE
    assert r.bad_curve in {c for c, p in strokes if p == p0}   # the first one the device recorded
