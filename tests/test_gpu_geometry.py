"""The geometric regularisers on the GPU (ns_geometry_loss: Eq. 11 derivative
loss, Eq. 12 bounding-box loss) against the oracle's FP64 values and exact
gradients.  Values within 1e-4 relative (FP32 sums of squared derivatives);
gradients per tensor ||g_gpu - g_ref|| <= 1e-3 ||g_ref|| and elementwise
|g_gpu - g_ref| <= 1e-3 max|g_ref|."""
import numpy as np
import pytest
import torch

import scenes
from oracle import geometry as og
from oracle import pipeline as op
from paper_2606_31764_b300.splat import Splatter, scene_tensors

pytestmark = pytest.mark.gpu

CASES = [
    ("open", lambda: scenes.small_open(61, n_curves=4, size=48, p=(1, 2, 3, 5))),
    ("closed-strokes", lambda: scenes.small_closed(62, n_curves=3, size=48, filled=False, degrees=(2, 3, 4, 5))),
    ("filled", lambda: scenes.small_closed(63, n_curves=3, size=48, filled=True, h=2.0)),
    ("filled-batched", lambda: scenes.small_closed(64, n_curves=2, size=40, filled=True, h=2.0, n_scenes=2)),
    ("config1", lambda: scenes.config1()),
]


def _rel_ok(gpu, ref, tol=1e-3):
    gpu = np.asarray(gpu, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    nr = np.linalg.norm(ref)
    if nr == 0:
        return np.abs(gpu).max() <= 1e-9
    return (np.linalg.norm(gpu - ref) <= tol * nr) and (np.abs(gpu - ref).max() <= tol * np.abs(ref).max())


def _run(sc, grads=True, **kw):
    sp = Splatter(sc)
    k, t, c = scene_tensors(sc)
    sp.fit(k, t, c)
    loss = torch.zeros(2, device="cuda")
    g = (torch.zeros_like(k), torch.zeros_like(t)) if grads else None
    sp.geometry(k, t, c, loss, g, **kw)
    torch.cuda.synchronize()
    out = dict(loss=loss.cpu().numpy().astype(np.float64), report=sp.report())
    if grads:
        out["dkey"] = g[0].cpu().numpy().reshape(-1, 4)
        out["dtau"] = g[1].cpu().numpy()
    return out


def _check(sc, ref, out):
    assert out["report"].status == 0
    for j, nm in ((0, "deriv"), (1, "bbox")):
        r = ref[nm]
        assert abs(out["loss"][j] - r) <= 1e-4 * abs(r) + 1e-6, (nm, out["loss"][j], r)
    assert _rel_ok(out["dtau"], ref["dtau"]), "dtau"
    for j, nm in ((0, "x"), (1, "y"), (3, "w")):
        assert _rel_ok(out["dkey"][:, j], ref["dkey"][:, j]), "dkey." + nm
    assert np.abs(out["dkey"][:, 2]).max() == 0.0   # widths are not regularised


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("penalty", ["relu", "softplus"])
def test_geometry_matches_oracle(name, make, penalty):
    sc = make()
    plans = op.plan(sc)
    assert all(p.well_separated() for p in plans)
    box = (6.0, 5.0, sc.width - 7.0, sc.height - 6.0)
    kind = og.RELU if penalty == "relu" else og.SOFTPLUS
    ref = og.geometry_loss_and_grads(sc, plans, order=3, lambda_deriv=0.5, lambda_bbox=2.0, box=box, kind=kind)
    out = _run(sc, lambda_deriv=0.5, lambda_bbox=2.0, penalty=penalty, box=box)
    _check(sc, ref, out)


@pytest.mark.parametrize("order", [1, 2, 4])
def test_other_derivative_orders(order):
    sc = scenes.small_open(65, n_curves=3, size=40, p=(2, 3, 4, 5))
    plans = op.plan(sc)
    ref = og.geometry_loss_and_grads(sc, plans, order=order, nodes=101, lambda_bbox=0.0)
    out = _run(sc, order=order, nodes=101, lambda_bbox=0.0)
    _check(sc, ref, out)


def test_canvas_box_default_and_values_only():
    """An empty box selects the canvas; without gradient outputs the values are
    the same; gradients are added to what the outputs already hold."""
    sc = scenes.small_open(66, n_curves=3, size=40)
    plans = op.plan(sc)
    ref = og.geometry_loss_and_grads(sc, plans, lambda_bbox=5.0, kind=og.SOFTPLUS)   # the library's default weights
    out = _run(sc, penalty="softplus")
    _check(sc, ref, out)
    vals = _run(sc, grads=False, penalty="softplus")
    assert np.array_equal(vals["loss"], out["loss"]) or np.allclose(vals["loss"], out["loss"], rtol=1e-6)
    sp = Splatter(sc)
    k, t, c = scene_tensors(sc)
    sp.fit(k, t, c)
    loss = torch.zeros(2, device="cuda")
    g = (torch.zeros_like(k), torch.zeros_like(t))
    sp.geometry(k, t, c, loss, g, penalty="softplus")
    sp.geometry(k, t, c, loss, g, penalty="softplus")
    assert _rel_ok(g[0].cpu().numpy(), 2 * out["dkey"].reshape(-1), 1e-5)
    assert _rel_ok(g[1].cpu().numpy(), 2 * out["dtau"], 1e-5)


@pytest.mark.parametrize("order", [1, 2, 3, 4])
@pytest.mark.parametrize("make", ["open", "closed", "filled"])
def test_taylor_span_kernel_matches_oracle(make, order):
    """Enough quadrature nodes per knot span that the per-curve kernel (span
    Taylor forms, the reverse once per span) takes every curve."""
    if make == "open":
        sc = scenes.small_open(67, n_curves=4, size=40, p=(1, 2, 3, 4, 5))
    else:
        sc = scenes.small_closed(68, n_curves=3, size=44, filled=make == "filled", h=2.0, degrees=(2, 3, 4, 5))
    plans = op.plan(sc)
    box = (5.0, 4.0, sc.width - 6.0, sc.height - 5.0)
    ref = og.geometry_loss_and_grads(sc, plans, order=order, nodes=700, lambda_deriv=0.7, lambda_bbox=1.5,
                                     box=box, kind=og.SOFTPLUS)
    out = _run(sc, order=order, nodes=700, lambda_deriv=0.7, lambda_bbox=1.5, box=box, penalty="softplus")
    _check(sc, ref, out)
