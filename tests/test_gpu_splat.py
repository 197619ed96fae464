"""Splat stage on the GPU against the oracle, both fed the same FP32 Gaussian
set: bins and sort order bit for bit, the image within 1e-5 absolute (parity
thresholds), per-Gaussian gradients of the blend adjoint within 1e-3."""
import numpy as np
import pytest
import torch

import scenes
from oracle import pipeline as op

from gpu_util import run_records, sorted_pairs, tile_ranges

pytestmark = pytest.mark.gpu

CASES = [
    ("open-40", lambda: scenes.small_open(31, n_curves=3, size=40)),
    ("open-gray-37x53", lambda: scenes.small_open(32, n_curves=4, size=53, height=37, channels=1)),
    ("filled-48", lambda: scenes.small_closed(33, n_curves=3, size=48, filled=True, h=2.0)),
    ("strokes-44", lambda: scenes.small_closed(34, n_curves=3, size=44, filled=False)),
    ("two-scenes-40", lambda: scenes.small_closed(35, n_curves=2, size=40, filled=True, h=2.0, n_scenes=2)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("mode", ["parity", "production"])
def test_bins_sort_and_image(name, make, mode):
    sc = make()
    if mode == "production":
        sc = sc.with_raster(**scenes.RASTER_DEFAULTS)
    g = op.gaussians_fp32(sc)
    sp, img, rep, inputs = run_records(sc, g["rec"], g["curve"])
    assert rep.status == 0
    tid_o, gid_o, ranges_o = op.pairs_records(sc, g["rec"], g["curve"])
    assert rep.pairs == tid_o.shape[0]
    tid, gid = sorted_pairs(sp, inputs, rep.pairs)
    np.testing.assert_array_equal(tid, tid_o)
    np.testing.assert_array_equal(gid, gid_o)
    rg = tile_ranges(sp, inputs, ranges_o.shape[0])
    np.testing.assert_array_equal(rg, ranges_o)
    ref, flags = op.render_records(sc, g["rec"], g["curve"], return_flags=True)
    out = img.cpu().numpy().astype(np.float64)
    err = np.abs(out - ref)
    if mode == "parity":
        assert err.max() <= 1e-5, err.max()
    else:
        ok = ~flags[..., None].repeat(sc.channels, -1)
        assert err[ok].max() <= 1e-5, err[ok].max()
        assert flags.mean() < 0.05


def test_image_is_deterministic():
    sc = scenes.small_closed(36, n_curves=3, size=48, filled=True, h=2.0)
    g = op.gaussians_fp32(sc)
    _, a, _, _ = run_records(sc, g["rec"], g["curve"])
    _, b, _, _ = run_records(sc, g["rec"], g["curve"])
    assert torch.equal(a, b)


@pytest.mark.parametrize("name,make", CASES[:4], ids=[c[0] for c in CASES[:4]])
def test_blend_adjoint(name, make):
    sc = make()
    g = op.gaussians_fp32(sc)
    sp, img, rep, (k, t, c) = run_records(sc, g["rec"], g["curve"])
    rng = np.random.default_rng(7)
    dimg = rng.standard_normal(img.shape).astype(np.float32)
    sp.backward(k, t, c, torch.as_tensor(dimg, device="cuda"), chain=False)
    G = g["rec"].shape[0]
    dg = sp.dgauss[:G].cpu().numpy().astype(np.float64)
    drec, dcol = op.record_grads(sc, g["rec"], g["curve"], dimg)
    # dgauss rows: {dmu_x, dmu_y, dsigma, 0, dopacity, dr, dg, db}
    for j, (gpu, ref) in enumerate(zip(dg[:, [0, 1, 2, 4]].T, drec.T)):
        scale = np.abs(ref).max()
        assert np.linalg.norm(gpu - ref) <= 1e-3 * np.linalg.norm(ref) + 1e-7, j
        assert np.abs(gpu - ref).max() <= 1e-3 * scale + 1e-7, j
    # per-curve colour gradient: sum of the per-Gaussian colour gradients
    C = sc.channels
    gcol = np.zeros((sc.n_curves, 3))
    np.add.at(gcol, g["curve"], dg[:, 5:8])
    ref = dcol[:, :C]
    assert np.abs(gcol[:, :C] - ref).max() <= 1e-3 * np.abs(ref).max() + 1e-7


def test_empty_and_offcanvas_sets():
    sc = scenes.small_open(37, n_curves=1, size=40)
    rec = np.array([[-100.0, -100.0, 1.0, 0.9], [20.0, 20.0, 0.0, 0.9], [20.0, 20.0, 1.0, 0.0]], np.float32)
    curve = np.zeros(3, np.int32)
    sp, img, rep, _ = run_records(sc, rec, curve)
    assert rep.status == 0 and rep.pairs == 0
    bg = np.asarray(sc.raster["bg"], np.float32)
    assert np.array_equal(img.cpu().numpy(), np.broadcast_to(bg, img.shape))
    sp, img, rep, _ = run_records(sc, rec[:0], curve[:0])
    assert rep.pairs == 0 and np.array_equal(img.cpu().numpy(), np.broadcast_to(bg, img.shape))


def test_pair_capacity_overflow_reports_size():
    sc = scenes.small_closed(38, n_curves=3, size=48, filled=True, h=2.0)
    g = op.gaussians_fp32(sc)
    G = g["rec"].shape[0]
    tid_o, _, _ = op.pairs_records(sc, g["rec"], g["curve"])
    sp, img, rep, _ = run_records(sc, g["rec"], g["curve"], capacity=(G, 100, 16))
    assert rep.status == 2 and rep.pairs == tid_o.shape[0]


def test_adam_step_matches_oracle():
    """ns_adam_step (with the clamps of Table S1) against the FP64 definition."""
    import ctypes as C
    from oracle import optim
    from paper_2606_31764_b300 import binding as B
    rng = np.random.default_rng(9)
    n = 100_003
    p = rng.uniform(-0.02, 2.0, n).astype(np.float32)
    tp = torch.as_tensor(p, device="cuda")
    tm = torch.zeros(n, device="cuda")
    tv = torch.zeros(n, device="cuda")
    m = np.zeros(n)
    v = np.zeros(n)
    pp = p.astype(np.float64)
    # key-point layout {x, y, s, w}: unbounded x, y; s >= 0; w in [0.01, 10] (Table S1)
    lo = (C.c_float * 4)(-np.inf, -np.inf, 0.0, 0.01)
    hi = (C.c_float * 4)(np.inf, np.inf, np.inf, 10.0)
    lo_np = np.tile([-np.inf, -np.inf, 0.0, 0.01], n // 4 + 1)[:n]
    hi_np = np.tile([np.inf, np.inf, np.inf, 10.0], n // 4 + 1)[:n]
    for step in range(1, 4):
        g = rng.standard_normal(n).astype(np.float32)
        tg = torch.as_tensor(g, device="cuda")
        B.call("ns_adam_step", C.c_void_p(tp.data_ptr()), C.c_void_p(tg.data_ptr()), C.c_void_p(tm.data_ptr()),
               C.c_void_p(tv.data_ptr()), C.c_int64(n), C.c_float(0.05), C.c_float(0.9), C.c_float(0.999),
               C.c_float(1e-8), C.c_int32(step), lo, hi, C.c_int32(4), None,
               C.c_void_p(torch.cuda.current_stream().cuda_stream))
        pp, m, v = optim.adam_step(pp, g, m, v, step, lr=0.05, lo=lo_np, hi=hi_np)
        torch.cuda.synchronize()
        assert np.abs(tp.cpu().numpy() - pp).max() <= 1e-6
        assert np.abs(tm.cpu().numpy() - m).max() <= 1e-6


VARIANTS = [(8, 1, 1), (8, 2, 2), (16, 1, 4), (16, 4, 1), (32, 2, 2), (32, 4, 4), (32, 1, 1)]


@pytest.mark.parametrize("tile,pf,pb", VARIANTS, ids=[f"t{t}-f{a}-b{b}" for t, a, b in VARIANTS])
def test_tile_and_pixels_per_thread_variants(tile, pf, pb):
    """Every tile size and blend decomposition: bins bit-exact, image 1e-5,
    adjoint within 1e-3 (the decomposition must not change any result)."""
    sc = scenes.small_closed(81, n_curves=3, size=70, filled=True, h=2.0, height=53)
    sc = sc.with_raster(tile=tile, ppt_fwd=pf, ppt_bwd=pb)
    g = op.gaussians_fp32(sc)
    sp, img, rep, (k, t, c) = run_records(sc, g["rec"], g["curve"])
    assert rep.status == 0
    tid_o, gid_o, ranges_o = op.pairs_records(sc, g["rec"], g["curve"])
    tid, gid = sorted_pairs(sp, (k, t, c), rep.pairs)
    np.testing.assert_array_equal(tid, tid_o)
    np.testing.assert_array_equal(gid, gid_o)
    ref = op.render_records(sc, g["rec"], g["curve"])
    assert np.abs(img.cpu().numpy() - ref).max() <= 1e-5
    rng = np.random.default_rng(3)
    dimg = rng.standard_normal(img.shape).astype(np.float32)
    sp.backward(k, t, c, torch.as_tensor(dimg, device="cuda"), chain=False)
    G = g["rec"].shape[0]
    dg = sp.dgauss[:G].cpu().numpy().astype(np.float64)
    drec, _ = op.record_grads(sc, g["rec"], g["curve"], dimg)
    for j, col in enumerate((0, 1, 2, 4)):    # rows {dmu_x, dmu_y, dsigma, 0, dopacity, dr, dg, db}
        ref_j = drec[:, j]
        assert np.linalg.norm(dg[:, col] - ref_j) <= 1e-3 * np.linalg.norm(ref_j) + 1e-7


def test_autotune_keeps_the_image():
    from paper_2606_31764_b300.splat import Splatter, scene_tensors
    sc = scenes.small_closed(82, n_curves=4, size=96, filled=True, h=1.0).with_raster(**scenes.RASTER_DEFAULTS)
    sp = Splatter(sc)
    k, t, c = scene_tensors(sc)
    sp.fit(k, t, c)
    before = sp.forward(k, t, c).clone()
    dimg = torch.ones_like(before)
    pf, pb = sp.autotune_blend(k, t, c, dimg, repeats=2)
    from paper_2606_31764_b300 import binding as B
    grp = B.BLEND_LANE_GROUPS
    assert pf in (1, 2, 4, 1 | grp, 2 | grp) and pb in (1, 2, 4, 1 | grp, 2 | grp)
    assert torch.equal(sp.image, before)
    after = sp.forward(k, t, c)
    assert torch.equal(after, before)
