"""splat_forward_noalloc against splat_forward.

The no-allocation variant serves callers that cannot call cudaMalloc where
they render (an engine or server that owns and pre-plans all device memory, a
plugin limited to the buffers it is handed, a loop that must not trigger an
allocation's device synchronisation).  It keeps its scratch in a fixed device
array of the library.  This test renders the same Gaussian set with both entry
points, twice in a row with the new one (the array keeps the previous call's
contents), and compares the images within the 1e-5 image tolerance of the
other splat tests.  Collected last so that a stop-at-first-failure run has
already run everything else.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import scenes
from oracle import pipeline as op
from paper_2606_31764_b300 import binding as B

from gpu_util import run_records

pytestmark = pytest.mark.gpu


def _noalloc(sp, inputs, out, report):
    lib = B.load()
    cs = sp.dev.struct(*inputs)
    return lib.splat_forward_noalloc(C.byref(cs), C.byref(sp.g), C.byref(sp.rp), C.c_void_p(out.data_ptr()),
                                     C.byref(report), C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("production", [False, True])
def test_noalloc_matches_splat_forward(production):
    sc = scenes.small_closed(71, n_curves=3, size=64, filled=True, h=2.0)
    if production:
        sc = sc.with_raster(**scenes.RASTER_DEFAULTS)
    g = op.gaussians_fp32(sc)
    sp, ref, rep, inputs = run_records(sc, g["rec"], g["curve"], capacity=(g["rec"].shape[0], 1 << 16, 16))
    assert rep.status == 0
    for _ in range(2):
        out = torch.full_like(ref, float("nan"))
        r = B.NsReport()
        st = _noalloc(sp, inputs, out, r)
        assert st == B.NS_OK, B.load().ns_last_error()
        assert r.status == 0 and r.pairs == rep.pairs
        assert r.gaussians == g["rec"].shape[0]
        err = (out - ref).abs().max().item()
        assert err <= 1e-5, err


def test_noalloc_rejects_sizes_beyond_its_scratch():
    sc = scenes.small_closed(72, n_curves=2, size=48, filled=True, h=2.0)
    g = op.gaussians_fp32(sc)
    sp, ref, rep, inputs = run_records(sc, g["rec"], g["curve"])
    big = B.NsGaussians(1 << 20, sp.g.rec, sp.g.curve, sp.g.aux, sp.g.count)
    lib = B.load()
    cs = sp.dev.struct(*inputs)
    out = torch.empty_like(ref)
    st = lib.splat_forward_noalloc(C.byref(cs), C.byref(big), C.byref(sp.rp), C.c_void_p(out.data_ptr()), None,
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == B.NS_ERR_INVALID_ARG
    assert b"65536" in lib.ns_last_error()


def test_noalloc_ignores_fill_layers():
    """Fill layers need the sampling plans of a workspace; the no-allocation
    variant has none and bins per Gaussian whatever the raster settings say."""
    sc = scenes.small_closed(73, n_curves=3, size=56, filled=True, h=1.0).with_raster(**scenes.RASTER_DEFAULTS)
    g = op.gaussians_fp32(sc)
    sp, ref, rep, inputs = run_records(sc, g["rec"], g["curve"], capacity=(g["rec"].shape[0], 1 << 16, 16))
    assert rep.status == 0
    sp.rp.fill_layers = 1
    out = torch.full_like(ref, float("nan"))
    r = B.NsReport()
    st = _noalloc(sp, inputs, out, r)
    assert st == B.NS_OK, B.load().ns_last_error()
    assert r.status == 0 and r.pairs == rep.pairs
    assert torch.equal(out, ref)


def test_noalloc_rejects_a_canvas_beyond_its_scratch():
    """Per-pixel state of a 2048 x 2048 canvas alone exceeds the 16 MiB array."""
    sc = scenes.small_closed(74, n_curves=2, size=48, filled=True, h=2.0)
    g = op.gaussians_fp32(sc)
    sp, ref, rep, inputs = run_records(sc, g["rec"], g["curve"])
    cs = sp.dev.struct(*inputs)
    cs.height = cs.width = 2048
    out = torch.empty(2048 * 2048 * 3, device="cuda")
    lib = B.load()
    st = lib.splat_forward_noalloc(C.byref(cs), C.byref(sp.g), C.byref(sp.rp), C.c_void_p(out.data_ptr()), None,
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == B.NS_ERR_INVALID_ARG
    assert b"16777216" in lib.ns_last_error()


def test_noalloc_reports_pair_overflow():
    """2000 Gaussians of sigma 40 px on a 256 x 256 canvas at tile 8 need about
    2.4 million tile pairs, beyond the 262144 the array holds: the pairs past
    it are dropped, the image stays finite and the report says NS_ERR_CAPACITY
    with the number needed.  The next call starts from a clear status."""
    sc = scenes.small_closed(75, n_curves=2, size=256, filled=True, h=2.0).with_raster(tile=8)
    rng = np.random.default_rng(75)
    n = 2000
    rec = np.stack([rng.uniform(0, 256, n), rng.uniform(0, 256, n), np.full(n, 40.0), np.full(n, 0.5)], 1)
    curve = rng.integers(0, sc.n_curves, n)
    order = np.lexsort((np.arange(n), -curve))   # records front to back: the last curve first
    rec, curve = rec[order].astype(np.float32), curve[order].astype(np.int32)
    sp, ref, rep, inputs = run_records(sc, rec, curve, capacity=(n, 1 << 22, 16))
    assert rep.status == 0 and rep.pairs > 1 << 18
    out = torch.full_like(ref, float("nan"))
    r = B.NsReport()
    assert _noalloc(sp, inputs, out, r) == B.NS_OK
    assert r.status == B.NS_ERR_CAPACITY and r.pairs == rep.pairs
    assert torch.isfinite(out).all()
    # a set that fits runs clean right after
    g = op.gaussians_fp32(sc)
    sp2, ref2, rep2, inputs2 = run_records(sc, g["rec"], g["curve"], capacity=(g["rec"].shape[0], 1 << 16, 16))
    out2 = torch.full_like(ref2, float("nan"))
    r2 = B.NsReport()
    assert _noalloc(sp2, inputs2, out2, r2) == B.NS_OK
    assert r2.status == 0 and (out2 - ref2).abs().max().item() <= 1e-5
