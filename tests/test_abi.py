"""The C ABI library loads and exports every entry point include/*.h declares
(no device calls: runs without a GPU)."""
import glob
import os
import re

import pytest

from paper_2606_31764_b300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(", txt,
                             re.M):
            names.add(m.group(1))
    return names - {"if", "while", "for", "return", "sizeof"}


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("nurbs_sample", "splat_forward", "splat_backward", "ns_workspace_size", "ns_poll_status"):
        assert name in d


def test_library_exports_every_declared_symbol():
    if not os.path.exists(binding.LIB_PATH):
        from paper_2606_31764_b300 import build
        build.build()
    lib = binding.load()
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(binding.exported_symbols()) == _declared()


def test_defaults_match_table_s1():
    import json
    lib = binding.load()
    sp = lib.ns_default_sample_params()
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "table_s1_defaults.json")))
    for k in ("delta_c", "rho", "delta_b", "h", "eta", "gamma", "kappa", "nl_mult"):
        assert getattr(sp, k) == pytest.approx(gold[k]), k
    gp = lib.ns_default_geometry_params()
    assert gp.lambda_deriv == pytest.approx(gold["lambda_deriv_calligraphy"])
    assert gp.lambda_bbox == pytest.approx(gold["lambda_bbox_calligraphy"])
    assert gp.order == 3


def test_host_side_argument_errors_need_no_gpu():
    import ctypes as C
    lib = binding.load()
    c = binding.NsCurves()
    c.n_scenes, c.n_curves, c.height, c.width, c.channels = 1, 0, 32, 32, 2   # channels must be 1 or 3
    cap = binding.NsCapacity(16, 16, 16)
    rp = lib.ns_default_raster_params()
    assert lib.ns_workspace_size(C.byref(c), C.byref(cap), C.byref(rp)) == 0
    assert b"channels" in lib.ns_last_error()
    c.channels = 3
    assert lib.ns_workspace_size(C.byref(c), C.byref(cap), C.byref(rp)) > 0
    rp.tile = 12
    assert lib.ns_workspace_size(C.byref(c), C.byref(cap), C.byref(rp)) == 0


def test_grid_step_schedule_matches_oracle():
    from oracle.optim import grid_step
    lib = binding.load()
    for (hmax, hmin, tb, te, T) in ((4.0, 1.0, 0.1, 0.8, 300), (8.0, 1.0, 0.1, 0.8, 300), (2.0, 0.5, 0.0, 1.0, 50)):
        for t in range(T):
            assert abs(lib.ns_grid_step(t, T, hmax, hmin, tb, te) - grid_step(t, T, hmax, hmin, tb, te)) <= 1e-6 * hmax


def test_geometry_loss_argument_errors_need_no_gpu():
    """ns_geometry_loss rejects a bad order or penalty on the host, before any
    device work."""
    import ctypes as C
    lib = binding.load()
    c = binding.NsCurves()
    c.n_scenes, c.n_curves, c.height, c.width, c.channels = 1, 0, 32, 32, 3
    cap = binding.NsCapacity(16, 16, 16)
    sp = lib.ns_default_sample_params()
    rp = lib.ns_default_raster_params()
    gp = lib.ns_default_geometry_params()
    assert (gp.order, gp.penalty, gp.nodes) == (3, binding.NS_PENALTY_RELU, 0)
    loss = C.c_void_p(16)   # never dereferenced: the checks fail first
    ws = C.c_void_p(256)
    for field, bad, word in (("order", 5, b"order"), ("order", 0, b"order"), ("penalty", 7, b"penalty"),
                             ("nodes", -1, b"nodes")):
        g = lib.ns_default_geometry_params()
        setattr(g, field, bad)
        gs = binding.NsGaussians()
        st = lib.ns_geometry_loss(C.byref(c), C.byref(gs), C.byref(sp), C.byref(rp), C.byref(g), C.byref(cap), loss,
                                  None, ws, C.c_size_t(1 << 20), None)
        assert st == binding.NS_ERR_INVALID_ARG
        assert word in lib.ns_last_error()


def test_stroke_degree_hint_mask():
    """The launch hint the Python tables give the library: bit 0 (given) and
    one bit per degree among the curves that are not filled; a batch of fills
    gives 1 (no stroke kernel to launch)."""
    from paper_2606_31764_b300.splat import stroke_degree_mask
    F, C = binding.NS_FILLED, binding.NS_CLOSED
    assert stroke_degree_mask([2, 3, 5], [F | C, F | C, F | C]) == 1
    assert stroke_degree_mask([2, 3, 5], [C, 0, F | C]) == 1 | (1 << 2) | (1 << 3)
    assert stroke_degree_mask([1, 1, 4], [0, 0, C]) == 1 | (1 << 1) | (1 << 4)
    assert stroke_degree_mask([], []) == 1


def test_curve_table_carries_the_hint_last():
    """ns_curves ends with the int32 launch hint after the colour pointer, so a
    table built field by field (or zeroed) without it means 'not given'."""
    names = [f[0] for f in binding.NsCurves._fields_]
    assert names[-2:] == ["color", "stroke_degrees"]
    assert binding.NsCurves().stroke_degrees == 0
