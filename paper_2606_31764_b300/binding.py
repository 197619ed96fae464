"""ctypes binding of the C ABI in include/nurbs_splat.h (argument marshalling only).

Every entry point keeps its C name.  Structures mirror the header field by
field.  Loading fails loudly when the shared library has not been built: there
is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnurbs_splat.so")

NS_OK, NS_ERR_INVALID_ARG, NS_ERR_CAPACITY, NS_ERR_INVALID_CURVE, NS_ERR_CUDA = range(5)
STATUS_NAMES = {0: "NS_OK", 1: "NS_ERR_INVALID_ARG", 2: "NS_ERR_CAPACITY", 3: "NS_ERR_INVALID_CURVE",
                4: "NS_ERR_CUDA"}
NS_CLOSED, NS_FILLED = 1, 2

_p = C.c_void_p


class NsCurves(C.Structure):
    _fields_ = [("n_scenes", C.c_int32), ("n_curves", C.c_int32), ("n_keys", C.c_int32), ("n_taus", C.c_int32),
                ("height", C.c_int32), ("width", C.c_int32), ("channels", C.c_int32),
                ("scene_curve_offset", _p), ("degree", _p), ("flags", _p), ("key_offset", _p),
                ("tau_offset", _p), ("key", _p), ("tau", _p), ("color", _p), ("stroke_degrees", C.c_int32)]


class NsSampleParams(C.Structure):
    _fields_ = [("delta_c", C.c_float), ("rho", C.c_float), ("delta_b", C.c_float), ("h", C.c_float),
                ("eta", C.c_float), ("gamma", C.c_float), ("pad_frac", C.c_float), ("kappa", C.c_int32),
                ("nl_mult", C.c_int32), ("fill_rule", C.c_int32), ("fill_cull", C.c_float),
                ("contour_mode", C.c_int32), ("fill_tile", C.c_int32)]


class NsRasterParams(C.Structure):
    _fields_ = [("tile", C.c_int32), ("k_sigma", C.c_float), ("alpha_min", C.c_float), ("alpha_max", C.c_float),
                ("t_min", C.c_float), ("bg", C.c_float * 3), ("ppt_fwd", C.c_int32), ("ppt_bwd", C.c_int32),
                ("fill_layers", C.c_int32)]


class NsCapacity(C.Structure):
    _fields_ = [("gaussians", C.c_int64), ("pairs", C.c_int64), ("boundary", C.c_int64)]


class NsGaussians(C.Structure):
    _fields_ = [("capacity", C.c_int64), ("rec", _p), ("curve", _p), ("aux", _p), ("count", _p), ("shape", _p)]


class NsGeometryParams(C.Structure):
    _fields_ = [("lambda_deriv", C.c_float), ("order", C.c_int32), ("nodes", C.c_int32), ("lambda_bbox", C.c_float),
                ("penalty", C.c_int32), ("box", C.c_float * 4)]


NS_PENALTY_RELU, NS_PENALTY_SOFTPLUS = 0, 1


class NsCurveGrads(C.Structure):
    _fields_ = [("dkey", _p), ("dtau", _p), ("dcolor", _p), ("frozen", C.c_int32)]


NS_FROZEN_WEIGHTS, NS_FROZEN_KNOTS = 1, 2


class NsReport(C.Structure):
    _fields_ = [("status", C.c_int32), ("bad_curve", C.c_int32), ("gaussians", C.c_int64), ("pairs", C.c_int64),
                ("boundary", C.c_int64), ("fill_culled", C.c_int64), ("blend_evals", C.c_int64),
                ("blend_bwd_evals", C.c_int64), ("blend_contribs", C.c_int64), ("blend_visits", C.c_int64),
                ("blend_bwd_visits", C.c_int64)]


# name -> (restype, argtypes); the declarations of include/nurbs_splat.h
SIGNATURES = {
    "ns_default_sample_params": (NsSampleParams, []),
    "ns_default_raster_params": (NsRasterParams, []),
    "ns_workspace_size": (C.c_size_t, [C.POINTER(NsCurves), C.POINTER(NsCapacity), C.POINTER(NsRasterParams)]),
    "nurbs_sample": (C.c_int, [C.POINTER(NsCurves), C.POINTER(NsSampleParams), C.POINTER(NsCapacity),
                               C.POINTER(NsGaussians), _p, C.c_size_t, _p]),
    "splat_forward": (C.c_int, [C.POINTER(NsCurves), C.POINTER(NsGaussians), C.POINTER(NsRasterParams),
                                C.POINTER(NsCapacity), _p, _p, C.c_size_t, _p]),
    "splat_backward": (C.c_int, [C.POINTER(NsCurves), C.POINTER(NsGaussians), C.POINTER(NsSampleParams),
                                 C.POINTER(NsRasterParams), C.POINTER(NsCapacity), _p, _p,
                                 C.POINTER(NsCurveGrads), C.c_int32, _p, C.c_size_t, _p]),
    "ns_grid_step": (C.c_float, [C.c_int32, C.c_int32, C.c_float, C.c_float, C.c_float, C.c_float]),
    "ns_mse_loss": (C.c_int, [_p, _p, C.c_int64, _p, _p, _p]),
    "ns_adam_step": (C.c_int, [_p, _p, _p, _p, C.c_int64, C.c_float, C.c_float, C.c_float, C.c_float,
                               C.c_int32, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_int32,
                               C.POINTER(C.c_float), _p]),
    "ns_poll_status": (C.c_int, [_p, C.POINTER(NsReport), _p]),
    "ns_clear_status": (C.c_int, [_p, _p]),
    "ns_workspace_copy": (C.c_int, [_p, C.POINTER(NsCurves), C.POINTER(NsCapacity), C.POINTER(NsRasterParams),
                                    C.c_int32, _p, C.c_size_t, _p]),
    "ns_autotune_blend": (C.c_int, [C.POINTER(NsCurves), C.POINTER(NsGaussians), C.POINTER(NsRasterParams),
                                    C.POINTER(NsCapacity), _p, _p, _p, C.c_size_t, C.c_int32, _p]),
    "ns_profile_next_launch": (C.c_int, [C.c_int32, _p, _p]),
    "splat_forward_noalloc": (C.c_int, [C.POINTER(NsCurves), C.POINTER(NsGaussians), C.POINTER(NsRasterParams),
                                        _p, C.POINTER(NsReport), _p]),
    "ns_default_geometry_params": (NsGeometryParams, []),
    "ns_geometry_loss": (C.c_int, [C.POINTER(NsCurves), C.POINTER(NsGaussians), C.POINTER(NsSampleParams),
                                   C.POINTER(NsRasterParams),
                                   C.POINTER(NsGeometryParams), C.POINTER(NsCapacity), _p, C.POINTER(NsCurveGrads),
                                   _p, C.c_size_t, _p]),
    "ns_udf_mse_loss": (C.c_int, [C.POINTER(NsCurves), C.POINTER(NsSampleParams), C.POINTER(NsRasterParams),
                                  C.POINTER(NsCapacity), _p, C.c_float, _p, _p, _p, _p, _p, C.c_size_t, _p]),
    "ns_xing_loss": (C.c_int, [C.POINTER(NsCurves), C.c_float, _p, _p, _p]),
    "ns_seed_scratch_size": (C.c_size_t, [C.c_int32, C.c_int32, C.c_int32]),
    "ns_seed_windows": (C.c_int, [_p, _p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _p, C.c_size_t,
                                  _p, _p, _p]),
    "ns_launch_count": (C.c_uint64, []),
    "ns_last_error": (C.c_char_p, []),
}

# ns_raster_params.ppt_fwd / ppt_bwd flag: lane-group blend decomposition (nurbs_splat.h)
BLEND_LANE_GROUPS = 16

KERNELS = dict(plan=1, boundary=2, emit=3, bin_count=4, bin_emit=5, radix_hist=6, radix_scatter=7, ranges=8,
               blend_fwd=9, blend_bwd=10, chain=11, chain_boundary=12, knot_grads=13, mse=14, adam=15, scan=16,
               other=17, chain_contour=18, deriv_loss=19, bbox_loss=20, fill_sdf=21)

_lib = None


class NsError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__(f"{fn} -> {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load the library (once) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing "
                           "(run `python -m paper_2606_31764_b300.build` or __graft_entry__.build())")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(fn_name: str, status: int):
    if status != NS_OK:
        raise NsError(fn_name, status, load().ns_last_error().decode())


def call(name: str, *args):
    """Call an entry point that returns ns_status; raise NsError on failure."""
    st = getattr(load(), name)(*args)
    check(name, st)
    return st


def exported_symbols():
    return list(SIGNATURES)
