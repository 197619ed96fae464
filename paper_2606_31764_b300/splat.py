"""PyTorch-facing layer over the C ABI: device tables, buffers sized by the
library's own counts, the three stages and a torch.autograd.Function.

PyTorch only provides device memory and the stream; every computation runs in
the library's kernels.
"""
from __future__ import annotations

import ctypes as C
import dataclasses

import torch

from . import binding as B


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else C.c_void_p(0)


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def sample_params(d: dict) -> B.NsSampleParams:
    p = B.NsSampleParams()
    for k in ("delta_c", "rho", "delta_b", "h", "eta", "gamma", "pad_frac"):
        setattr(p, k, float(d[k]))
    p.kappa = int(d["kappa"])
    p.nl_mult = int(d["nl_mult"])
    p.fill_rule = int(d["fill_rule"])
    p.fill_cull = float(d.get("fill_cull", 0.0))
    p.contour_mode = int(d.get("contour_mode", 0))
    p.fill_tile = int(d.get("fill_tile", 0))
    return p


def raster_params(d: dict) -> B.NsRasterParams:
    r = B.NsRasterParams()
    r.tile = int(d["tile"])
    r.k_sigma = float(d["k_sigma"])
    r.alpha_min = float(d["alpha_min"])
    r.alpha_max = float(d["alpha_max"])
    r.t_min = float(d["t_min"])
    for i in range(3):
        r.bg[i] = float(d["bg"][i])
    r.ppt_fwd = int(d.get("ppt_fwd", 0))
    r.ppt_bwd = int(d.get("ppt_bwd", 0))
    r.fill_layers = int(d.get("fill_layers", 0))
    return r


@dataclasses.dataclass
class Report:
    status: int
    bad_curve: int
    gaussians: int
    pairs: int
    boundary: int
    fill_culled: int
    blend_evals: int
    blend_bwd_evals: int
    blend_contribs: int
    blend_visits: int = 0
    blend_bwd_visits: int = 0


def stroke_degree_mask(degree, flags) -> int:
    """The library's launch hint ns_curves.stroke_degrees from host copies of
    the curves' degrees and flags: bit 0 set (the hint is given) and bit p for
    every degree p among the curves that are not filled."""
    mask = 1
    for p, f in zip(list(degree), list(flags)):
        if not (int(f) & B.NS_FILLED) and 1 <= int(p) <= 5:
            mask |= 1 << int(p)
    return mask


class DeviceCurves:
    """The static curve tables of a scene batch on the device (int32 CSR)."""

    def __init__(self, scene, device="cuda"):
        i32 = dict(dtype=torch.int32, device=device)
        self.n_scenes = scene.n_scenes
        self.height, self.width, self.channels = scene.height, scene.width, scene.channels
        self.scene_curve_offset = torch.as_tensor(scene.scene_curve_offset, **i32)
        self.degree = torch.as_tensor(scene.degree, **i32)
        self.flags = torch.as_tensor(scene.flags, **i32)
        self.key_offset = torch.as_tensor(scene.key_offset, **i32)
        self.tau_offset = torch.as_tensor(scene.tau_offset, **i32)
        self.n_curves = int(scene.degree.shape[0])
        self.n_keys = int(scene.key.shape[0])
        self.n_taus = int(scene.tau.shape[0])
        self.stroke_degrees = stroke_degree_mask(scene.degree, scene.flags)

    def struct_sizes(self) -> B.NsCurves:
        """The table with placeholder parameter pointers: enough for
        ns_workspace_size, which reads sizes only."""
        c = B.NsCurves()
        c.n_scenes, c.n_curves, c.n_keys, c.n_taus = self.n_scenes, self.n_curves, self.n_keys, self.n_taus
        c.height, c.width, c.channels = self.height, self.width, self.channels
        c.scene_curve_offset = _ptr(self.scene_curve_offset)
        c.degree, c.flags = _ptr(self.degree), _ptr(self.flags)
        c.key_offset, c.tau_offset = _ptr(self.key_offset), _ptr(self.tau_offset)
        c.key = c.tau = c.color = C.c_void_p(256)
        c.stroke_degrees = self.stroke_degrees
        return c

    def struct(self, key, tau, color) -> B.NsCurves:
        for t, n in ((key, self.n_keys * 4), (tau, self.n_taus), (color, self.n_curves * 4)):
            if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or t.numel() != n:
                raise ValueError("key/tau/color must be contiguous float32 CUDA tensors of the scene's sizes")
        c = B.NsCurves()
        c.n_scenes, c.n_curves, c.n_keys, c.n_taus = self.n_scenes, self.n_curves, self.n_keys, self.n_taus
        c.height, c.width, c.channels = self.height, self.width, self.channels
        c.scene_curve_offset = _ptr(self.scene_curve_offset)
        c.degree, c.flags = _ptr(self.degree), _ptr(self.flags)
        c.key_offset, c.tau_offset = _ptr(self.key_offset), _ptr(self.tau_offset)
        c.key, c.tau, c.color = _ptr(key), _ptr(tau), _ptr(color)
        c.stroke_degrees = self.stroke_degrees
        return c


class Splatter:
    """Buffers and calls for one scene batch: nurbs_sample -> splat_forward ->
    splat_backward on a shared workspace.  Capacities grow to the sizes the
    library reports (`fit`); after that a step enqueues only kernels (no host
    synchronisation), so it can be captured in a CUDA graph."""

    def __init__(self, scene, sample=None, raster=None, capacity=(1 << 16, 1 << 17, 1 << 12), device="cuda"):
        self.dev = DeviceCurves(scene, device)
        self.device = device
        self.sp = sample_params(sample or scene.sample)
        self.rp = raster_params(raster or scene.raster)
        if "fill_cull" not in (sample or scene.sample):
            # fill points that cannot reach the rasterizer's alpha_min need no exact SDF
            self.sp.fill_cull = float(self.rp.alpha_min)
        self.cap = B.NsCapacity(*[int(x) for x in capacity])
        self.image = torch.empty(scene.n_scenes, scene.height, scene.width, scene.channels, device=device)
        self._alloc()

    def _alloc(self):
        lib = B.load()
        G = max(int(self.cap.gaussians), 1)
        self.rec = torch.empty(G, 4, device=self.device)
        self.curve = torch.empty(G, dtype=torch.int32, device=self.device)
        self.aux = torch.empty(G, dtype=torch.int32, device=self.device)
        self.count = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.aniso = int(self.sp.contour_mode) == 1
        self.shape = torch.empty(G, 4, device=self.device) if self.aniso else None
        self.dgauss = torch.empty(G, 12 if self.aniso else 8, device=self.device)
        cs = self.dev.struct_sizes()
        n = lib.ns_workspace_size(C.byref(cs), C.byref(self.cap), C.byref(self.rp))
        if n == 0:
            raise B.NsError("ns_workspace_size", B.NS_ERR_INVALID_ARG, lib.ns_last_error().decode())
        self.ws = torch.empty(n, dtype=torch.uint8, device=self.device)
        self.g = B.NsGaussians(int(self.cap.gaussians), _ptr(self.rec), _ptr(self.curve), _ptr(self.aux),
                               _ptr(self.count), _ptr(self.shape))
        B.call("ns_clear_status", _ptr(self.ws), _stream())

    @property
    def ws_bytes(self):
        return self.ws.numel()

    def report(self) -> Report:
        r = B.NsReport()
        B.call("ns_poll_status", _ptr(self.ws), C.byref(r), _stream())
        return Report(r.status, r.bad_curve, r.gaussians, r.pairs, r.boundary, r.fill_culled, r.blend_evals,
                      r.blend_bwd_evals, r.blend_contribs, r.blend_visits, r.blend_bwd_visits)

    # -- stages ---------------------------------------------------------
    def sample(self, key, tau, color):
        cs = self.dev.struct(key, tau, color)
        B.call("nurbs_sample", C.byref(cs), C.byref(self.sp), C.byref(self.cap), C.byref(self.g),
               _ptr(self.ws), C.c_size_t(self.ws_bytes), _stream())

    def forward_gaussians(self, key, tau, color, image=None):
        cs = self.dev.struct(key, tau, color)
        img = self.image if image is None else image
        B.call("splat_forward", C.byref(cs), C.byref(self.g), C.byref(self.rp), C.byref(self.cap), _ptr(img),
               _ptr(self.ws), C.c_size_t(self.ws_bytes), _stream())
        return img

    def forward(self, key, tau, color, image=None):
        self.sample(key, tau, color)
        return self.forward_gaussians(key, tau, color, image)

    @staticmethod
    def frozen_bits(frozen):
        """("weights", "knots") -> NS_FROZEN_* bits (the paper's ablation variants)."""
        bits = {"weights": B.NS_FROZEN_WEIGHTS, "knots": B.NS_FROZEN_KNOTS}
        return sum(bits[f] for f in set(frozen))

    def backward(self, key, tau, color, dimage, grads=None, chain=True, frozen=(), rows=False):
        """splat_backward; frozen may name "weights" and/or "knots": their
        gradients are not formed (dtau is left untouched for frozen knots).
        rows=True also writes every per-Gaussian gradient row to self.dgauss
        alongside the chain."""
        cs = self.dev.struct(key, tau, color)
        if grads is None:
            grads = (torch.empty_like(key), torch.empty_like(tau), torch.empty_like(color))
        out = B.NsCurveGrads(_ptr(grads[0]), None if "knots" in frozen else _ptr(grads[1]), _ptr(grads[2]),
                             self.frozen_bits(frozen)) if chain else None
        # per-Gaussian gradients (rows {dmu_x, dmu_y, dsigma, 0, do, dr, dg, db}) go
        # to self.dgauss when no chain is asked for; with the chain the workspace
        # holds them and the library skips what the chain does not use
        B.call("splat_backward", C.byref(cs), C.byref(self.g), C.byref(self.sp), C.byref(self.rp),
               C.byref(self.cap), _ptr(dimage.contiguous()), _ptr(self.dgauss) if (rows or not chain) else None,
               C.byref(out) if out is not None else None, C.c_int32(1), _ptr(self.ws),
               C.c_size_t(self.ws_bytes), _stream())
        return grads

    def geometry(self, key, tau, color, loss, grads=None, lambda_deriv=1.0, order=3, nodes=0, lambda_bbox=5.0,
                 penalty="relu", box=None, frozen=()):
        """Geometric regularisers (Eq. 11 derivative loss, Eq. 12 box loss) on the
        plan of the last sample() (ns_geometry_loss).  loss: device float[2],
        overwritten with the weighted terms; grads: (dkey, dtau, ...) device
        tensors the gradients are ADDED to, or None for the values only.
        Default weights: Table S1's calligraphy setting (1 and 5).
        box: (x_min, y_min, x_max, y_max), default the canvas."""
        cs = self.dev.struct(key, tau, color)
        gp = B.NsGeometryParams()
        gp.lambda_deriv, gp.order, gp.nodes, gp.lambda_bbox = lambda_deriv, order, nodes, lambda_bbox
        gp.penalty = {"relu": B.NS_PENALTY_RELU, "softplus": B.NS_PENALTY_SOFTPLUS}[penalty]
        for i, v in enumerate(box or (0.0, 0.0, 0.0, 0.0)):
            gp.box[i] = v
        out = (B.NsCurveGrads(_ptr(grads[0]), None if "knots" in frozen else _ptr(grads[1]), None,
                              self.frozen_bits(frozen)) if grads is not None else None)
        B.call("ns_geometry_loss", C.byref(cs), C.byref(self.g), C.byref(self.sp), C.byref(self.rp), C.byref(gp),
               C.byref(self.cap),
               _ptr(loss), C.byref(out) if out is not None else None, _ptr(self.ws), C.c_size_t(self.ws_bytes),
               _stream())
        return loss

    def udf_mse(self, key, tau, color, image, target, new_curve, tau_w, dimage, loss):
        """Distance-weighted image loss of the layer-wise loop (ns_udf_mse_loss):
        new_curve is a device int32 tensor [n_scenes] naming each scene's new
        filled path (or -1); tau_w the weight radius in pixels."""
        cs = self.dev.struct(key, tau, color)
        B.call("ns_udf_mse_loss", C.byref(cs), C.byref(self.sp), C.byref(self.rp), C.byref(self.cap),
               _ptr(new_curve), C.c_float(tau_w), _ptr(image), _ptr(target), _ptr(dimage), _ptr(loss),
               _ptr(self.ws), C.c_size_t(self.ws_bytes), _stream())
        return loss

    def xing(self, key, tau, color, loss, dkey=None, lam=0.01):
        """Self-crossing penalty of the key-point polygons (ns_xing_loss); its
        gradient is added to dkey when given."""
        cs = self.dev.struct(key, tau, color)
        B.call("ns_xing_loss", C.byref(cs), C.c_float(lam), _ptr(loss), _ptr(dkey), _stream())
        return loss

    def mse(self, image, target, dimage, loss):
        B.call("ns_mse_loss", _ptr(image), _ptr(target), C.c_int64(image.numel()), _ptr(dimage), _ptr(loss),
               _stream())

    def autotune_blend(self, key, tau, color, dimage=None, repeats=3):
        """Let the library time the blend decompositions on this batch and keep
        the fastest (ns_autotune_blend).  Needs a completed forward; synchronises."""
        cs = self.dev.struct(key, tau, color)
        B.call("ns_autotune_blend", C.byref(cs), C.byref(self.g), C.byref(self.rp), C.byref(self.cap),
               _ptr(self.image), _ptr(dimage) if dimage is not None else None, _ptr(self.ws),
               C.c_size_t(self.ws_bytes), C.c_int32(repeats), _stream())
        return int(self.rp.ppt_fwd), int(self.rp.ppt_bwd)

    def adam(self, key, tau, color, grads, state, step, lr=(0.1, 0.01, 0.01), betas=(0.9, 0.999), eps=1e-8,
             frozen=()):
        """One Adam step on key points, knot intervals and colours with the clamps
        of Table S1 (w in [0.01, 10], tau in [0, 2]; widths >= 0; colours and
        opacities in [0, 1]).  `state` holds the moment buffers (made on first use).
        lr: (key, tau, color) learning rates; the key and colour entries may be
        4-tuples, one rate per component ({x, y, s, w}, {r, g, b, o}).
        Frozen knots skip the tau update; frozen weights get no gradient from
        the backward, so with moments that started at zero they stay fixed."""
        inf = float("inf")
        groups = ((key, grads[0], 4, (-inf, -inf, 0.0, 0.01), (inf, inf, inf, 10.0), lr[0]),
                  (tau, grads[1], 1, (0.0,), (2.0,), lr[1]),
                  (color, grads[2], 4, (0.0,) * 4, (1.0,) * 4, lr[2]))
        for i, (p, g, grp, lo, hi, r) in enumerate(groups):
            if i == 1 and "knots" in frozen:
                continue
            if i not in state:
                state[i] = (torch.zeros_like(p), torch.zeros_like(p))
            m, v = state[i]
            rates = tuple(r) if isinstance(r, (tuple, list)) else (float(r),) * grp
            if len(rates) != grp:
                raise ValueError("a per-component learning rate needs one value per component")
            B.call("ns_adam_step", _ptr(p), _ptr(g), _ptr(m), _ptr(v), C.c_int64(p.numel()), C.c_float(1.0),
                   C.c_float(betas[0]), C.c_float(betas[1]), C.c_float(eps), C.c_int32(step),
                   (C.c_float * grp)(*lo), (C.c_float * grp)(*hi), C.c_int32(grp), (C.c_float * grp)(*rates),
                   _stream())

    # -- sizing ---------------------------------------------------------
    def fit(self, key, tau, color, headroom=1.25, max_rounds=4):
        """Run sample + forward, read the sizes the library needed, and grow
        the capacities until nothing overflows.  Synchronises."""
        for _ in range(max_rounds):
            self.forward(key, tau, color)
            r = self.report()
            if r.status not in (B.NS_OK, B.NS_ERR_CAPACITY):
                raise B.NsError("nurbs_sample/splat_forward", r.status,
                                f"device status {B.STATUS_NAMES.get(r.status)} (bad curve {r.bad_curve})")
            need = (r.gaussians, r.pairs, r.boundary)
            have = (self.cap.gaussians, self.cap.pairs, self.cap.boundary)
            if r.status == B.NS_OK and all(n <= h for n, h in zip(need, have)):
                return r
            self.cap = B.NsCapacity(*[max(h, int(n * headroom) + 1) for n, h in zip(need, have)])
            self._alloc()
        raise RuntimeError("capacities did not converge")

    def workspace_array(self, which, nbytes, dtype):
        out = torch.empty(nbytes // torch.empty(0, dtype=dtype).element_size(), dtype=dtype, device=self.device)
        cs = self.dev.struct(*self._last) if hasattr(self, "_last") else None
        if cs is None:
            raise RuntimeError("call remember() with the key/tau/color tensors first")
        B.call("ns_workspace_copy", _ptr(self.ws), C.byref(cs), C.byref(self.cap), C.byref(self.rp),
               C.c_int32(which), _ptr(out), C.c_size_t(nbytes), _stream())
        return out

    def remember(self, key, tau, color):
        self._last = (key, tau, color)


class NurbsSplatFunction(torch.autograd.Function):
    """image = NurbsSplatFunction.apply(key, tau, color, splatter); the backward
    runs splat_backward and returns gradients for key, tau and color."""

    @staticmethod
    def forward(ctx, key, tau, color, splatter):
        img = splatter.forward(key, tau, color, image=torch.empty_like(splatter.image))
        ctx.splatter = splatter
        ctx.save_for_backward(key, tau, color)
        return img

    @staticmethod
    def backward(ctx, dimage):
        key, tau, color = ctx.saved_tensors
        dk, dt, dc = ctx.splatter.backward(key, tau, color, dimage.contiguous())
        return dk, dt, dc, None


def seed_windows(image, target, radius, scratch=None):
    """Per scene the pixel whose (2 radius + 1)^2 window holds the largest
    squared error (ns_seed_windows): returns (xy int32 [S, 2], value [S]) on the
    device."""
    S, H, W, Cc = image.shape
    lib = B.load()
    n = lib.ns_seed_scratch_size(S, H, W)
    if scratch is None or scratch.numel() < n:
        scratch = torch.empty(n, dtype=torch.uint8, device=image.device)
    xy = torch.empty(S, 2, dtype=torch.int32, device=image.device)
    val = torch.empty(S, device=image.device)
    B.call("ns_seed_windows", _ptr(image.contiguous()), _ptr(target.contiguous()), C.c_int32(S), C.c_int32(H),
           C.c_int32(W), C.c_int32(Cc), C.c_int32(radius), _ptr(scratch), C.c_size_t(scratch.numel()), _ptr(xy),
           _ptr(val), _stream())
    return xy, val


def scene_tensors(scene, device="cuda"):
    """The learnable inputs of a scene as contiguous float32 device tensors."""
    k = torch.as_tensor(scene.key, device=device).reshape(-1).contiguous()
    t = torch.as_tensor(scene.tau, device=device).contiguous()
    c = torch.as_tensor(scene.color, device=device).reshape(-1).contiguous()
    return k, t, c
