"""Layer-wise image vectorisation with NURBS Splatting (§4.2, the LIVE
adaptation): paths are added one round at a time, each started at the window
of largest reconstruction error, and all paths are then optimised with Adam
against a distance-weighted image loss plus the self-crossing penalty (Eq. 15),
with the fill grid step annealed from coarse to fine within each round
(Eq. 14).

Everything per iteration runs in the library's kernels: sampling, splatting,
the losses and their gradients, the backward chain and Adam.  This module only
keeps the curve tables of the growing batch on the host and issues the calls.

Readings (the paper gives the loop's ingredients, not all its settings):
  - A new path is a closed, filled degree-3 curve with 12 key points evenly on
    a circle of radius r0 around the seed pixel (§5's LIVE set-up), unit
    weights and knot intervals, the target's colour at the seed and opacity 1.
  - r0 defaults to 5 % of the shorter image side; the seed window has the same
    radius.
  - The learning rates (2.0 for positions, 0.01 for the rest, §5) decay
    exponentially to 0.4 times their start over a round's iterations.
  - The derivative loss is off by default, as in the paper's LIVE experiment
    (degree 3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from . import binding as B
from .splat import Splatter, seed_windows

CLOSED, FILLED = 1, 2


@dataclass
class CurveBatch:
    """Host copy of a batch's curve tables, in the layout the library reads."""
    n_scenes: int
    height: int
    width: int
    channels: int
    sample: dict
    raster: dict
    curves: list = field(default_factory=list)   # per scene: list of (p, key [n,4], tau [n], color [4], flags)

    def pack(self):
        degree, flags, keys, taus, colors, sco = [], [], [], [], [], [0]
        for s in range(self.n_scenes):
            for (p, key, tau, color, fl) in self.curves[s]:
                degree.append(p)
                flags.append(fl)
                keys.append(np.asarray(key, np.float32).reshape(-1, 4))
                taus.append(np.asarray(tau, np.float32).reshape(-1))
                colors.append(np.asarray(color, np.float32).reshape(4))
            sco.append(len(degree))
        self.degree = np.asarray(degree, np.int32)
        self.flags = np.asarray(flags, np.int32)
        self.scene_curve_offset = np.asarray(sco, np.int32)
        self.key_offset = np.r_[0, np.cumsum([k.shape[0] for k in keys])].astype(np.int32)
        self.tau_offset = np.r_[0, np.cumsum([t.shape[0] for t in taus])].astype(np.int32)
        self.key = np.concatenate(keys) if keys else np.zeros((0, 4), np.float32)
        self.tau = np.concatenate(taus) if taus else np.zeros(0, np.float32)
        self.color = np.stack(colors) if colors else np.zeros((0, 4), np.float32)
        return self

    @property
    def n_curves(self):
        return int(self.degree.shape[0])


def circle_path(cx, cy, r, color, n_keys=12, degree=3, width=1.0):
    """Key points evenly on a circle (counter-clockwise), unit weights and
    intervals: a closed filled path."""
    a = 2 * math.pi * np.arange(n_keys) / n_keys
    key = np.stack([cx + r * np.cos(a), cy + r * np.sin(a), np.full(n_keys, width), np.ones(n_keys)], 1)
    return (degree, key, np.ones(n_keys), np.r_[np.asarray(color, np.float64)[:3], 1.0], CLOSED | FILLED)


class LayerwiseVectorizer:
    """The LIVE-style loop on a batch of targets [S, H, W, C] (float32)."""

    def __init__(self, target, sample, raster, rounds=10, iters=300, r0=None, tau_udf=10.0, lambda_xing=0.01,
                 lambda_deriv=0.0, h_max=4.0, h_min=1.0, t_b=0.1, t_e=0.8,
                 lr=((2.0, 2.0, 0.01, 0.01), 0.01, 0.01), lr_end=0.4,
                 capacity=(1 << 18, 1 << 20, 1 << 14)):
        self.target = torch.as_tensor(np.ascontiguousarray(target, np.float32), device="cuda")
        S, H, W, Cc = self.target.shape
        self.batch = CurveBatch(S, H, W, Cc, dict(sample), dict(raster), [[] for _ in range(S)])
        self.rounds, self.iters = rounds, iters
        self.r0 = r0 or max(3.0, round(0.05 * min(H, W)))
        self.tau_udf, self.lambda_xing, self.lambda_deriv = tau_udf, lambda_xing, lambda_deriv
        self.sched = (h_max, h_min, t_b, t_e)
        self.lr, self.lr_end = lr, lr_end
        self.capacity = capacity
        self.sp = None
        self.losses = []

    # -- one round --------------------------------------------------------
    def _device_params(self):
        b = self.batch
        return (torch.as_tensor(b.key, device="cuda").reshape(-1).contiguous(),
                torch.as_tensor(b.tau, device="cuda").contiguous(),
                torch.as_tensor(b.color, device="cuda").reshape(-1).contiguous())

    def _pull(self, k, t, c):
        """Copy the optimised parameters back into the host tables."""
        kh = k.view(-1, 4).cpu().numpy()
        th = t.cpu().numpy()
        ch = c.view(-1, 4).cpu().numpy()
        i = 0
        for s in range(self.batch.n_scenes):
            for j, (p, key, tau, color, fl) in enumerate(self.batch.curves[s]):
                k0, k1 = self.batch.key_offset[i], self.batch.key_offset[i + 1]
                t0, t1 = self.batch.tau_offset[i], self.batch.tau_offset[i + 1]
                self.batch.curves[s][j] = (p, kh[k0:k1].copy(), th[t0:t1].copy(), ch[i].copy(), fl)
                i += 1

    def add_paths(self, image):
        """Seed one new path per scene at its largest-error window."""
        xy, _ = seed_windows(image, self.target, int(self.r0))
        xy = xy.cpu().numpy()
        tgt = self.target.cpu().numpy()
        for s in range(self.batch.n_scenes):
            x, y = int(xy[s, 0]), int(xy[s, 1])
            col = tgt[s, y, x]
            col = np.r_[col, [col[0]] * (3 - len(col))] if len(col) < 3 else col[:3]
            self.batch.curves[s].append(circle_path(x + 0.5, y + 0.5, self.r0, col))
        self.batch.pack()
        # the index of each scene's new path: the last curve of the scene
        return np.asarray(self.batch.scene_curve_offset[1:] - 1, np.int32)

    def prepare(self, new_curve):
        """Device tables, buffers sized at the finest grid step, loss buffers."""
        b = self.batch
        self.params = self._device_params()
        k, t, c = self.params
        self.sp = Splatter(b, capacity=self.capacity)
        self.sp.sp.h = float(self.sched[1])
        self.sp.fit(k, t, c)
        self.newc = torch.as_tensor(new_curve, dtype=torch.int32, device="cuda")
        self.image = torch.empty_like(self.target)
        self.dimage = torch.empty_like(self.target)
        self.loss = torch.zeros(1, device="cuda")
        self.xloss = torch.zeros(1, device="cuda")
        self.geo_loss = torch.zeros(2, device="cuda")
        self.grads = (torch.empty_like(k), torch.empty_like(t), torch.empty_like(c))
        self.state = {}

    def iterate(self):
        """The round's iterations (all on the device, no host synchronisation)."""
        lib = B.load()
        k, t, c = self.params
        h_max, h_min, t_b, t_e = self.sched
        T = self.iters
        for it in range(T):
            self.sp.sp.h = float(lib.ns_grid_step(it, T, h_max, h_min, t_b, t_e))
            self.sp.sample(k, t, c)
            self.sp.forward_gaussians(k, t, c, self.image)
            self.sp.udf_mse(k, t, c, self.image, self.target, self.newc, self.tau_udf, self.dimage, self.loss)
            self.sp.backward(k, t, c, self.dimage, grads=self.grads)
            if self.lambda_xing:
                self.sp.xing(k, t, c, self.xloss, self.grads[0], self.lambda_xing)
            if self.lambda_deriv:
                self.sp.geometry(k, t, c, self.geo_loss, self.grads, lambda_deriv=self.lambda_deriv,
                                 lambda_bbox=0.0)
            decay = self.lr_end ** (it / max(1, T - 1))
            lr = tuple(tuple(y * decay for y in x) if isinstance(x, tuple) else x * decay for x in self.lr)
            self.sp.adam(k, t, c, self.grads, self.state, it + 1, lr=lr)

    def finish(self):
        """Record the round's last loss and copy the parameters to the host."""
        self.losses.append(float(self.loss.item()))
        self._pull(*self.params)
        return self.image

    def optimise(self, new_curve):
        self.prepare(new_curve)
        self.iterate()
        return self.finish()

    def run(self):
        bg = torch.as_tensor(list(self.batch.raster.get("bg", (1.0, 1.0, 1.0)))[:self.batch.channels],
                             dtype=torch.float32, device="cuda")
        image = bg.expand_as(self.target).contiguous()   # the empty canvas
        for _ in range(self.rounds):
            new_curve = self.add_paths(image)
            image = self.optimise(new_curve)
        return image
