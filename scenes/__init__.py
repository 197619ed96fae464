"""Seeded synthetic scene generators shared by the oracle and the CUDA path.

This module only draws inputs: key points, rational weights, knot intervals,
widths, colours, opacities, target images and the per-call settings.  It holds
none of the method's arithmetic (no basis functions, no sampling, no
compositing), so that both implementations can consume the same inputs without
sharing code.

The paper's datasets (calligraphy fonts, emoji sets, SLDVec initialisations) are
not available; the five workloads below stand in for their shapes, sizes and
distributions (stroke lengths, control-net lengths, degrees, closed/filled mix,
lognormal shape sizes).  No dataset item is reproduced.

Layout (all arrays little-endian, C-contiguous):
  scene_curve_offset int32 [S+1]   curves of scene s are [off[s], off[s+1]),
                                   listed back to front (painter's order: a
                                   later curve is drawn over an earlier one)
  degree      int32 [nc]           p in 1..5
  flags       int32 [nc]           bit0 CLOSED, bit1 FILLED (FILLED implies CLOSED)
  key_offset  int32 [nc+1]         CSR into key
  tau_offset  int32 [nc+1]         CSR into tau (open: n_k - p entries, closed: n_k)
  key         float32 [nk, 4]      key point {x, y, width s, weight w} in pixels
  tau         float32 [nt]         knot intervals
  color       float32 [nc, 4]      {r, g, b, opacity}; a C-channel image uses
                                   the first C colour components
  target      float32 [S, H, W, C] target image for the L2 loss
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FLAG_CLOSED = 1
FLAG_FILLED = 2

# Default settings, Table S1 of the paper (symbols and defaults) plus the
# readings the paper leaves open (pad fraction, thresholds, tile size).
SAMPLE_DEFAULTS = dict(
    delta_c=10.0,     # contour density, samples per pixel of arc length
    rho=2.0,          # global Gaussian scale ratio
    kappa=4,          # endpoint replication count
    nl_mult=3,        # N_L = nl_mult * max(W, H) arc-length quadrature samples
    delta_b=0.5,      # boundary sample density
    h=1.0,            # fill grid step in pixels
    eta=1.5,          # fill coverage factor
    gamma=5.0,        # SDF sigmoid sharpness
    pad_frac=0.1,     # bounding-box padding as a fraction of the extent
    fill_rule=0,      # 0: inside iff winding number > 0.5 (paper), 1: nonzero
)
RASTER_DEFAULTS = dict(
    tile=16,
    k_sigma=3.5,
    alpha_min=1.0 / 255.0,
    alpha_max=0.99,
    t_min=1e-4,
    bg=(1.0, 1.0, 1.0),
)
# Thresholds under which FP32 and FP64 renders are comparable at 1e-5: no alpha
# skip, a negligible termination threshold and a 6-sigma tile cutoff.
RASTER_PARITY = dict(RASTER_DEFAULTS, k_sigma=6.0, alpha_min=0.0, t_min=1e-7)


@dataclasses.dataclass
class Scene:
    name: str
    n_scenes: int
    height: int
    width: int
    channels: int
    scene_curve_offset: np.ndarray
    degree: np.ndarray
    flags: np.ndarray
    key_offset: np.ndarray
    tau_offset: np.ndarray
    key: np.ndarray
    tau: np.ndarray
    color: np.ndarray
    target: np.ndarray
    sample: dict
    raster: dict

    @property
    def n_curves(self) -> int:
        return int(self.degree.shape[0])

    def curve_scene(self) -> np.ndarray:
        out = np.zeros(self.n_curves, np.int32)
        for s in range(self.n_scenes):
            out[self.scene_curve_offset[s]:self.scene_curve_offset[s + 1]] = s
        return out

    def with_raster(self, **kw) -> "Scene":
        return dataclasses.replace(self, raster=dict(self.raster, **kw))

    def with_sample(self, **kw) -> "Scene":
        return dataclasses.replace(self, sample=dict(self.sample, **kw))

    def subset(self, scene_ids) -> "Scene":
        """A new batch holding only the listed scenes (re-packed CSR)."""
        b = _Builder(len(scene_ids), self.height, self.width, self.channels)
        for new_s, s in enumerate(scene_ids):
            for c in range(self.scene_curve_offset[s], self.scene_curve_offset[s + 1]):
                k0, k1 = self.key_offset[c], self.key_offset[c + 1]
                t0, t1 = self.tau_offset[c], self.tau_offset[c + 1]
                b.add(new_s, int(self.degree[c]), self.key[k0:k1], self.tau[t0:t1],
                      self.color[c], bool(self.flags[c] & FLAG_CLOSED),
                      bool(self.flags[c] & FLAG_FILLED))
        tgt = self.target[list(scene_ids)]
        return b.build(self.name + "-subset", tgt, dict(self.sample), dict(self.raster))


class _Builder:
    def __init__(self, n_scenes, height, width, channels):
        self.S, self.H, self.W, self.C = n_scenes, height, width, channels
        self.scene_of = []
        self.degree, self.flags, self.keys, self.taus, self.colors = [], [], [], [], []

    def add(self, scene, p, key, tau, color, closed, filled):
        key = np.asarray(key, np.float32).reshape(-1, 4)
        tau = np.asarray(tau, np.float32).reshape(-1)
        nk = key.shape[0]
        need = nk if closed else nk - p
        if tau.shape[0] != need:
            raise ValueError(f"curve with {nk} key points, degree {p}, closed={closed} "
                             f"needs {need} knot intervals, got {tau.shape[0]}")
        if self.scene_of and scene < self.scene_of[-1]:
            raise ValueError("curves must be added scene by scene")
        self.scene_of.append(scene)
        self.degree.append(p)
        self.flags.append((FLAG_CLOSED if closed else 0) | (FLAG_FILLED if filled else 0))
        self.keys.append(key)
        self.taus.append(tau)
        self.colors.append(np.asarray(color, np.float32).reshape(4))

    def build(self, name, target, sample, raster) -> Scene:
        nc = len(self.degree)
        sco = np.zeros(self.S + 1, np.int32)
        for s in self.scene_of:
            sco[s + 1] += 1
        sco = np.cumsum(sco).astype(np.int32)
        ko = np.zeros(nc + 1, np.int32)
        to = np.zeros(nc + 1, np.int32)
        ko[1:] = np.cumsum([k.shape[0] for k in self.keys])
        to[1:] = np.cumsum([t.shape[0] for t in self.taus])
        key = np.concatenate(self.keys) if nc else np.zeros((0, 4), np.float32)
        tau = np.concatenate(self.taus) if nc else np.zeros(0, np.float32)
        color = np.stack(self.colors) if nc else np.zeros((0, 4), np.float32)
        return Scene(name, self.S, self.H, self.W, self.C, sco,
                     np.asarray(self.degree, np.int32), np.asarray(self.flags, np.int32),
                     ko, to, np.ascontiguousarray(key, np.float32), np.ascontiguousarray(tau, np.float32),
                     np.ascontiguousarray(color, np.float32),
                     np.ascontiguousarray(target, np.float32), sample, raster)


# ----------------------------------------------------------------------------
# shape helpers (plain geometry of the inputs)

def circle_keys(cx, cy, r, width=2.0):
    """Eight key points of a closed quadratic circle, starting at a weight-1 edge
    midpoint and going counter-clockwise (positive signed area): edge midpoints
    carry weight 1, square corners weight sqrt(2)/2.  With core knot intervals
    [0, 1, 0, 1, ...] the closed periodic construction of the paper reproduces
    the circle exactly."""
    pts = []
    for q in range(4):
        a = q * 0.5 * math.pi
        pts.append((cx + r * math.cos(a), cy + r * math.sin(a), width, 1.0))
        a2 = a + 0.25 * math.pi
        pts.append((cx + r * math.sqrt(2.0) * math.cos(a2), cy + r * math.sqrt(2.0) * math.sin(a2),
                    width, math.sqrt(2.0) / 2.0))
    return np.asarray(pts, np.float64)


def circle_tau(scale=1.0):
    return np.asarray([0.0, 1.0] * 4, np.float64) * scale


def _affine(keys, A, c):
    """Apply x -> A (x - c) + c to the positions (NURBS are affine invariant)."""
    out = keys.copy()
    xy = keys[:, :2] - c
    out[:, :2] = xy @ A.T + c
    return out


def star_keys(rng, cx, cy, r, n, width_lo=2.0, width_hi=2.0, jitter=0.2):
    """Star-shaped closed control polygon around (cx, cy), counter-clockwise."""
    th = 2 * math.pi * (np.arange(n) + rng.uniform(-0.3, 0.3, n)) / n
    rad = r * np.exp(jitter * rng.standard_normal(n))
    rad = np.clip(rad, 0.5 * r, 1.6 * r)
    x = cx + rad * np.cos(th)
    y = cy + rad * np.sin(th)
    s = rng.uniform(width_lo, width_hi, n)
    w = rng.uniform(0.5, 2.0, n)
    return np.stack([x, y, s, w], 1)


def blob_target(rng, n_scenes, H, W, C, n_blobs=24):
    """Target images: a white canvas with soft coloured blobs."""
    yy, xx = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    out = np.ones((n_scenes, H, W, C), np.float32)
    for s in range(n_scenes):
        img = np.ones((H, W, C), np.float64)
        for _ in range(n_blobs):
            mx, my = rng.uniform(0, W), rng.uniform(0, H)
            sd = rng.uniform(0.03, 0.12) * max(W, H)
            a = 0.8 * np.exp(-((xx - mx) ** 2 + (yy - my) ** 2) / (2 * sd * sd))
            col = rng.uniform(0, 1, C)
            img = img * (1 - a[..., None]) + a[..., None] * col
        out[s] = img.astype(np.float32)
    return out


# ----------------------------------------------------------------------------
# the five workloads

def config1(seed=1001):
    """Single open cubic NURBS, 8 key points uniform in a 64x64 canvas, weights
    U[0.5, 2], knot intervals U[0.5, 1.5], width 2 px, opacity 0.9, 64x64 RGB.
    Contour density 1 sample/px gives the ~200-Gaussian workload."""
    rng = np.random.default_rng(seed)
    H = W = 64
    b = _Builder(1, H, W, 3)
    nk, p = 8, 3
    key = np.zeros((nk, 4))
    key[:, 0] = rng.uniform(4, 60, nk)
    key[:, 1] = rng.uniform(4, 60, nk)
    key[:, 2] = 2.0
    key[:, 3] = rng.uniform(0.5, 2.0, nk)
    tau = rng.uniform(0.5, 1.5, nk - p)
    col = np.r_[rng.uniform(0, 1, 3), 0.9]
    b.add(0, p, key, tau, col, False, False)
    tgt = blob_target(rng, 1, H, W, 3, 8)
    return b.build("open-cubic-64", tgt, dict(SAMPLE_DEFAULTS, delta_c=1.0), dict(RASTER_DEFAULTS))


def config2(seed=1002, n_paths=16, size=256, h=2.0):
    """16 closed filled paths at 256x256 RGB: 8 exact quadratic circles/ellipses
    (weights 1, sqrt(2)/2), 8 cubic star shapes with 6-16 key points, fill grid
    step 2 px (~50k Gaussians)."""
    rng = np.random.default_rng(seed)
    H = W = size
    b = _Builder(1, H, W, 3)
    for i in range(n_paths):
        cx, cy = rng.uniform(0.2 * W, 0.8 * W), rng.uniform(0.2 * H, 0.8 * H)
        r = rng.uniform(0.14, 0.22) * size
        col = np.r_[rng.uniform(0, 1, 3), rng.uniform(0.7, 1.0)]
        if i % 2 == 0:
            k = circle_keys(cx, cy, r)
            th = rng.uniform(0, math.pi)
            R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
            D = np.diag([1.0, rng.uniform(0.6, 1.0)])
            k = _affine(k, R @ D @ R.T, np.array([cx, cy]))
            b.add(0, 2, k, circle_tau(rng.uniform(0.5, 1.5)), col, True, True)
        else:
            n = int(rng.integers(6, 17))
            k = star_keys(rng, cx, cy, r, n)
            b.add(0, 3, k, rng.uniform(0.5, 1.5, n), col, True, True)
    tgt = blob_target(rng, 1, H, W, 3)
    return b.build("filled-16-256", tgt, dict(SAMPLE_DEFAULTS, h=h), dict(RASTER_DEFAULTS))


def _random_walk(rng, n, length, W, H, turn=0.3):
    step = length / max(n - 1, 1)
    x, y = rng.uniform(0.2 * W, 0.8 * W), rng.uniform(0.2 * H, 0.8 * H)
    th = rng.uniform(0, 2 * math.pi)
    pts = np.zeros((n, 2))
    for i in range(n):
        pts[i] = x, y
        th += turn * rng.standard_normal()
        nx, ny = x + step * math.cos(th), y + step * math.sin(th)
        if not (2 <= nx <= W - 2):
            th = math.pi - th
            nx = x + step * math.cos(th)
        if not (2 <= ny <= H - 2):
            th = -th
            ny = y + step * math.sin(th)
        x, y = min(max(nx, 2), W - 2), min(max(ny, 2), H - 2)
    return pts


def config3(seed=1003, n_strokes=256, size=512, total_length=150_000.0, nk_lo=64, nk_hi=512):
    """Long-spline abstraction: 256 open cubic strokes with 64-512 key points,
    smooth random walks, widths U[0.5, 4] px, weights U[0.5, 2], 512x512
    grayscale; total control-polygon length ~150k px so that ~1.5M contour
    Gaussians come out at delta_c = 10."""
    rng = np.random.default_rng(seed)
    H = W = size
    b = _Builder(1, H, W, 1)
    nks = rng.integers(nk_lo, nk_hi + 1, n_strokes)
    lens = total_length * nks / nks.sum()
    for i in range(n_strokes):
        nk = int(nks[i])
        xy = _random_walk(rng, nk, lens[i], W, H)
        key = np.zeros((nk, 4))
        key[:, :2] = xy
        key[:, 2] = rng.uniform(0.5, 4.0, nk)
        key[:, 3] = rng.uniform(0.5, 2.0, nk)
        col = np.r_[np.full(3, rng.uniform(0, 0.6)), rng.uniform(0.6, 1.0)]
        b.add(0, 3, key, rng.uniform(0.5, 1.5, nk - 3), col, False, False)
    tgt = blob_target(rng, 1, H, W, 1, 64)
    return b.build("long-spline-512", tgt, dict(SAMPLE_DEFAULTS), dict(RASTER_DEFAULTS))


def _closed_path(rng, b, scene, cx, cy, r, p, nk, filled, width_lo, width_hi):
    if p == 2 and nk == 8 and rng.uniform() < 0.5:
        k = circle_keys(cx, cy, r, width=rng.uniform(width_lo, width_hi))
        tau = circle_tau(rng.uniform(0.5, 1.5))
    else:
        k = star_keys(rng, cx, cy, r, nk, width_lo, width_hi)
        tau = rng.uniform(0.5, 1.5, nk)
    col = np.r_[rng.uniform(0, 1, 3), rng.uniform(0.7, 1.0)]
    b.add(scene, p, k, tau, col, True, filled)


def config4(seed=1004, n_scenes=64, size=256):
    """Batched calligraphy-like scenes: 64 scenes of 256x256 RGB, each with 1-40
    closed paths (p = 2-4, 8-48 key points, lognormal radius with median 20 px);
    half filled at h = 1, half variable-width closed strokes."""
    rng = np.random.default_rng(seed)
    H = W = size
    b = _Builder(n_scenes, H, W, 3)
    for s in range(n_scenes):
        for _ in range(int(rng.integers(1, 41))):
            p = int(rng.integers(2, 5))
            nk = int(rng.integers(8, 49))
            r = float(np.clip(20.0 * math.exp(0.6 * rng.standard_normal()), 4, 0.45 * size))
            cx, cy = rng.uniform(r, W - r), rng.uniform(r, H - r)
            _closed_path(rng, b, s, cx, cy, r, p, nk, bool(rng.uniform() < 0.5), 0.5, 4.0)
    tgt = blob_target(rng, n_scenes, H, W, 3, 12)
    return b.build("batched-64x256", tgt, dict(SAMPLE_DEFAULTS, h=1.0), dict(RASTER_DEFAULTS))


def config5(seed=1005, n_paths=2048, size=1024, median_r=19.0):
    """Vectorization scale: 1024x1024 RGB, 2048 closed filled paths with
    p in {2,3,4,5} and 8-64 key points, lognormal sizes; ~8M fill Gaussians at
    grid step h = 1 (the step the grid-step annealing schedule ends at)."""
    rng = np.random.default_rng(seed)
    H = W = size
    b = _Builder(1, H, W, 3)
    for _ in range(n_paths):
        p = int(rng.integers(2, 6))
        nk = int(rng.integers(8, 65))
        r = float(np.clip(median_r * math.exp(0.5 * rng.standard_normal()), 5, 0.3 * size))
        cx, cy = rng.uniform(0, W), rng.uniform(0, H)
        _closed_path(rng, b, 0, cx, cy, r, p, nk, True, 2.0, 2.0)
    tgt = blob_target(rng, 1, H, W, 3, 48)
    return b.build("vectorize-2048-1024", tgt, dict(SAMPLE_DEFAULTS, h=1.0), dict(RASTER_DEFAULTS))


CONFIGS = {1: config1, 2: config2, 3: config3, 4: config4, 5: config5}


def grid_step_schedule_inputs(t, T, h_max=4.0, h_min=1.0, t_b=0.1, t_e=0.8):
    """Arguments of the cosine grid-step schedule (Eq. 14): returned unevaluated
    so that each implementation evaluates the schedule itself."""
    return dict(t=t, T=T, h_max=h_max, h_min=h_min, t_b=t_b, t_e=t_e)


def small_open(seed, n_curves=3, size=40, p=3, nk_range=(5, 9), width=(1.5, 3.0), delta_c=2.0,
               channels=3, height=None):
    """Small open-stroke scenes for parity tests (several tiles, ragged edges)."""
    rng = np.random.default_rng(seed)
    H = height or size
    W = size
    b = _Builder(1, H, W, channels)
    for _ in range(n_curves):
        nk = int(rng.integers(nk_range[0], nk_range[1] + 1))
        pc = p if isinstance(p, int) else int(rng.choice(p))
        nk = max(nk, pc + 1)
        key = np.zeros((nk, 4))
        key[:, 0] = rng.uniform(2, W - 2, nk)
        key[:, 1] = rng.uniform(2, H - 2, nk)
        key[:, 2] = rng.uniform(*width, nk)
        key[:, 3] = rng.uniform(0.5, 2.0, nk)
        col = np.r_[rng.uniform(0, 1, 3), rng.uniform(0.6, 0.95)]
        b.add(0, pc, key, rng.uniform(0.5, 1.5, nk - pc), col, False, False)
    tgt = blob_target(rng, 1, H, W, channels, 6)
    return b.build("small-open", tgt, dict(SAMPLE_DEFAULTS, delta_c=delta_c), dict(RASTER_PARITY))


def from_curves(curves, height, width, channels=3, sample=None, raster=None, name="custom"):
    """A one-scene batch from explicit curves: each entry is a dict with keys
    p, key ([n_k, 4] rows {x, y, s, w}), tau, and optionally color, closed,
    filled.  Used by tests that need hand-made inputs."""
    b = _Builder(1, height, width, channels)
    for cv in curves:
        b.add(0, int(cv["p"]), cv["key"], cv["tau"], cv.get("color", (0.2, 0.4, 0.6, 0.9)),
              bool(cv.get("closed", False)), bool(cv.get("filled", False)))
    tgt = np.ones((1, height, width, channels), np.float32)
    return b.build(name, tgt, dict(SAMPLE_DEFAULTS, **(sample or {})), dict(RASTER_PARITY, **(raster or {})))


def small_closed(seed, n_curves=3, size=48, filled=True, h=2.0, degrees=(2, 3, 4, 5), n_scenes=1,
                 width=(1.0, 3.0), height=None):
    """Small closed (filled or stroked) scenes for parity tests; filled =
    "alternate" makes every second path a stroke."""
    rng = np.random.default_rng(seed)
    H = height or size
    W = size
    b = _Builder(n_scenes, H, W, 3)
    for s in range(n_scenes):
        for i in range(n_curves):
            p = int(rng.choice(degrees))
            nk = int(rng.integers(max(p, 6), 12))
            r = rng.uniform(0.15, 0.3) * min(W, H)
            cx, cy = rng.uniform(0.3 * W, 0.7 * W), rng.uniform(0.3 * H, 0.7 * H)
            fill = (i % 2 == 0) if filled == "alternate" else filled
            _closed_path(rng, b, s, cx, cy, r, p, nk, fill, *width)
    tgt = blob_target(rng, n_scenes, H, W, 3, 6)
    return b.build("small-closed", tgt, dict(SAMPLE_DEFAULTS, h=h, delta_c=2.0), dict(RASTER_PARITY))
