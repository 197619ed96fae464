#!/usr/bin/env python
"""Benchmark of the NURBS splatting step: fwd+bwd Gaussians/s.

One step = nurbs_sample -> splat_forward -> L2 loss -> splat_backward (blend
adjoint + chain into key points, knot intervals, colours and opacities) over
one batch of synthetic scenes resident in HBM.  The workload is the 1024x1024
vectorisation-scale scene (2048 closed filled NURBS paths, p in {2..5}, 8-64
key points, fill grid step h = 1, ~8M Gaussians).  The step is captured as a
CUDA graph; the timed region replays one graph holding K steps back to back.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import scenes  # noqa: E402

PEAKS_FALLBACK = dict(hbm_gbs=6400.0, sm_max_mhz=2032.0)

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# one ncu capture per kernel of the 512-path version of the workload at tile 8
# with fill layers, with the units that launch processed and the hash of the
# kernel source it ran.  The bench scales the bytes to its own launch by the
# units processed, and reports null if the source, the tile or the binning has
# changed since the capture.  The plan's entry is the sum of its two kernels
# (knots and span forms, arc lengths).  The fill SDF is left out: at 512 paths
# the records it writes stay in L2, at 2048 they do not, so its traffic does
# not grow in proportion.
TRAFFIC = dict(
    blend_bwd=dict(bytes=57382144, units=2027197, unit="gaussians", tile=8, layers=1,
                   src="paper_2606_31764_b300/csrc/ns_raster.cu", sha="848396ae473232c2"),
    blend_fwd=dict(bytes=27754496, units=2027197, unit="gaussians", tile=8, layers=1,
                   src="paper_2606_31764_b300/csrc/ns_raster.cu", sha="848396ae473232c2"),
    chain=dict(bytes=17374976, units=2027197, unit="gaussians", tile=None, layers=None,
               src="paper_2606_31764_b300/csrc/ns_backward.cu", sha="cbd74131f2f815b2"),
    bin_count=dict(bytes=51200, units=2027197, unit="gaussians", tile=8, layers=1,
                   src="paper_2606_31764_b300/csrc/ns_raster.cu", sha="848396ae473232c2"),
    bin_emit=dict(bytes=52736, units=2027197, unit="gaussians", tile=8, layers=1,
                  src="paper_2606_31764_b300/csrc/ns_raster.cu", sha="848396ae473232c2"),
    plan=dict(bytes=2103040, units=512, unit="curves", tile=None, layers=None,
              src="paper_2606_31764_b300/csrc/ns_sample.cu", sha="317e7b77fbcba6be"),
    boundary=dict(bytes=1277696, units=512, unit="curves", tile=None, layers=None,
                  src="paper_2606_31764_b300/csrc/ns_sample.cu", sha="317e7b77fbcba6be"),
)


def traffic_per_launch(kernel, units_now, tile, layers):
    """Captured DRAM bytes scaled to this launch, or None when stale."""
    import hashlib
    t = TRAFFIC.get(kernel)
    if t is None or (t["tile"] is not None and t["tile"] != tile):
        return None
    if t["layers"] is not None and t["layers"] != int(layers):
        return None
    sha = hashlib.sha256(open(os.path.join(ROOT, t["src"]), "rb").read()).hexdigest()[:16]
    if sha != t["sha"]:
        return None
    return int(round(t["bytes"] * units_now[t["unit"]] / t["units"]))
METRIC = "fwd+bwd Gaussians/s at 1024^2 (batched, graph-captured step)"
FLOP_SEGMENT = 20        # one (grid point, boundary segment) SDF test: distance 14 + crossing 6
FLOP_EVAL = 10           # one alpha evaluation (Eq. 9): dx, dy, d^2, scale, exp arg, *o, cap, skip test
FLOP_CONTRIB_FWD = 10    # composite one pair (Eq. 8), 3 channels
FLOP_CONTRIB_BWD = 33    # adjoint of one composited pair, 3 channels
# Algorithmic cost of one visited (pixel, list entry) pair of Eq. 8-9's loop, FP32
# operations only (the exponential and the reciprocal run on the MUFU pipe):
# forward alpha 8 + compositing 5; backward alpha 8 + division, colour and
# alpha adjoints and the mu, sigma, opacity terms 22.
FLOP_VISIT_FWD = 13
FLOP_VISIT_BWD = 30


def workload_name(paths=2048):
    return (f"vectorize-{paths}-1024: 1024x1024 RGB, {paths} closed filled NURBS paths p in {{2,3,4,5}}, "
            "8-64 key points, fill grid step h=1")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-per-scene", action="store_true")
    ap.add_argument("--paths", type=int, default=2048, help="paths of the 1024x1024 workload (2048 = full)")
    ap.add_argument("--tiles", default="8,16,32", help="tile sizes the autotuner tries (comma separated)")
    ap.add_argument("--fill-layers", default="0,1",
                    help="binnings the autotuner tries: 0 per Gaussian, 1 fill layers (comma separated)")
    ap.add_argument("--cpu-sample-curves", type=int, default=64)
    ap.add_argument("--headline-only", action="store_true",
                    help="profiling runs: only the headline step (no e2e, regulariser or schedule measurements)")
    ap.add_argument("--ref-sample-curves", type=int, default=8)
    ap.add_argument("--ppt", default="",
                    help="profiling runs: fixed blend decompositions 'fwd,bwd' instead of timing them")
    ap.add_argument("--fill-tiles", default="16,8",
                    help="fill tile edges (Gaussians per sampling block: their squares) the autotuner tries")
    return ap.parse_args()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=float(d["hbm_gbs"]), sm_max_mhz=float(d.get("sm_max_mhz", 2032.0)), source="measured")
    return dict(PEAKS_FALLBACK, source="fallback")


# ----------------------------------------------------------------------------
# distributed plumbing (one process per GPU; replicas of independent scenes)

def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
        return dist, rank, ws
    return None, 0, 1


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x):
    if dist is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------
# clocks sampled during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["unavailable"], samples=0)
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["no samples"], samples=0)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return dict(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=sorted(reasons), samples=len(rows))


# ----------------------------------------------------------------------------
# the GPU step

def packed(torch, tensors):
    """One float32 device buffer holding copies of the tensors, each at a
    16-byte aligned offset; returns the buffer and the views."""
    offs, n = [], 0
    for t in tensors:
        offs.append(n)
        n += (t.numel() + 3) // 4 * 4
    buf = torch.zeros(max(n, 4), dtype=torch.float32, device="cuda")
    views = []
    for t, o in zip(tensors, offs):
        v = buf[o:o + t.numel()].view(t.shape)
        v.copy_(t)
        views.append(v)
    return buf, views


class Step:
    """Preallocated buffers and the four calls of one training step."""

    def __init__(self, scene, capacity, raster=None, adam=False, geometry=None, frozen=()):
        import torch
        from paper_2606_31764_b300.splat import Splatter, scene_tensors
        self.torch = torch
        self.scene = scene
        self.adam = adam
        self.geometry = geometry
        self.frozen = tuple(frozen)
        self.adam_state = {}
        self.sp = Splatter(scene, raster=raster, capacity=capacity)
        key, tau, color = scene_tensors(scene)
        # the step's inputs (key points, intervals, colours) are views of one
        # device buffer and its results (gradients, loss) of another, so that
        # a caller moves each with one copy; every view starts on a 16-byte
        # boundary (the kernels read key points and colours as float4)
        self.inbuf, (self.key, self.tau, self.color) = packed(torch, (key, tau, color))
        self.outbuf, (dk, dt, dc, self.loss) = packed(
            torch, (torch.empty_like(key), torch.empty_like(tau), torch.empty_like(color),
                    torch.zeros(1, device="cuda")))
        self.grads = (dk, dt, dc)
        self._in_views = [(v.shape, v.storage_offset()) for v in (self.key, self.tau, self.color)]
        self._out_views = [(v.shape, v.storage_offset()) for v in (dk, dt, dc, self.loss)]
        self.rep = self.sp.fit(self.key, self.tau, self.color)
        self.target = torch.as_tensor(scene.target, device="cuda").contiguous()
        self.image = self.sp.image
        self.dimage = torch.empty_like(self.image)
        self.geo_loss = torch.zeros(2, device="cuda")

    def __call__(self):
        sp = self.sp
        sp.sample(self.key, self.tau, self.color)
        sp.forward_gaussians(self.key, self.tau, self.color, self.image)
        sp.mse(self.image, self.target, self.dimage, self.loss)
        sp.backward(self.key, self.tau, self.color, self.dimage, grads=self.grads, frozen=self.frozen)
        if self.geometry is not None:   # regularisers (Eq. 11-12) add their gradients
            sp.geometry(self.key, self.tau, self.color, self.geo_loss, self.grads, frozen=self.frozen,
                        **self.geometry)
        if self.adam:   # fixed step number: the captured graph replays the same bias correction
            sp.adam(self.key, self.tau, self.color, self.grads, self.adam_state, step=10, frozen=self.frozen)

    def gaussians(self):
        return int(self.sp.count.item())

    def rebind(self, inbuf, outbuf):
        """Point the step's inputs and results at other buffers of the same
        layout (for a second graph of the same step)."""
        def views(buf, spec):
            return [buf.as_strided(shape, buf.new_empty(shape).stride(), off) for shape, off in spec]
        self.inbuf, self.outbuf = inbuf, outbuf
        self.key, self.tau, self.color = views(inbuf, self._in_views)
        dk, dt, dc, self.loss = views(outbuf, self._out_views)
        self.grads = (dk, dt, dc)


def autotune(torch, scene, tiles, capacity, steps=3, adam=False, geometry=None, layers=(0, 1), fill_tiles=(16, 8),
             ppt=None):
    """Tile size and binning (per Gaussian, or fill layers) by timing whole
    steps; the blend decomposition by the library's ns_autotune_blend on each
    candidate's workspace."""
    best, best_ms, table = None, None, {}
    for tile, fl in [(t, f) for t in tiles for f in layers]:
        st = Step(scene, capacity, raster=dict(scene.raster, tile=tile, fill_layers=fl), adam=adam,
                  geometry=geometry)
        st()
        if ppt:
            st.sp.rp.ppt_fwd, st.sp.rp.ppt_bwd = ppt
        else:
            st.sp.autotune_blend(st.key, st.tau, st.color, st.dimage, repeats=3)
        st()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            st()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        rep_t = st.sp.report()
        table[f"{tile}" + ("-layers" if fl else "")] = dict(ms=round(ms, 4), ppt_fwd=int(st.sp.rp.ppt_fwd),
                                                             ppt_bwd=int(st.sp.rp.ppt_bwd), pairs=int(rep_t.pairs),
                                                             visits_fwd=int(rep_t.blend_visits),
                                                             visits_bwd=int(rep_t.blend_bwd_visits))
        if best_ms is None or ms < best_ms:
            if best is not None:
                del best
            best, best_ms = st, ms
        else:
            del st
        torch.cuda.empty_cache()
    chosen = dict(tile=int(best.sp.rp.tile), ppt_fwd=int(best.sp.rp.ppt_fwd), ppt_bwd=int(best.sp.rp.ppt_bwd),
                  fill_layers=int(best.sp.rp.fill_layers), tried=table)
    # Gaussians per sampling block (the fill tile of the SDF and the fill
    # chain) on the chosen raster
    raster = dict(scene.raster, tile=chosen["tile"], fill_layers=chosen["fill_layers"], ppt_fwd=chosen["ppt_fwd"],
                  ppt_bwd=chosen["ppt_bwd"])
    ft_table, best_ft, best_ft_ms = {}, 16, None
    for ft in fill_tiles:
        st = best if ft == 16 else Step(scene.with_sample(fill_tile=ft), capacity, raster=raster, adam=adam,
                                         geometry=geometry)
        if len(fill_tiles) == 1:   # nothing to choose
            best, best_ft = st, ft
            break
        st()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            st()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        ft_table[str(ft * ft)] = round(ms, 4)
        if best_ft_ms is None or ms < best_ft_ms:
            best, best_ft, best_ft_ms = st, ft, ms
        else:
            del st
        torch.cuda.empty_cache()
    chosen["fill_gaussians_per_block"] = best_ft * best_ft
    chosen["tried_fill_gaussians_per_block"] = ft_table
    return best, chosen


def capture(torch, fn, n_steps=1, arm=None):
    """A CUDA graph of n_steps calls of fn; arm(i) arms profiling before step i."""
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for i in range(n_steps):
            if arm is not None:
                arm(i)
            fn()
    return g


def plan_costs(step):
    """Per-step unit counts from the sampling plans: SDF segment tests and
    contour samples."""
    import torch
    sp = step.sp
    nc = step.scene.n_curves
    sp.remember(step.key, step.tau, step.color)
    raw = sp.workspace_array(3, 64 * nc, torch.int32).cpu().numpy().reshape(nc, 16)
    kind, M, cnt = raw[:, 5], raw[:, 6], raw[:, 7]
    fill = kind == 3
    return dict(segment_tests=int((cnt[fill].astype(np.int64) * M[fill]).sum()),
                fill_gaussians=int(cnt[fill].sum()), contour_gaussians=int(cnt[~fill].sum()))


def run_gpu(args, dist, rank, world):
    import torch
    from paper_2606_31764_b300 import binding as B

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    lib = B.load()
    peaks = load_peaks()
    sc = scenes.config5(seed=1005 + rank, n_paths=args.paths)
    step, tuning = autotune(torch, sc, [int(x) for x in args.tiles.split(",")],
                            capacity=(10_000_000, 40_000_000, 400_000),
                            layers=tuple(int(x) for x in args.fill_layers.split(",")),
                            fill_tiles=tuple(int(x) for x in args.fill_tiles.split(",")),
                            ppt=tuple(int(x) for x in args.ppt.split(",")) if args.ppt else None)
    step()
    torch.cuda.synchronize()
    rep = step.sp.report()
    if rep.status != 0:
        raise RuntimeError(f"device status {rep}")
    G = step.gaussians()
    costs = plan_costs(step)

    # kernels per step (counted by the library while one step is enqueued)
    n0 = lib.ns_launch_count()
    step()
    launches_per_step = int(lib.ns_launch_count() - n0)
    g1 = capture(torch, step)
    for _ in range(args.warmup):
        g1.replay()
    torch.cuda.synchronize()

    # per-kernel times: a K-step graph with events around every listed kernel
    # in every step, replayed once outside the timed region (the event nodes
    # cost a few microseconds each); it also names the dominant kernel
    prof = ["plan", "boundary", "fill_sdf", "emit", "bin_count", "bin_emit", "radix_scatter", "ranges", "blend_fwd", "mse", "blend_bwd",
            "chain", "chain_contour", "chain_boundary", "knot_grads"]

    def make_events(names):
        ev = {k: [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)] for k in names}
        for k in names:                 # torch creates the CUDA events on first record
            for a, b in ev[k]:
                a.record()
                b.record()
        torch.cuda.synchronize()
        return ev

    def armer(ev):
        def arm(i):
            for k, pairs in ev.items():
                a, b = pairs[i]
                B.call("ns_profile_next_launch", C.c_int32(B.KERNELS[k]), C.c_void_p(a.cuda_event),
                       C.c_void_p(b.cuda_event))
        return arm

    ev_all = make_events(prof)
    gP = capture(torch, step, args.steps, armer(ev_all))
    lib.ns_profile_next_launch(0, None, None)
    gP.replay()          # warm
    torch.cuda.synchronize()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record()
    gP.replay()
    p1.record()
    torch.cuda.synchronize()
    ms_step_all_events = p0.elapsed_time(p1) / args.steps
    per_kernel = {k: float(np.mean([a.elapsed_time(b) for a, b in ev_all[k]])) for k in prof}
    dom = max(per_kernel, key=per_kernel.get)

    # the timed K-step graph: events around the dominant kernel only (its
    # launch duration inside the timed region gives the roofline)
    ev_dom = make_events([dom])
    gK = capture(torch, step, args.steps, armer(ev_dom))
    lib.ns_profile_next_launch(0, None, None)
    gK.replay()          # warm the K-step graph once
    torch.cuda.synchronize()
    rep = step.sp.report()

    clocks = ClockSampler(torch.cuda.current_device())
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(dist)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0.record()
    gK.replay()
    e1.record()
    torch.cuda.synchronize()
    barrier(dist)
    ck = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    ms_total = max_over_ranks(dist, ms_total)
    ms_step = ms_total / args.steps
    dom_ms_live = float(np.mean([a.elapsed_time(b) for a, b in ev_dom[dom]]))
    value = world * G * args.steps / (ms_total / 1e3)

    # roofline of the dominant kernel
    clk = peaks["sm_max_mhz"] * 1e6
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    fp32_peak = 2.0 * 128 * sms * clk / 1e12        # TFLOP/s, FMA = 2 FLOP
    performed = dict(blend_fwd=(rep.blend_evals * FLOP_EVAL + rep.blend_contribs * FLOP_CONTRIB_FWD) / 1e12,
                     blend_bwd=(rep.blend_bwd_evals * FLOP_EVAL + rep.blend_contribs * FLOP_CONTRIB_BWD) / 1e12)
    layers = bool(step.sp.rp.fill_layers)
    # the blend work is counted per visited (pixel, list entry) pair of Eq. 8-9's
    # loop over the per-Gaussian tile lists.  Fill layers composite the same
    # Gaussians in the same order without such lists; the visits are a property
    # of the lists and the image, so they come from the per-Gaussian kernels'
    # counters in the autotuner's trial at the same tile size (else the FP32
    # work the layer kernels performed is reported)
    pg = tuning["tried"].get(str(int(step.sp.rp.tile)), {}) if layers else {}
    visits_fwd = pg.get("visits_fwd", 0) if layers else rep.blend_visits
    visits_bwd = pg.get("visits_bwd", 0) if layers else rep.blend_bwd_visits
    visit_src = ("per-Gaussian trial at this tile size" if layers else "this step's counters")
    work = dict(
        fill_sdf=("hbm", costs["fill_gaussians"] * 24 / 1e9, "GB/s", peaks["hbm_gbs"]),
        blend_fwd=("alu", visits_fwd * FLOP_VISIT_FWD / 1e12 if visits_fwd else performed["blend_fwd"],
                   "TFLOP/s", fp32_peak),
        blend_bwd=("alu", visits_bwd * FLOP_VISIT_BWD / 1e12 if visits_bwd else performed["blend_bwd"],
                   "TFLOP/s", fp32_peak),
        radix_scatter=("hbm", rep.pairs * 16 / 1e9, "GB/s", peaks["hbm_gbs"]),
        # fill layers: the emission reads the curve of every Gaussian, not its record
        bin_emit=("hbm", ((G * 4 if layers else G * 20) + rep.pairs * 8) / 1e9, "GB/s", peaks["hbm_gbs"]),
    )
    work_text = dict(
        fill_sdf="the fill records written, 24 B per grid point (record, curve, aux); the band performs about "
                 "3 distance tests per grid point where the plain definition (Eq. S1-S2) takes Q x B "
                 f"({costs['segment_tests']} per step, see sample.segment_tests)",
        blend_fwd=(f"algorithmic: {visits_fwd} visited (pixel, list entry) pairs of Eq. 8-9 ({visit_src}) x "
                   f"{FLOP_VISIT_FWD} FP32 FLOP" if visits_fwd else
                   "performed: 10 FP32 FLOP per alpha evaluation + 10 per composited pair (fill layers)"),
        blend_bwd=(f"algorithmic: {visits_bwd} visited (pixel, list entry) pairs of Eq. 8-9 ({visit_src}) x "
                   f"{FLOP_VISIT_BWD} FP32 FLOP" if visits_bwd else
                   "performed: 10 FP32 FLOP per alpha evaluation + 33 per composited pair (fill layers)"),
        radix_scatter="16 B per pair and pass (read + write of key and value)",
        bin_emit="curve ids (fill layers) or records and curve ids read, 8 B per pair written",
    )
    kernels = {}
    for k, ms in per_kernel.items():
        d = dict(ms=round(ms, 4), share_of_step=round(ms / ms_step_all_events, 4))
        if k in work:
            bound, amount, unit, peak = work[k]
            ach = amount / (ms / 1e3)
            d.update(bound=bound, achieved=round(ach, 3), unit=unit, frac=round(ach / peak, 4), work=work_text[k])
        if k in performed:
            # the FLOPs the kernel itself executed (its culling skips most pairs)
            d["performed_frac"] = round(performed[k] / (ms / 1e3) / fp32_peak, 4)
        kernels[k] = d
    units_now = dict(pairs=int(rep.pairs), gaussians=G, curves=sc.n_curves)
    tile_now = int(step.sp.rp.tile)
    for k in kernels:
        kernels[k]["traffic"] = traffic_per_launch(k, units_now, tile_now, layers)
    roof = None
    if dom in work:
        bound, amount, unit, peak = work[dom]
        ach = amount / (dom_ms_live / 1e3)   # its launch duration inside the timed replay
        roof = dict(kernel=dom, ms=round(dom_ms_live, 4), bound=bound, achieved=round(ach, 3), peak=round(peak, 2),
                    unit=unit,
                    frac=round(ach / peak, 4), traffic=traffic_per_launch(dom, units_now, tile_now, layers),
                    peak_source=("FP32 lanes x SMs x max SM clock" if bound == "alu"
                                 else f"{peaks['source']} HBM copy bandwidth"))
        roof["work"] = work_text[dom]
        if dom in performed:
            roof["performed_frac"] = round(performed[dom] / (dom_ms_live / 1e3) / fp32_peak, 4)

    # end to end through the public API with host buffers
    e2e = None if args.headline_only else run_e2e(torch, step, g1, args)

    out = dict(metric=METRIC, value=round(value, 1), unit="Gaussians/s", n_gpus=world, steps=args.steps,
               warmup=args.warmup, ms_per_step=round(ms_step, 4), higher_is_better=True,
               scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
               config=dict(workload=workload_name(args.paths),
                           gaussians_per_step=G, pairs_per_step=int(rep.pairs), curves=sc.n_curves,
                           fill_culled=int(rep.fill_culled),
                           l2=(f"inputs larger than L2 (records+pairs {(G * 32 + rep.pairs * 16) / 1e6:.0f} MB "
                               "> 126 MB)" if G * 32 + rep.pairs * 16 > 126e6 else
                               f"records+pairs {(G * 32 + rep.pairs * 16) / 1e6:.0f} MB fit the 126 MB L2: "
                               "a small case, not the timed workload"),
                           timed="one CUDA-graph replay of K steps", parallelism=f"replicas x{world}"),
               gpu_launches=launches_per_step * args.steps, launches_per_step=launches_per_step,
               autotune=tuning,
               clocks=ck, roofline=roof, kernels=kernels,
               kernel_events=dict(ms_per_step=round(ms_step_all_events, 4),
                                  note="kernels: mean launch times from a second replay of the K-step graph with "
                                       "events around every listed kernel (shares of that replay's step); the "
                                       "timed replay has events around the dominant kernel only"),
               e2e=e2e,
               live_gaussians_per_s=round(world * (G - int(rep.fill_culled)) * args.steps / (ms_total / 1e3), 1),
               blend=blend_units(rep, tuning, per_kernel, layers),
               sample=costs)
    if args.headline_only:
        return out, step
    out["geometry"] = run_geometry(torch, step, args)
    out["schedule"] = run_schedule(torch, step, tuning)
    if not args.no_per_scene:
        out["per_scene"] = run_per_scene(torch, step, args, value,
                                         raster={k: int(tuning[k]) for k in ("tile", "fill_layers", "ppt_fwd", "ppt_bwd")})
        out["long_spline"] = run_long_spline(torch, args)
        out["layerwise"] = run_layerwise(torch)
    return out, step


def blend_units(rep, tuning, per_kernel, layers):
    """Blend work in the unit of the scope table: pair-evals = sum over tiles
    of |list| x tile pixels, the (pixel, Gaussian) pairs Eq. 8-9's loop would
    walk before early termination, with |list| the per-Gaussian tile lists
    (with fill layers, those the per-Gaussian binning of the same tile size
    produced in the autotuner's trial); besides the alpha evaluations the
    kernels performed and the pairs composited."""
    tile = int(tuning["tile"])
    pg = rep.pairs if not layers else tuning["tried"].get(str(tile), {}).get("pairs")
    out = dict(visits_fwd=int(rep.blend_visits), visits_bwd=int(rep.blend_bwd_visits),
               evals_fwd=int(rep.blend_evals), evals_bwd=int(rep.blend_bwd_evals),
               composited=int(rep.blend_contribs), per_gaussian_pairs=None if pg is None else int(pg))
    if pg is not None:
        pe = int(pg) * tile * tile
        out.update(pair_evals_listed=pe,
                   pair_evals_per_s_fwd=round(pe / (per_kernel["blend_fwd"] / 1e3), 1),
                   pair_evals_per_s_bwd=round(pe / (per_kernel["blend_bwd"] / 1e3), 1))
    out["evals_per_s_fwd"] = round(rep.blend_evals / (per_kernel["blend_fwd"] / 1e3), 1)
    out["evals_per_s_bwd"] = round(rep.blend_bwd_evals / (per_kernel["blend_bwd"] / 1e3), 1)
    return out


def run_layerwise(torch, rounds=4, iters=100):
    """The layer-wise vectorisation loop (§4.2) on a seeded 480x480 RGB blob
    target: `rounds` rounds of one new path each, `iters` iterations per round
    with the grid step annealed 4 -> 1 (Eq. 14), distance-weighted loss +
    self-crossing penalty + Adam.  Eager launches (the grid step changes every
    iteration); timed per round with CUDA events around the iterations."""
    from paper_2606_31764_b300.live import LayerwiseVectorizer
    rng = np.random.default_rng(1006)
    tgt = scenes.blob_target(rng, 1, 480, 480, 3, 24)
    lv = LayerwiseVectorizer(tgt, scenes.SAMPLE_DEFAULTS, scenes.RASTER_DEFAULTS, rounds=rounds, iters=iters)
    image = torch.ones_like(lv.target)   # the empty white canvas
    per_round = []
    for r in range(rounds):
        new_curve = lv.add_paths(image)
        lv.prepare(new_curve)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record()
        lv.iterate()
        e1.record()
        torch.cuda.synchronize()
        image = lv.finish()
        per_round.append(dict(paths=lv.batch.n_curves, ms_per_iteration=round(e0.elapsed_time(e1) / iters, 4),
                              wall_ms_per_iteration=round((time.perf_counter() - t0) * 1e3 / iters, 4),
                              loss=round(lv.losses[-1], 6)))
    return dict(workload="layerwise-480: one 480x480 RGB blob target, 12-key cubic circles added per round",
                rounds=rounds, iterations_per_round=iters, per_round=per_round,
                note="the round's set-up (seeding, buffer sizing) is outside the per-iteration times")


def run_schedule(torch, step, tuning):
    """Grid-step annealing (Eq. 14) on the headline batch: h(t) for T = 300
    iterations from h_max = 8 to h_min = 1 between t/T = 0.1 and 0.8, sampled at
    11 evenly spaced iterations.  Each sampled step is captured as a graph of
    its own (the grid step is a launch parameter) and timed with each binning
    (per Gaussian, fill layers) at the tuned tile, keeping the faster: fill
    layers win on fine grids, per-Gaussian pairs on coarse ones.  The
    schedule average is the sum of Gaussians over the sum of times."""
    from paper_2606_31764_b300 import binding as B
    lib = B.load()
    T, h0 = 300, float(step.sp.sp.h)
    rp = step.sp.rp
    saved = (int(rp.fill_layers), int(rp.ppt_fwd), int(rp.ppt_bwd))
    modes = []
    for fl in (0, 1):
        key = f"{int(rp.tile)}" + ("-layers" if fl else "")
        if key in tuning["tried"]:
            modes.append((fl, tuning["tried"][key]["ppt_fwd"], tuning["tried"][key]["ppt_bwd"]))
    rows = []
    for i in range(11):
        t = int(round(i * (T - 1) / 10))
        h = float(lib.ns_grid_step(t, T, 8.0, 1.0, 0.1, 0.8))
        step.sp.sp.h = h
        best = None
        for fl, pf, pb in modes:
            rp.fill_layers, rp.ppt_fwd, rp.ppt_bwd = fl, pf, pb
            g = capture(torch, step, 3)
            g.replay()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 3
            if best is None or ms < best[0]:
                best = (ms, fl)
            del g
        rows.append(dict(t=t, h=round(h, 4), gaussians=step.gaussians(), ms=round(best[0], 4),
                         fill_layers=best[1]))
    step.sp.sp.h = h0
    rp.fill_layers, rp.ppt_fwd, rp.ppt_bwd = saved
    step()
    torch.cuda.synchronize()
    G = sum(r["gaussians"] for r in rows)
    ms = sum(r["ms"] for r in rows)
    return dict(what="grid-step annealing 8 -> 1 px (Eq. 14, T = 300, t_b = 0.1, t_e = 0.8), 11 sampled iterations, "
                     "the faster binning per grid step",
                gaussians_per_s=round(G / (ms / 1e3), 1), ms_per_iteration=round(ms / len(rows), 4), steps=rows)


def run_geometry(torch, step, args):
    """The regularisers (Eq. 11 with r = 3 over N_L midpoint nodes per curve,
    Eq. 12 over the boundary points) with gradients, on the headline batch's
    sampling plan: K calls timed with CUDA events, not part of the headline
    step."""
    sc = step.scene
    grads = (torch.zeros_like(step.key), torch.zeros_like(step.tau))
    loss = torch.zeros(2, device="cuda")
    for _ in range(2):
        step.sp.geometry(step.key, step.tau, step.color, loss, grads)
    K = max(3, args.steps)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        step.sp.geometry(step.key, step.tau, step.color, loss, grads)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    nodes = sc.n_curves * int(sc.sample["nl_mult"]) * max(sc.width, sc.height)
    rep = step.sp.report()
    return dict(what="ns_geometry_loss with gradients: derivative loss (r = 3) + box loss, Table S1 weights",
                ms=round(ms, 4), nodes=nodes, boundary_points=int(rep.boundary),
                nodes_per_s=round(nodes / (ms / 1e3), 1), loss=[round(float(v), 4) for v in loss.cpu()])


def run_long_spline(torch, args):
    """The contour-path workload: 256 open cubic strokes with 64-512 key points
    (~1.5M Gaussians) on a 512x512 grayscale canvas, fwd + bwd + the
    calligraphy regularisers (Eq. 11 with r = 3, Eq. 12, Table S1 weights) +
    Adam step, graph-captured, timed like the headline (K steps in one graph;
    the per-kernel events in a second graph)."""
    from paper_2606_31764_b300 import binding as B
    sc = scenes.config3()
    geo = dict(lambda_deriv=1.0, lambda_bbox=5.0, order=3)
    st, tuning = autotune(torch, sc, [int(x) for x in args.tiles.split(",")], capacity=(3_000_000, 24_000_000, 16),
                          adam=True, geometry=geo, layers=(0,), fill_tiles=(16,))   # open strokes only: no fills
    st()
    K = max(3, args.steps)
    prof = ["emit", "bin_emit", "radix_scatter", "blend_fwd", "blend_bwd", "chain_contour", "deriv_loss",
            "bbox_loss"]
    ev = {k: [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
          for k in prof}
    for k in prof:
        for a, b in ev[k]:
            a.record()
            b.record()
    torch.cuda.synchronize()

    def arm(i):
        for k in prof:
            a, b = ev[k][i]
            B.call("ns_profile_next_launch", C.c_int32(B.KERNELS[k]), C.c_void_p(a.cuda_event),
                   C.c_void_p(b.cuda_event))

    # per-kernel events in one graph, the step time on a graph without them
    g = capture(torch, st, K, arm)
    g.replay()
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    kern = {k: round(float(np.mean([a.elapsed_time(b) for a, b in ev[k]])), 4) for k in prof}
    del g
    g0 = capture(torch, st, K)
    g0.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    g0.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    del g0
    G = st.gaussians()
    rep = st.sp.report()
    ablation = run_ablation(torch, sc, st, tuning, geo, K)
    aniso = run_tangent_variant(torch, sc, tuning, geo, K)
    return dict(workload="long-spline-512: 256 open cubic strokes, 64-512 key points, 512x512 gray, "
                         "+ derivative and box losses + Adam",
                geometry_nodes_per_step=sc.n_curves * int(sc.sample["nl_mult"]) * max(sc.width, sc.height),
                gaussians_per_step=G, pairs_per_step=int(rep.pairs), ms_per_step=round(ms, 4),
                gaussians_per_s=round(G / (ms / 1e3), 1), autotune=tuning,
                kernels=kern, ablation=ablation, tangent_aligned=aniso)


def run_tangent_variant(torch, sc, tuning, geo, K, delta_c=1.0):
    """The anisotropic prototype on the same strokes: tangent-aligned contour
    Gaussians at a tenth of the contour density (sigma_t spans the larger
    sample spacing), same step otherwise."""
    sc2 = sc.with_sample(contour_mode=1, delta_c=delta_c)
    s2 = Step(sc2, capacity=(3_000_000, 24_000_000, 16), raster=dict(sc2.raster, tile=tuning["tile"]), adam=True,
              geometry=geo)
    s2.sp.autotune_blend(s2.key, s2.tau, s2.color, s2.dimage, repeats=3)
    s2()
    g2 = capture(torch, s2, K)
    g2.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    g2.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    G = s2.gaussians()
    out = dict(delta_c=delta_c, gaussians_per_step=G, ms_per_step=round(ms, 4),
               gaussians_per_s=round(G / (ms / 1e3), 1), ppt=(int(s2.sp.rp.ppt_fwd), int(s2.sp.rp.ppt_bwd)))
    del g2, s2
    torch.cuda.empty_cache()
    return out


def run_ablation(torch, sc, st, tuning, geo, K):
    """The frozen-parameter variants of Table 1 on the long-spline step (same
    tile and blend decomposition): ms per step with rational weights, knot
    intervals, or both held fixed (their gradients not formed, no update)."""
    out = {"full": None}
    for name, frozen in (("w/o weights", ("weights",)), ("w/o knots", ("knots",)),
                         ("w/o w&k", ("weights", "knots")), ("full", ())):
        s2 = Step(sc, capacity=(3_000_000, 24_000_000, 16), raster=dict(sc.raster, tile=tuning["tile"]), adam=True,
                  geometry=geo, frozen=frozen)
        s2.sp.rp.ppt_fwd, s2.sp.rp.ppt_bwd = tuning["ppt_fwd"], tuning["ppt_bwd"]
        s2()
        g2 = capture(torch, s2, K)
        g2.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g2.replay()
        e1.record()
        torch.cuda.synchronize()
        out[name] = round(e0.elapsed_time(e1) / K, 4)
        del g2, s2
        torch.cuda.empty_cache()
    return dict(ms_per_step=out, note="same step as above; each variant captured and timed on its own")


def run_e2e(torch, step, g1, args):
    """Same metric through the public API with host buffers.  Every step copies
    key points, knot intervals and colours from pinned host memory (one copy:
    the step's inputs are views of one device buffer), runs the step and reads
    the loss and all gradients back (one copy of the results buffer).  The
    inputs and results are double-buffered, and the copies run on a stream of
    their own, so that step i+1's upload and step i's download overlap the
    neighbouring steps' compute; the steps themselves run one after another on
    one stream and one workspace.  The K steps and their copies are captured
    as one CUDA graph (the copies on a forked branch joined at the end), as a
    training loop would launch them."""
    A_in, A_out = step.inbuf, step.outbuf
    B_in, B_out = A_in.clone(), A_out.clone()
    ins, outs = (A_in, B_in), (A_out, B_out)
    hin = A_in.cpu().pin_memory()
    hout = [torch.empty(A_out.shape, dtype=A_out.dtype, pin_memory=True) for _ in range(2)]
    h2d = hin.numel() * 4
    d2h = A_out.numel() * 4
    G = step.gaussians()
    K = max(10, args.steps)
    cs = torch.cuda.Stream()

    def pipeline():
        s0 = torch.cuda.current_stream()
        up = [torch.cuda.Event() for _ in range(2)]       # inputs of buffer b uploaded
        done = [torch.cuda.Event() for _ in range(2)]     # the step on buffer b finished
        down = [torch.cuda.Event() for _ in range(2)]     # results of buffer b downloaded
        fork = torch.cuda.Event()
        fork.record(s0)
        cs.wait_event(fork)
        with torch.cuda.stream(cs):              # step 0's inputs
            ins[0].copy_(hin, non_blocking=True)
            up[0].record(cs)
        for i in range(K):
            b = i & 1
            if i + 1 < K:                        # the next step's inputs, once the step before it has read buffer 1-b
                with torch.cuda.stream(cs):
                    if i >= 1:
                        cs.wait_event(done[1 - b])
                    ins[1 - b].copy_(hin, non_blocking=True)
                    up[1 - b].record(cs)
            s0.wait_event(up[b])
            if i >= 2:
                s0.wait_event(down[b])           # results of buffer b from two steps back are out
            step.rebind(ins[b], outs[b])
            step()
            done[b].record(s0)
            with torch.cuda.stream(cs):
                cs.wait_event(done[b])
                hout[b].copy_(outs[b], non_blocking=True)
                down[b].record(cs)
        s0.wait_stream(cs)

    try:
        gE = capture(torch, pipeline)
    finally:
        step.rebind(A_in, A_out)
    gE.replay()          # warm
    torch.cuda.synchronize()
    s0 = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s0)
    gE.replay()
    e1.record(s0)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    del gE
    # the results the last step downloaded equal those of the step run directly
    # on the device inputs (the same parameters every step; the gradients'
    # atomic sums may round differently)
    step()
    torch.cuda.synchronize()
    ref = step.outbuf.cpu().double()
    err = float((hout[(K - 1) & 1].double() - ref).norm() / max(float(ref.norm()), 1e-30))
    if not err <= 1e-4:
        raise RuntimeError(f"e2e results differ from the device step's: relative error {err:.3g}")
    return dict(value=round(G * K / (ms / 1e3), 1), unit="Gaussians/s", h2d_bytes_per_step=h2d,
                d2h_bytes_per_step=d2h, steps=K, ms_per_step=round(ms / K, 4), results_rel_err=float(f"{err:.3g}"),
                copies="one H2D and one D2H per step from and to pinned host memory, on a copy stream "
                       "overlapping the neighbouring steps; the K steps and their copies in one CUDA graph")


def run_per_scene(torch, step, args, batched_value, raster=None):
    """The unbatched comparison: the batched 64-scene workload (256x256 RGB,
    1-40 closed paths per scene, half filled at h = 1) launched scene by scene
    with host reads of the counts between stages and no graph, against the
    same scenes in one batched, graph-captured step."""
    from paper_2606_31764_b300.splat import Splatter, scene_tensors
    sc = scenes.config4()
    K = max(2, min(args.steps, 5))
    # batched
    sc = sc.with_raster(**(raster or {}))   # the headline's tuned raster, for both paths
    bstep = Step(sc, capacity=(4_000_000, 8_000_000, 200_000))
    gb = capture(torch, bstep)
    for _ in range(2):
        gb.replay()
    torch.cuda.synchronize()
    Gb = bstep.gaussians()
    t0 = time.perf_counter()
    for _ in range(K):
        gb.replay()
    torch.cuda.synchronize()
    tb = (time.perf_counter() - t0) / K
    del gb
    # per scene
    subs = [sc.subset([s]) for s in range(sc.n_scenes)]
    steps = [Step(x, capacity=(200_000, 400_000, 20_000)) for x in subs]
    Gs = sum(s.gaussians() for s in steps)

    def one_pass():
        for s in steps:
            s.sp.sample(s.key, s.tau, s.color)
            s.sp.report()                      # host reads the counts
            s.sp.forward_gaussians(s.key, s.tau, s.color, s.image)
            s.sp.report()
            s.sp.mse(s.image, s.target, s.dimage, s.loss)
            s.sp.backward(s.key, s.tau, s.color, s.dimage, grads=s.grads)
            torch.cuda.synchronize()

    one_pass()
    t0 = time.perf_counter()
    for _ in range(K):
        one_pass()
    tp = (time.perf_counter() - t0) / K
    return dict(workload="batched-64x256: 64 scenes 256x256 RGB, 1-40 closed paths each",
                batched_gaussians_per_s=round(Gb / tb, 1), per_scene_gaussians_per_s=round(Gs / tp, 1),
                speedup=round((Gb / tb) / (Gs / tp), 2), gaussians_per_step=Gb, ms_batched=round(tb * 1e3, 3),
                ms_per_scene_path=round(tp * 1e3, 3), raster=raster)


# ----------------------------------------------------------------------------
# CPU oracle on a bounded sample

def oracle_sample_scene(n_curves, seed=1005):
    """The first n_curves paths of the 1024x1024 workload (same generator)."""
    sc = scenes.config5(seed=seed)
    b = scenes._Builder(1, sc.height, sc.width, sc.channels)
    for c in range(n_curves):
        k0, k1 = sc.key_offset[c], sc.key_offset[c + 1]
        t0, t1 = sc.tau_offset[c], sc.tau_offset[c + 1]
        b.add(0, int(sc.degree[c]), sc.key[k0:k1], sc.tau[t0:t1], sc.color[c], True, True)
    return b.build("vectorize-sample", sc.target, dict(sc.sample), dict(sc.raster))


def run_oracle_sample(n_curves, threads=None):
    """The oracle's fwd+bwd on the first n_curves paths, timed on `threads`
    host threads (default: every core of the machine)."""
    import torch
    from oracle import pipeline as op
    sub = oracle_sample_scene(n_curves)
    old = torch.get_num_threads()
    torch.set_num_threads(threads or os.cpu_count() or old)
    try:
        t0 = time.perf_counter()
        ref = op.loss_and_grads(sub)
        dt = time.perf_counter() - t0
        used = torch.get_num_threads()
    finally:
        torch.set_num_threads(old)
    G = int(sum(p.count for p in ref["plans"]))
    return sub, ref, dt, G, used


def oracle_context(n_curves_1t=8, n_scenes_cfg4=4):
    """Oracle timings beside the headline: one thread on a small sample of the
    1024x1024 workload, and the batched 64-scene workload's first scenes on
    every core, with the full workload's time extrapolated per scene."""
    import torch
    from oracle import pipeline as op
    _, _, dt1, G1, _ = run_oracle_sample(n_curves_1t, threads=1)
    sc4 = scenes.config4().subset(list(range(n_scenes_cfg4)))
    old = torch.get_num_threads()
    torch.set_num_threads(os.cpu_count() or old)
    try:
        t0 = time.perf_counter()
        ref4 = op.loss_and_grads(sc4)
        dt4 = time.perf_counter() - t0
        th = torch.get_num_threads()
    finally:
        torch.set_num_threads(old)
    G4 = int(sum(p.count for p in ref4["plans"]))
    full4 = scenes.config4()
    return dict(
        one_thread=dict(value=round(G1 / dt1, 1), unit="Gaussians/s", cores=1, seconds=round(dt1, 2),
                        sample=f"first {n_curves_1t} of the 2048 paths of the 1024x1024 workload, {G1} Gaussians, "
                               "one fwd+bwd"),
        batched_64x256=dict(value=round(G4 / dt4, 1), unit="Gaussians/s", cores=th, seconds=round(dt4, 2),
                            sample=f"first {n_scenes_cfg4} of the 64 scenes of the batched 256x256 workload, "
                                   f"{G4} Gaussians, one fwd+bwd",
                            extrapolated_full_s=round(dt4 * full4.n_scenes / n_scenes_cfg4, 1),
                            extrapolation="per-scene cost of the sample times 64 scenes"))


def parity_at_timed_config(sub, ref, tuning):
    """The GPU step in the configuration the bench times (the autotuner's tile,
    binning and decompositions) on the oracle's sample of the workload:
    gradient errors (max over tensors of ||g - g_ref|| / ||g_ref||) and the
    image error in three forms: at the parity thresholds; at the production
    thresholds outside pixels whose threshold decision lies within 1e-4 of its
    tie in the oracle; and at the production thresholds unfiltered (where a
    flipped alpha_min decision moves a pixel by up to alpha_min times a colour
    difference)."""
    import torch
    from oracle import pipeline as op
    tuned = {k: int(tuning[k]) for k in ("tile", "fill_layers", "ppt_fwd", "ppt_bwd")}
    cap = (300_000, 1_600_000, 20_000)
    step = Step(sub, capacity=cap, raster=dict(sub.raster, **tuned))
    step()
    torch.cuda.synchronize()
    errs = {}
    for nm, g, r in (("dkey", step.grads[0], ref["dkey"]), ("dtau", step.grads[1], ref["dtau"]),
                     ("dcolor", step.grads[2], ref["dcolor"])):
        gg = g.cpu().numpy().astype(np.float64).reshape(-1)
        rr = np.asarray(r, np.float64).reshape(-1)
        errs[nm] = float(np.linalg.norm(gg - rr) / max(np.linalg.norm(rr), 1e-30))
    img = step.image.cpu().numpy().astype(np.float64)
    del step
    k, t, c = op.leaves(sub, False)
    with torch.no_grad():
        _, _, flags = op.render(sub, k, t, c, plans=ref["plans"], return_flags=True)
    flags = flags.numpy()
    d = np.abs(img - ref["image"])
    ok = np.broadcast_to(~flags[..., None], d.shape)
    subp = sub.with_raster(**scenes.RASTER_PARITY)
    with torch.no_grad():
        refp, _ = op.render(subp, k, t, c, plans=ref["plans"])
    stepp = Step(subp, capacity=cap, raster=dict(subp.raster, **tuned))
    stepp()
    torch.cuda.synchronize()
    dp = float(np.abs(stepp.image.cpu().numpy().astype(np.float64) - refp.numpy()).max())
    del stepp
    image = dict(parity_thresholds=dp, production_outside_near_threshold=float(d[ok].max(initial=0.0)),
                 production_unfiltered=float(d.max()), near_threshold_pixels=int(flags.sum()),
                 pixels=int(flags.size), flag_rel=1e-4, gate=1e-5, raster=tuned)
    return max(errs.values()), errs, image


def main():
    args = parse()
    dist, rank, world = dist_setup(args)
    if args.impl == "reference":
        if rank != 0:
            return
        sub, ref, dt, G, cores = run_oracle_sample(args.ref_sample_curves)   # also the warm-up
        times = []
        from oracle import pipeline as op
        for _ in range(args.steps):
            t0 = time.perf_counter()
            op.loss_and_grads(sub)
            times.append(time.perf_counter() - t0)
        ms = 1e3 * float(np.mean(times))
        val = G / (ms / 1e3)
        sample = (f"first {args.ref_sample_curves} of the 2048 paths of the 1024x1024 workload, full canvas, "
                  f"{G} Gaussians per step")
        print(json.dumps(dict(impl="reference", metric=METRIC, value=round(val, 1), unit="Gaussians/s",
                              n_gpus=world, steps=args.steps, warmup=args.warmup, ms_per_step=round(ms, 2),
                              higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                              data="synthetic", config=dict(workload=workload_name(), sample=sample),
                              cpu_baseline=dict(value=round(val, 1), unit="Gaussians/s", cores=cores,
                                                kind="oracle", sample=sample),
                              e2e=dict(value=round(val, 1), unit="Gaussians/s", h2d_bytes_per_step=0,
                                       d2h_bytes_per_step=0))))
        return
    out, _ = run_gpu(args, dist, rank, world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sub, ref, dt, G, cores = run_oracle_sample(args.cpu_sample_curves)
        out["cpu_baseline"] = dict(value=round(G / dt, 1), unit="Gaussians/s", cores=cores, kind="oracle",
                                   sample=f"first {args.cpu_sample_curves} of the 2048 paths of the 1024x1024 "
                                          f"workload on the full canvas, {G} Gaussians, one fwd+bwd",
                                   seconds=round(dt, 2),
                                   extrapolated_full_s=round(dt * 2048 / args.cpu_sample_curves, 1),
                                   extrapolation="per-path cost of the sample times 2048 paths")
        out["cpu_baseline"].update(oracle_context())
        gre, errs, image = parity_at_timed_config(sub, ref, out["autotune"])
        out["grad_rel_err"] = round(gre, 7)
        out["grad_rel_err_detail"] = {k: round(v, 7) for k, v in errs.items()}
        out["image_err_vs_oracle"] = image
        out["image_max_abs_err_vs_oracle"] = image["parity_thresholds"]
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
