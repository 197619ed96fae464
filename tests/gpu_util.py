"""Helpers of the GPU parity tests: run the CUDA path through the C ABI."""
import numpy as np
import torch

from paper_2606_31764_b300 import binding as B
from paper_2606_31764_b300.splat import Splatter, scene_tensors


def run_records(scene, rec, curve, capacity=None, shape=None):
    """splat_forward on a given FP32 Gaussian set (with its tangent-aligned
    shapes when the scene samples in contour_mode 1).  Returns the splatter,
    the image, the report and the device inputs."""
    G = rec.shape[0]
    cap = capacity or (max(G, 1), max(64 * G, 1024), 16)
    sp = Splatter(scene, capacity=cap)
    sp.rec[:G] = torch.as_tensor(rec, device="cuda")
    sp.curve[:G] = torch.as_tensor(curve, device="cuda")
    if shape is not None:
        sp.shape[:G] = torch.as_tensor(shape, device="cuda")
    sp.aux[:G] = -1
    sp.count.fill_(G)
    k, t, c = scene_tensors(scene)
    img = sp.forward_gaussians(k, t, c).clone()
    rep = sp.report()
    return sp, img, rep, (k, t, c)


def sorted_pairs(sp, inputs, n_pairs):
    sp.remember(*inputs)
    tid = sp.workspace_array(0, 4 * n_pairs, torch.int32).cpu().numpy().astype(np.int64)
    gid = sp.workspace_array(1, 4 * n_pairs, torch.int32).cpu().numpy().astype(np.int64)
    return tid, gid


def tile_ranges(sp, inputs, n_tiles):
    sp.remember(*inputs)
    return sp.workspace_array(2, 8 * n_tiles, torch.int32).cpu().numpy().reshape(-1, 2).astype(np.int64)


def plans(sp, inputs, n_curves):
    """Per-curve plan records: (floats [nc,5], ints [nc,11])."""
    sp.remember(*inputs)
    raw = sp.workspace_array(3, 64 * n_curves, torch.int32).cpu().numpy().reshape(n_curves, 16)
    return raw[:, :5].view(np.float32), raw[:, 5:16]


def run_scene(scene, capacity=None):
    """nurbs_sample + splat_forward on a scene, capacities fitted."""
    sp = Splatter(scene, capacity=capacity or (1 << 14, 1 << 16, 1 << 12))
    k, t, c = scene_tensors(scene)
    rep = sp.fit(k, t, c)
    img = sp.forward(k, t, c).clone()
    G = int(sp.count.item())
    return sp, img, rep, (k, t, c), G


def run_step(scene, capacity=None):
    """Forward, L2 loss against the scene target, backward through the curves."""
    sp, img, rep, (k, t, c), G = run_scene(scene, capacity)
    tgt = torch.as_tensor(scene.target, device="cuda").contiguous()
    dimg = torch.empty_like(img)
    loss = torch.zeros(1, device="cuda")
    sp.mse(img, tgt, dimg, loss)
    dk, dt, dc = sp.backward(k, t, c, dimg)
    torch.cuda.synchronize()
    return dict(sp=sp, image=img.cpu().numpy(), loss=float(loss.item()), dkey=dk.cpu().numpy().reshape(-1, 4),
                dtau=dt.cpu().numpy(), dcolor=dc.cpu().numpy().reshape(-1, 4), report=rep, G=G,
                inputs=(k, t, c))
