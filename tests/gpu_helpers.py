"""Comparison helpers shared by the GPU test files (CUDA path through the C ABI vs the oracle)."""
import numpy as np
import torch

from paper_2402_00525_gb300 import renderer as R


def gpu_render(scene, cams, prm, debug=True, capacity=None):
    g = R.scene_to_device(scene)
    r = R.Renderer(scene.n, cams, prm, debug=debug, capacity=capacity)
    rgb, depth, tf = r.forward(g)
    torch.cuda.synchronize()
    out = dict(rgb=[x.cpu().numpy() for x in r.split(rgb)], depth=[x.cpu().numpy() for x in r.split(depth)],
               tfinal=[x.cpu().numpy() for x in r.split(tf)], renderer=r, g=g)
    if debug:
        nbl, h = r.debug_stats()
        out["nblend"] = [x.cpu().numpy() for x in r.split(nbl)]
        out["hash"] = [x.cpu().numpy().view(np.uint64) for x in r.split(h)]
        out["delta"] = [x.cpu().numpy() for x in r.split(r.debug_delta())]
    return out


def compare_view(gpu, k, ora, tiles_mask=None, min_decided=0.99, label=""):
    dec = ora["decided"].copy()
    if tiles_mask is not None:
        dec &= tiles_mask
        denom = tiles_mask.sum()
    else:
        denom = dec.size
    frac = dec.sum() / max(denom, 1)
    assert frac >= min_decided, "%s decided fraction %.4f" % (label, frac)
    nb = gpu["nblend"][k]
    hs = gpu["hash"][k]
    bad = dec & ((nb != ora["nblend"]) | (hs != ora["hash"]))
    assert bad.sum() == 0, "%s: %d decided pixels differ in blend order (of %d)" % (label, bad.sum(), dec.sum())
    drgb = np.abs(gpu["rgb"][k] - ora["rgb"])[dec]
    assert drgb.size == 0 or drgb.max() <= 1e-4, "%s rgb max diff %g" % (label, drgb.max())
    dd = np.abs(gpu["depth"][k] - ora["depth"])[dec]
    assert dd.size == 0 or (dd / (1 + np.abs(ora["depth"][dec]))).max() <= 1e-4
    dt = np.abs(gpu["tfinal"][k] - ora["tfinal"])[dec]
    assert dt.size == 0 or dt.max() <= 1e-5
    return frac


def tile_mask(cam, tiles):
    m = np.zeros((cam.height, cam.width), bool)
    for t in tiles:
        tx, ty = t % cam.tiles_x, t // cam.tiles_x
        m[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16] = True
    return m
