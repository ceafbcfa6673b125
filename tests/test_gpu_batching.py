"""Batching (many views of uneven resolution, many scenes, one launch per stage), CUDA-graph
replay, and the per-pixel sort error, through the C ABI.

Bars:
  * a batched call renders every view exactly as a call for that view (or scene) alone:
    equal blend count and order hash on every pixel and bitwise-equal colour, depth and T
    (the per-pixel arithmetic is the same; only the launch grouping differs);
  * gradients of a batched backward equal the per-scene ones to float-atomic reordering
    (relative L2 <= 1e-5 on the small scenes, 1e-4 on the 8-scene training batch);
  * a replayed CUDA graph equals the eager calls it recorded (bitwise for the forward);
  * the sort error delta of Sec. 3.3 equals the oracle's on decided pixels to FP32 rounding
    of the per-pixel depths (|diff| <= 1e-5 (1 + delta) + 1e-5 * blends * max|t|).
"""
import numpy as np
import pytest

from paper_2402_00525_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2402_00525_gb300 import renderer as R  # noqa: E402
from gpu_helpers import compare_view, gpu_render, tile_mask  # noqa: E402


def _assert_same_render(a, b, label):
    for k in ("rgb", "depth", "tfinal"):
        assert torch.equal(a[k], b[k]), "%s: %s differs" % (label, k)
    for k in ("nblend", "hash"):
        assert torch.equal(a[k], b[k]), "%s: %s differs" % (label, k)


def _forward(r, g):
    rgb, depth, tf = r.forward(g)
    nbl, h = r.debug_stats()
    return dict(rgb=rgb.clone(), depth=depth.clone(), tfinal=tf.clone(), nblend=nbl.clone(), hash=h.clone())


def _small_scenes():
    scenes = [I.cluster_scene(3000, 11, nclusters=4, centre_range=1.0, scale_range=(0.005, 0.1)),
              I.uniform_scene(0, 12),
              I.uniform_scene(777, 13, sh_degree=1),
              I.cluster_scene(20000, 14, nclusters=8, centre_range=1.5, scale_range=(0.003, 0.2))]
    cams = [[I.look_at((0.3, -0.2, -5), (0, 0, 0), (0, 1, 0), 200, 150, 50.0),
             I.look_at((-4, 0.5, -2), (0, 0, 0), (0, 1, 0), 96, 128, 60.0)],
            [I.look_at((0, 0, -3), (0, 0, 0), (0, 1, 0), 64, 48, 60.0)],
            [I.look_at((0, 0, -3), (0, 0, 0), (0, 1, 0), 77, 33, 60.0),
             I.look_at((2, 1, -2.5), (0, 0, 0), (0, 1, 0), 130, 110, 55.0),
             I.look_at((0, -3, -0.5), (0, 0, 0), (0, 0, 1), 50, 50, 40.0)],
            [I.look_at((0.5, -0.3, -6), (0, 0, 0), (0, 1, 0), 333, 250, 50.0)]]
    return scenes, cams


def _per_scene_slices(cams):
    off, out = 0, []
    for cs in cams:
        n = sum(c.width * c.height for c in cs)
        out.append(slice(off, off + n))
        off += n
    return out


def test_batched_scenes_equal_one_call_per_scene():
    scenes, cams = _small_scenes()
    prm = I.RenderParams()
    gs = [R.scene_to_device(s) for s in scenes]
    rb = R.Renderer([s.n for s in scenes], [c for cs in cams for c in cs], prm, debug=True,
                    views_per_scene=[len(cs) for cs in cams])
    big = _forward(rb, gs)
    assert rb.status().error_bits == 0
    for k, (s, g, cs, sl) in enumerate(zip(scenes, gs, cams, _per_scene_slices(cams))):
        r1 = R.Renderer(s.n, cs, prm, debug=True)
        one = _forward(r1, g)
        _assert_same_render({kk: v[sl] for kk, v in big.items()}, one, "scene %d" % k)
    # the empty scene renders the background
    bg = big["rgb"][_per_scene_slices(cams)[1]]
    assert torch.all(bg == torch.tensor(prm.bg, dtype=torch.float32, device=bg.device))


def test_batched_backward_equals_one_call_per_scene():
    scenes, cams = _small_scenes()
    prm = I.RenderParams()
    gs = [R.scene_to_device(s) for s in scenes]
    allc = [c for cs in cams for c in cs]
    P = sum(c.width * c.height for c in allc)
    rng = np.random.default_rng(5)
    d_rgb = torch.from_numpy(rng.normal(size=(P, 3)).astype(np.float32)).cuda()
    d_dep = torch.from_numpy(rng.normal(size=P).astype(np.float32) * 0.1).cuda()
    rb = R.Renderer([s.n for s in scenes], allc, prm, backward=True, views_per_scene=[len(cs) for cs in cams])
    rb.forward(gs)
    grads_b = [{k: torch.zeros_like(g[k]) for k in R.FIELDS} for g in gs]
    rb.backward(gs, d_rgb, d_dep, grads_b)
    for k, (s, g, cs, sl) in enumerate(zip(scenes, gs, cams, _per_scene_slices(cams))):
        r1 = R.Renderer(s.n, cs, prm, backward=True)
        r1.forward(g)
        gr = {kk: torch.zeros_like(g[kk]) for kk in R.FIELDS}
        r1.backward(g, d_rgb[sl], d_dep[sl], gr)
        for f in R.FIELDS:
            a, b = grads_b[k][f].double(), gr[f].double()
            rel = (a - b).norm() / max(b.norm().item(), 1e-30)
            assert rel <= 1e-5, "scene %d %s rel %.3g" % (k, f, rel)


def test_graph_replay_equals_eager_forward_and_backward():
    scenes, cams = _small_scenes()
    prm = I.RenderParams()
    gs = [R.scene_to_device(s) for s in scenes]
    allc = [c for cs in cams for c in cs]
    P = sum(c.width * c.height for c in allc)
    rb = R.Renderer([s.n for s in scenes], allc, prm, backward=True, debug=True,
                    views_per_scene=[len(cs) for cs in cams], headroom=2.0)
    rb.forward(gs)                                   # sizes the workspace (host check)
    rng = np.random.default_rng(6)
    d_rgb = torch.from_numpy(rng.normal(size=(P, 3)).astype(np.float32)).cuda()
    out = tuple(torch.empty(sh, device="cuda") for sh in ((P, 3), (P,), (P,)))
    grads = [{k: torch.zeros_like(g[k]) for k in R.FIELDS} for g in gs]
    graph = rb.capture(gs, out, d_rgb=d_rgb, d_depth=None, grads=grads)
    # move the Gaussians in place, replay, and compare with eager calls at the new inputs
    for g in gs:
        g["means"].add_(0.01)
    for gr in grads:
        for t in gr.values():
            t.zero_()
    graph.replay()
    torch.cuda.synchronize()
    got = dict(rgb=out[0].clone(), depth=out[1].clone(), tfinal=out[2].clone())
    got_nbl, got_h = [x.clone() for x in rb.debug_stats()]
    got_grads = [{k: t.clone() for k, t in gr.items()} for gr in grads]
    rgb, depth, tf = rb.forward(gs)
    eager_grads = [{k: torch.zeros_like(g[k]) for k in R.FIELDS} for g in gs]
    rb.backward(gs, d_rgb, None, eager_grads)
    torch.cuda.synchronize()
    assert torch.equal(got["rgb"], rgb) and torch.equal(got["depth"], depth) and torch.equal(got["tfinal"], tf)
    nbl, h = rb.debug_stats()
    assert torch.equal(got_nbl, nbl) and torch.equal(got_h, h)
    for a, b in zip(got_grads, eager_grads):
        for f in R.FIELDS:
            rel = (a[f].double() - b[f].double()).norm() / max(b[f].double().norm().item(), 1e-30)
            assert rel <= 1e-5, f


def test_sort_error_delta_matches_oracle(oracle):
    sc, cams, prm = I.plain_forward_workload()
    for p in (prm, I.RenderParams(head=4), I.RenderParams(head=1, mid=8, tail=64)):
        gpu = gpu_render(sc, cams, p)
        ora = oracle.render(sc, cams[0], p)
        compare_view(gpu, 0, ora, label="delta head %d" % p.head)
        dec = ora["decided"]
        dg, do = gpu["delta"][0][dec], ora["delta"][dec]
        tmax = np.abs(ora["depth"]).max() + 10.0
        tol = 1e-5 * (1 + do) + 1e-5 * ora["nblend"][dec] * tmax
        assert np.all(np.abs(dg - do) <= tol), "head %d: max |d delta| %.3g" % (p.head, np.abs(dg - do).max())
        print("head", p.head, "delta avg %.4f max %.4f" % (do.mean(), do.max()))


def test_mixed_resolution_64_views_batched_equals_per_view(oracle):
    """The 64-view mixed-resolution workload on the 3M scene (320x240 .. 2560x1440): one
    batched launch sequence equals 64 single-view calls bit for bit, and sampled tiles of two
    views of different sizes match the oracle."""
    sc, cams, prm = I.batching_workload()
    g = R.scene_to_device(sc)
    rb = R.Renderer(sc.n, cams, prm, debug=True)
    big = _forward(rb, g)
    assert rb.status().error_bits == 0
    off = 0
    r1 = None
    for k, c in enumerate(cams):
        n = c.width * c.height
        sl = slice(off, off + n)
        off += n
        if r1 is None:
            r1 = R.Renderer(sc.n, [c], prm, debug=True)
        else:
            r1.set_cameras([c])
        one = _forward(r1, g)
        _assert_same_render({kk: v[sl] for kk, v in big.items()}, one, "view %d" % k)
    del r1
    gpu = dict(rgb=[x.cpu().numpy() for x in rb.split(big["rgb"])],
               depth=[x.cpu().numpy() for x in rb.split(big["depth"])],
               tfinal=[x.cpu().numpy() for x in rb.split(big["tfinal"])],
               nblend=[x.cpu().numpy() for x in rb.split(big["nblend"])],
               hash=[x.cpu().numpy().view(np.uint64) for x in rb.split(big["hash"])])
    rng = np.random.default_rng(8)
    for k in (0, 4):       # 320x240 and 2560x1440
        tiles = rng.choice(cams[k].num_tiles, min(30, cams[k].num_tiles), replace=False)
        with oracle.OracleRun(sc, cams[k], prm, tiles=tiles) as r:
            ora = r.render()
        frac = compare_view(gpu, k, ora, tiles_mask=tile_mask(cams[k], tiles), min_decided=0.5,
                            label="64-view batch, view %d" % k)
        print("view", k, cams[k].width, "x", cams[k].height, "decided", frac)


def test_batched_training_eight_scenes_graph(oracle):
    """The 8-scene training batch (cluster scenes of 100k..3M Gaussians, scaled by 1/10 here,
    4 views each at 640x480..1920x1080): forward + backward recorded in one CUDA graph equal
    per-scene eager calls; one scene's gradient matches the oracle adjoint on sampled tiles."""
    scenes, cams, prm = I.batched_training_workload(scale=0.1)
    gs = [R.scene_to_device(s) for s in scenes]
    allc = [c for cs in cams for c in cs]
    P = sum(c.width * c.height for c in allc)
    rng = np.random.default_rng(9)
    d_rgb = torch.from_numpy((rng.normal(size=(P, 3)) / P).astype(np.float32)).cuda()
    rb = R.Renderer([s.n for s in scenes], allc, prm, backward=True, views_per_scene=[4] * len(scenes),
                    headroom=1.5)
    rb.forward(gs)
    out = tuple(torch.empty(sh, device="cuda") for sh in ((P, 3), (P,), (P,)))
    grads = [{k: torch.zeros_like(g[k]) for k in R.FIELDS} for g in gs]
    graph = rb.capture(gs, out, d_rgb=d_rgb, grads=grads)
    for gr in grads:
        for t in gr.values():
            t.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert rb.status().error_bits == 0
    for k, (s, g, cs, sl) in enumerate(zip(scenes, gs, cams, _per_scene_slices(cams))):
        r1 = R.Renderer(s.n, cs, prm, backward=True)
        rgb, _, _ = r1.forward(g)
        assert torch.equal(rgb, out[0][sl]), "scene %d forward" % k
        gr = {kk: torch.zeros_like(g[kk]) for kk in R.FIELDS}
        r1.backward(g, d_rgb[sl], None, gr)
        for f in R.FIELDS:
            # random-sign loss weights over up to 1080p views: per-Gaussian sums of thousands of
            # cancelling float atomics, whose order differs between any two runs
            a, b = grads[k][f].double(), gr[f].double()
            rel = (a - b).norm() / max(b.norm().item(), 1e-30)
            assert rel <= 1e-4, "scene %d %s rel %.3g" % (k, f, rel)


def test_differentiation_720p_sampled_tiles_match_oracle_adjoint(oracle):
    """The 500k-Gaussian 1280x720 differentiation workload: L1 loss against the render of the
    perturbed scene. The gradient restricted to 48 sampled tiles (loss weights zero elsewhere
    and on undecided pixels) matches the FP64 adjoint per parameter block."""
    sc, target, cam, prm = I.differentiation_workload()
    g = R.scene_to_device(sc)
    gt = R.scene_to_device(target)
    rt = R.Renderer(target.n, [cam], prm)
    trgb, _, _ = rt.forward(gt)
    trgb = trgb.cpu().numpy().reshape(cam.height, cam.width, 3)
    del rt
    rr = R.Renderer(sc.n, [cam], prm, backward=True, debug=True)
    rgb, _, _ = rr.forward(g)
    rgb_np = rgb.cpu().numpy().reshape(cam.height, cam.width, 3)
    rng = np.random.default_rng(10)
    tiles = rng.choice(cam.num_tiles, 48, replace=False)
    with oracle.OracleRun(sc, cam, prm, tiles=tiles, record=True) as r:
        ora = r.render()
        mask = tile_mask(cam, tiles) & ora["decided"]
        assert mask.sum() >= 0.75 * tile_mask(cam, tiles).sum()
        w = np.sign(rgb_np.astype(np.float64) - trgb) / (3.0 * cam.num_pixels)
        w[~mask] = 0
        adj = r.backward(w)
    grads = {k: torch.zeros_like(g[k]) for k in R.FIELDS}
    rr.backward(g, torch.from_numpy(w.reshape(-1, 3).astype(np.float32)).cuda(), None, grads)
    torch.cuda.synchronize()
    for k in R.FIELDS:
        a = grads[k].cpu().numpy().astype(np.float64).ravel()
        b = adj[k].ravel()
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        cos = a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30)
        print(k, "rel-L2 %.3g cos %.8f" % (rel, cos))
        assert rel <= 1e-4 and cos >= 0.9999, k


def test_autotuner_keeps_the_image_under_same_result_policy():
    from paper_2402_00525_gb300 import autotune as A
    sc, cams, prm = I.plain_forward_workload()
    space = dict(tail=(64, 96), mid=(8, 12), head=(16,), lb_threshold=(16, 32), slice_k=(0, 64))
    chosen, trials, bd = A.tune(sc, cams, prm, policy="same-result", space=space, reps=2, warmup=1)
    assert (chosen.tail, chosen.mid, chosen.head) == (prm.tail, prm.mid, prm.head)
    inv = [t for t in trials if (t.tail, t.mid, t.head) == (prm.tail, prm.mid, prm.head)]
    # two thresholds x (per-tile sort at two slice sizes, global sort): all the base image
    assert len(inv) == 6 and all(t.same_image for t in inv)
    # larger queues never sort worse on average on this scene (Sec. 3.3: a wider window)
    big = [t for t in trials if t.tail == 96 and t.mid == 12]
    assert big and big[0].delta_avg <= 1.1 * bd["delta_avg"] + 1e-6
    chosen2, _, _ = A.tune(sc, cams, prm, policy="no-worse", space=space, reps=2, warmup=1)
    assert chosen2.head == 16


def test_graph_bound_workspace_reports_overflow_and_refuses_to_grow():
    """A workspace recorded into a CUDA graph cannot move: when a replay needs more sort entries
    than it holds, the status block says so (the kernels stay in bounds) and a checked forward
    raises instead of reallocating under the graph."""
    sc = I.uniform_scene(2000, 31, scale_range=(0.01, 0.05))
    cam = I.look_at((0, 0, -3), (0, 0, 0), (0, 1, 0), 128, 128, 60.0)
    prm = I.RenderParams()
    g = R.scene_to_device(sc)
    probe = R.Renderer(sc.n, [cam], prm)
    probe.forward(g)
    need = int(probe.status().num_entries)
    r = R.Renderer(sc.n, [cam], prm, capacity=need + 16)
    r.forward(g)
    assert r.status().error_bits == 0
    out = tuple(torch.empty(sh, device="cuda") for sh in ((cam.num_pixels, 3), (cam.num_pixels,), (cam.num_pixels,)))
    graph = r.capture(g, out)
    g["log_scales"].add_(0.7)                        # twice the size: many more (Gaussian, tile) entries
    graph.replay()
    torch.cuda.synchronize()
    st = r.status()
    assert st.error_bits & 1 and st.num_entries > st.capacity
    with pytest.raises(R.N.CapacityError):
        r.forward(g)
