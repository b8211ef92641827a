"""Online training on the GPU (Section 3.4): finite differences through the
C ABI, the 1000-frame online-training workload, and what the trained cache
gains over sampling without it."""
import numpy as np
import pytest
import torch

import nvc_synth as S
from oracle import nvc as O
from helpers import rel_err, scaled_params

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2506_05930_gb300 import nvc


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def test_gpu_gradient_matches_central_finite_differences():
    """The hand-written adjoint behind the autograd entry points
    (nvc_mlp_forward / nvc_mlp_backward) against central differences of the
    oracle's float64 BCE loss (h = 1e-3) on 128 random parameters with
    nonzero gradient, on the online-training workload's network.  Samples
    within 1e-2 of an activation kink are left out (a 1e-3 step could cross
    it)."""
    cfg = S.config_by_name("online_train").with_(batch_positions=512, leaky_slope=0.01,
                                                  train_precision="fp32")
    sc = S.scene_unit_cube(seed=0)
    view = S.gbuffer_camera_path(seed=0, frame=10)
    p = scaled_params(cfg, seed=4, table_scale=2.0).astype(np.float64)
    pos = O.training_positions(512, sc.world_min, sc.world_max, view.pos, 3, 10)
    y = O.visibility(pos, sc.lights, sc.spheres, sc.boxes, np.float32)
    table, Ws = O.split_params(cfg, p)
    _, _, zs = O.mlp_forward(Ws, O.encode(cfg, table, pos), cfg.leaky_slope)
    keep = np.all([np.min(np.abs(z), axis=1) > 1e-2 for z in zs], axis=0)
    pos, y = pos[keep], y[keep]
    n = len(pos)
    assert n > 100
    cache = nvc.VisibilityCache(cfg)
    cache.set_params(p.astype(np.float32))
    logits = torch.empty((n, 4), device="cuda")
    nvc.nvc_mlp_forward(cache.handle, dev(pos), logits)
    z = host(logits).astype(np.float64)
    dl = ((1 / (1 + np.exp(-z)) - y) / z.size).astype(np.float32)    # d BCE-mean / d logits
    grad = torch.empty(cache.n_params, device="cuda")
    nvc.nvc_mlp_backward(cache.handle, dev(pos), dev(dl), grad)
    g_gpu = host(grad)
    _, g_or = O.gradients(cfg, p, pos, y)
    rng = np.random.default_rng(0)
    cand = np.flatnonzero(np.abs(g_or) > 1e-3 * np.abs(g_or).max())
    pick = rng.choice(cand, 128, replace=False)
    h = 1e-3
    fd = np.empty(128)
    for k, i in enumerate(pick):
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd[k] = (O.gradients(cfg, pp, pos, y)[0] - O.gradients(cfg, pm, pos, y)[0]) / (2 * h)
    assert rel_err(g_or[pick], fd) < 1e-6          # the oracle's own adjoint
    assert rel_err(g_gpu[pick], fd) < 1e-5         # the CUDA adjoint through the C ABI


def _variance_and_di(cfg, cache, scene, sc, pts):
    """Mean closed-form variance of the one-sample estimator and Neural-DI
    relative error for the GPU's sampler weights on held-out points."""
    pos, nrm = dev(pts.pos), dev(pts.nrm)
    w = torch.empty((pts.n, cfg.n_outputs), device="cuda")
    nvc.nvc_sampler_weights(cache.handle, scene, pos, nrm, w)
    out = cache.shade(scene, pos, nrm, seed=1, frame=0, fused=cfg.precision != "fp32")
    V = O.visibility(pts.pos, sc.lights, sc.spheres, sc.boxes, np.float32)
    c = O.contributions(pts.pos, pts.nrm, sc.lights)
    _, var = O.estimator_moments(V, c, O.selection_law(host(w)))
    exact = O.exact_di(V, c)
    lit = exact > 1e-3
    di_err = np.mean(np.abs(host(out["radiance"])[lit] - exact[lit]) / exact[lit])
    return var.mean(), di_err


def test_online_training_1000_frames_converges_and_beats_no_cache():
    """The online-training workload: 1000 frames along the camera path,
    16,384 positions x 4 lights per frame, BCE, Adam (0.9, 0.99), lr 1e-2,
    FP16 compute with FP32 master weights and loss scale 128.  The loss
    falls by an order of magnitude, the cache approaches brute-force visibility (MAE < 0.05 on
    held-out points), and sampling with it has lower variance than sampling
    without a cache (v = 1) and than the untrained network; Neural DI gets
    closer to exact direct illumination."""
    cfg = S.config_by_name("online_train")
    sc = S.scene_unit_cube(seed=0)
    scene = nvc.Scene.from_synth(sc)
    cache = nvc.VisibilityCache(cfg)
    p0 = S.init_params(cfg, seed=0)
    cache.set_params(p0)
    held = S.gbuffer_points(99, 48, 48, lo=(0.2, 0.2, 0.2), hi=(0.8, 0.8, 0.8))
    var0, di0 = _variance_and_di(cfg, cache, scene, sc, held)
    loss = torch.empty(1000, dtype=torch.float64, device="cuda")
    for f in range(1000):
        view = S.gbuffer_camera_path(seed=0, frame=f)
        nvc.nvc_train_step(cache.handle, scene, dev(view.pos), 7, f, loss[f:f + 1])
    cnt = cache.counters()
    assert cnt["step"] == 1000 and cnt["skipped"] == 0
    L = host(loss)
    w = [L[i:i + 100].mean() for i in range(0, 1000, 100)]
    # the camera keeps moving, so the loss is not monotone; it must have
    # dropped by an order of magnitude and stayed there
    assert w[-1] < 0.1 * w[0] and max(w[5:]) < 0.1 * w[0], w
    V = O.visibility(held.pos, sc.lights, sc.spheres, sc.boxes, np.float32)
    mae = np.mean(np.abs(host(cache.infer(dev(held.pos))) - V))
    assert mae < 0.05, mae
    var1, di1 = _variance_and_di(cfg, cache, scene, sc, held)
    # without a cache: every light's visibility taken as 1
    c32 = O.contributions(held.pos, held.nrm, sc.lights, np.float32)
    c = O.contributions(held.pos, held.nrm, sc.lights)
    _, var_none = O.estimator_moments(V, c, O.selection_law(O.light_weights_f32(np.ones_like(c32), c32)))
    assert var1 < 0.8 * var_none.mean(), (var1, var_none.mean())
    assert var1 < var0
    assert di1 < 0.5 * di0, (di0, di1)


def test_adaptation_after_an_abrupt_scene_change(capsys):
    """Section 3.5: after the geometry changes abruptly the cache predicts
    the old shadows until online training catches up, and a second
    training step per frame shortens that.  The 1080p workload's cache is
    trained for 300 frames, then every occluder jumps 2 units in x; the
    visibility error on the view is followed for 32 frames with one and
    with two training steps per frame."""
    cfg = S.config_by_name("frame_1080p")
    sc = S.scene_heightfield(seed=1, n_lights=32, n_spheres=32, n_boxes=32)
    gb = S.gbuffer_heightfield(seed=1, width=320, height=180)
    pos = dev(gb.pos)
    before = nvc.Scene.from_synth(sc)
    shift = np.array([2.0, 0.0, 0.0], np.float32)
    moved_sph = sc.spheres.copy()
    moved_sph[:, :3] += shift
    moved_box = sc.boxes.copy()
    moved_box[:, :3] += shift
    moved_box[:, 3:] += shift
    after = nvc.Scene(sc.lights, moved_sph, moved_box, sc.world_min, sc.world_max)
    truth = torch.empty((gb.n, 32), device="cuda")
    nvc.nvc_trace_visibility(after, pos, truth)
    base = nvc.VisibilityCache(cfg)
    base.set_params(S.init_params(cfg, seed=0))
    for f in range(300):
        nvc.nvc_train_step(base.handle, before, pos, 11, f)
    state = [host(t) for t in base.state()]
    step0 = base.counters()["step"]
    base.close()

    def err(cache):
        d = cache.infer(pos) - truth
        return float((d * d).mean())

    curves = {}
    for steps in (1, 2):
        cache = nvc.VisibilityCache(cfg)
        cache.set_params(*state, step=step0)
        curve = [err(cache)]
        for f in range(32):
            for s in range(steps):
                nvc.nvc_train_step(cache.handle, after, pos, 13, 1000 + 2 * f + s)
            curve.append(err(cache))
        curves[steps] = curve
        cache.close()
    with capsys.disabled():
        print("\nMSE after the change, frames 0/4/8/16/32:",
              {k: [round(v[i], 4) for i in (0, 4, 8, 16, 32)] for k, v in curves.items()})
    one, two = curves[1], curves[2]
    assert one[0] > 2 * one[32]                 # the jump is visible, and training recovers
    assert one[16] < 0.5 * one[0]               # within 16 frames the error at least halves
    assert two[8] < one[8]                      # two steps per frame adapt faster


@pytest.mark.parametrize("name,batch", [("frame_1080p", 8192), ("frame_1080p", 1000),
                                        ("tiny_fp32", 1024)])
def test_fused_training_data_equals_the_separate_launch(name, batch):
    """Training data made inside the tensor-core training kernel (Section
    4.4's fused data generation): the positions and shadow-ray targets are
    the oracle's bit for bit -- the same as the separate launch's -- so the
    loss is the same double-precision sum, and the gradient differs only by
    the order of the float atomics that collect it.  A batch that is not a
    multiple of the 128-sample tile is included."""
    cfg = S.config_by_name(name).with_(train_precision="fp16", loss="bce", loss_scale=128.0,
                                       leaky_slope=0.01, batch_positions=batch)
    if name == "tiny_fp32":
        sc, gb = S.scene_unit_cube(seed=0), S.gbuffer_points(0, 64, 64)
    else:
        sc = S.scene_heightfield(seed=1, n_lights=32, n_spheres=32, n_boxes=32)
        gb = S.gbuffer_heightfield(seed=1, width=96, height=54)
    p = scaled_params(cfg, seed=2, table_scale=0.5)
    scene = nvc.Scene.from_synth(sc)
    screen = dev(gb.pos)
    out = {}
    for fused in (False, True):
        cache = nvc.VisibilityCache(cfg)
        cache.set_params(p)
        nvc.nvc_set_training_data_fused(cache.handle, fused)
        g, loss = cache.train_gradient(scene, screen, seed=5, frame=3)
        pos = torch.empty((batch, 3), device="cuda")
        tgt = torch.empty((batch, cfg.n_outputs), device="cuda")
        nvc.nvc_training_batch(cache.handle, pos, tgt)
        out[fused] = (host(g), host(loss)[0], host(pos), host(tgt))
        cache.close()
    ref_pos = O.training_positions(batch, sc.world_min, sc.world_max, gb.pos, 5, 3)
    ref_tgt = O.visibility(ref_pos, sc.lights, sc.spheres, sc.boxes, np.float32)
    for fused in (False, True):
        assert np.array_equal(out[fused][2], ref_pos), fused
        assert np.array_equal(out[fused][3], ref_tgt), fused
    assert 0.05 < ref_tgt.mean() < 0.95
    assert out[True][1] == out[False][1]
    assert rel_err(out[True][0], out[False][0]) <= 1e-5


def test_fused_training_data_steps_and_frames_train():
    """Whole training steps and graph-captured frames with the fused data:
    the loss follows the separate-launch path step for step, to the
    atomics-order difference the gradients carry into Adam."""
    cfg = S.config_by_name("frame_1080p").with_(batch_positions=2048)
    sc = S.scene_heightfield(seed=1, n_lights=32, n_spheres=32, n_boxes=32)
    gb = S.gbuffer_heightfield(seed=1, width=128, height=72)
    scene = nvc.Scene.from_synth(sc)
    pos, nrm = dev(gb.pos), dev(gb.nrm)
    p = scaled_params(cfg, seed=2, table_scale=0.5)
    losses = {}
    for fused in (False, True):
        cache = nvc.VisibilityCache(cfg)
        cache.set_params(p)
        nvc.nvc_set_training_data_fused(cache.handle, fused)
        n = gb.n
        view = nvc.View(pos, nrm, 0, torch.empty(n, dtype=torch.int32, device="cuda"),
                        torch.empty(n, device="cuda"), torch.empty(n, device="cuda"),
                        torch.empty(n, device="cuda"))
        loss = torch.empty(1, dtype=torch.float64, device="cuda")
        ls = []
        for f in range(12):
            nvc.nvc_frame(cache.handle, scene, [view], 0, 3, f, loss, use_graph=f % 2 == 1)
            ls.append(host(loss)[0])
        losses[fused] = np.array(ls)
        assert cache.counters()["step"] == 12
        cache.close()
    np.testing.assert_allclose(losses[True], losses[False], rtol=1e-3)
    assert losses[True][-1] < losses[True][0]


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_adam_refreshes_the_weight_image_and_table_copy(precision):
    """The Adam kernel writes the tensor cores' 16-bit weight image and the
    half-precision table copy from the updated weights (no separate packing
    pass): after training steps, shading equals that of a fresh handle given
    the same state (whose image and copy are packed from it), bit for bit."""
    from helpers import cfg_frame, scaled_params
    cfg = cfg_frame(precision=precision, train_precision="fp16", batch_positions=256)
    sc = S.scene_heightfield(seed=3, n_lights=32, n_spheres=16, n_boxes=16)
    gb = S.gbuffer_heightfield(seed=3, width=97, height=61)
    scene = nvc.Scene.from_synth(sc)
    pos = torch.from_numpy(gb.pos).cuda()
    nrm = torch.from_numpy(gb.nrm).cuda()
    a = nvc.VisibilityCache(cfg)
    a.set_params(scaled_params(cfg, seed=4, table_scale=0.5))
    for f in range(3):
        a.train_step(scene, pos, 1, f)
    p, m, v = a.state()
    b = nvc.VisibilityCache(cfg)
    b.set_params(p, m, v, step=a.counters()["step"])
    for cache in (a, b):
        nvc.nvc_set_shade_variant(cache.handle, 7)
    oa = a.shade(scene, pos, nrm, seed=2, frame=5, fused=True)
    ob = b.shade(scene, pos, nrm, seed=2, frame=5, fused=True)
    for k in oa:
        assert torch.equal(oa[k], ob[k]), k
    assert a.counters()["step"] == 3
    a.close()
    b.close()
