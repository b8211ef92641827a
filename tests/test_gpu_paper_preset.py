"""The paper's own training settings and training-sample placement
(Section 3.4) through the C ABI, against the oracle.

- Placement: world-space only, screen-space only, or any split of the
  batch; the positions are bit-exact, and a handle's placement reaches its
  training steps.
- The paper preset (10 levels x 4 features, 2 x 32 hidden, leaky ReLU 0.01,
  He init, L2 loss, learning rate 0.05 -> 0.001 over 200 steps): the FP32
  gradient and Adam steps anywhere on the ramp follow the oracle, and the
  FP16 tensor-core training path (40 inputs padded to 48) sits on the fp16
  rounding model.
- The placement trade-off the paper reports, measured: screen-space samples
  fit the visible surfaces, world-space samples carry to surfaces the camera
  has not seen, and the equal split does both.
"""
import numpy as np
import pytest
import torch

import nvc_synth as S
from oracle import nvc as O
from helpers import cfg_tiny, rel_err, scaled_params

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2506_05930_gb300 import nvc, _lib


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


# --------------------------------------------------------------- placement --

@pytest.mark.parametrize("n_world", [-1, 0, 1, 333, 999, 1000])
def test_training_positions_split_bitexact(n_world):
    sc = S.scene_heightfield(seed=1, n_lights=4, n_spheres=2, n_boxes=2)
    gb = S.gbuffer_heightfield(seed=1, width=40, height=30)
    scene = nvc.Scene.from_synth(sc)
    B = 1000
    out = torch.full((B, 3), -1.0, device="cuda")
    nvc.nvc_training_positions_split(scene, dev(gb.pos), B, n_world, 0x1234567890ABCDEF, 17, out)
    ref = O.training_positions(B, sc.world_min, sc.world_max, gb.pos, 0x1234567890ABCDEF, 17,
                               None if n_world < 0 else n_world)
    assert np.array_equal(host(out), ref)
    # without screen positions every row is world space, whatever the split
    nvc.nvc_training_positions_split(scene, None, B, n_world, 5, 2, out)
    assert np.array_equal(host(out), O.training_positions(B, sc.world_min, sc.world_max,
                                                          None, 5, 2))


def test_training_placement_rejects_bad_splits():
    sc = S.scene_unit_cube(seed=0)
    scene = nvc.Scene.from_synth(sc)
    out = torch.empty((10, 3), device="cuda")
    for bad in (-2, 11):
        with pytest.raises(_lib.NVCError):
            nvc.nvc_training_positions_split(scene, None, 10, bad, 0, 0, out)
    cache = nvc.VisibilityCache(cfg_tiny())
    for bad in (-2, cache.cfg.batch_positions + 1):
        with pytest.raises(_lib.NVCError):
            nvc.nvc_set_training_placement(cache.handle, bad)
    cache.close()


@pytest.mark.parametrize("n_world", [0, 700, 1024, -1])
def test_placement_reaches_the_training_gradient(n_world):
    """The handle's placement decides the positions a training step uses:
    the gradient equals the oracle's on O.training_positions(n_world)."""
    cfg = cfg_tiny(loss="bce", leaky_slope=0.01)
    sc = S.scene_unit_cube(seed=0)
    gb = S.gbuffer_points(0, 64, 64)
    cache = nvc.VisibilityCache(cfg)
    p = scaled_params(cfg, seed=0, table_scale=0.5)
    cache.set_params(p)
    nvc.nvc_set_training_placement(cache.handle, n_world)
    g, loss = cache.train_gradient(nvc.Scene.from_synth(sc), dev(gb.pos), seed=3, frame=5)
    pos = O.training_positions(cfg.batch_positions, sc.world_min, sc.world_max, gb.pos, 3, 5,
                               None if n_world < 0 else n_world)
    y = O.visibility(pos, sc.lights, sc.spheres, sc.boxes, np.float32)
    loss_ref, g_ref = O.gradients(cfg, p, pos, y)
    assert abs(host(loss)[0] - loss_ref) <= 1e-6 * abs(loss_ref)
    assert rel_err(host(g), g_ref) <= 1e-5
    cache.close()


# ------------------------------------------------------------ paper preset --

def _paper_setup(batch, **kw):
    cfg = S.config_by_name("paper").with_(batch_positions=batch, **kw)
    sc = S.scene_heightfield(seed=1, n_lights=32, n_spheres=32, n_boxes=32)
    gb = S.gbuffer_heightfield(seed=1, width=96, height=54)
    p = scaled_params(cfg, seed=2, table_scale=0.5)
    cache = nvc.VisibilityCache(cfg)
    return cfg, sc, gb, p, cache


def test_paper_preset_fp32_gradient_matches_oracle():
    """10 x 4 features (40 inputs), 2 x 32 hidden, leaky ReLU 0.01, L2 loss,
    He-normal weights, on the 32-light heightfield scene."""
    cfg, sc, gb, p, cache = _paper_setup(4096)
    assert cfg.init == "he_normal" and cfg.loss == "l2" and cfg.n_inputs == 40
    cache.set_params(p)
    g, loss = cache.train_gradient(nvc.Scene.from_synth(sc), dev(gb.pos), seed=3, frame=5)
    pos = O.training_positions(cfg.batch_positions, sc.world_min, sc.world_max, gb.pos, 3, 5)
    y = O.visibility(pos, sc.lights, sc.spheres, sc.boxes, np.float32)
    loss_ref, g_ref = O.gradients(cfg, p, pos, y)
    assert abs(host(loss)[0] - loss_ref) <= 1e-6 * abs(loss_ref)
    assert rel_err(host(g), g_ref) <= 1e-5
    cache.close()


@pytest.mark.parametrize("step", [0, 149, 250])
def test_paper_preset_adam_step_on_the_learning_rate_ramp(step):
    """One Adam step after `step` earlier ones (zero moments): the update has
    the size of the ramp's rate, lr(t) = 0.05 + (0.001 - 0.05) min(t - 1,
    200) / 200, with the bias corrections of step t, on both sides."""
    cfg, sc, gb, p, cache = _paper_setup(2048)
    z = np.zeros_like(p)
    cache.set_params(p, z, z, step)
    scene = nvc.Scene.from_synth(sc)
    loss = cache.train_step(scene, dev(gb.pos), seed=0, frame=0)
    st = O.TrainState.fresh(p)
    st.step = step
    loss_ref = O.train_step(cfg, st, sc, gb.pos, seed=0, frame=0)
    assert abs(host(loss)[0] - loss_ref) <= 1e-6 * loss_ref
    assert cache.counters()["step"] == step + 1
    theta = host(cache.state()[0]).astype(np.float64)
    pos = O.training_positions(cfg.batch_positions, sc.world_min, sc.world_max, gb.pos, 0, 0)
    y = O.visibility(pos, sc.lights, sc.spheres, sc.boxes, np.float32)
    _, g = O.gradients(cfg, p, pos, y)
    clear = np.abs(g) > 1e-4 * np.abs(g).max()
    assert clear.sum() > 1000
    lr = O.learning_rate(cfg, step + 1)
    assert abs(lr - (0.05 + (0.001 - 0.05) * min(step, 200) / 200)) < 1e-12
    np.testing.assert_allclose(theta[clear], st.params[clear], atol=2e-6 + 1e-4 * lr)
    assert np.max(np.abs(theta - p)) > 0.5 * lr


def test_paper_preset_fp16_tensor_core_gradient():
    """The paper preset on the FP16 tensor-core training path: 40 encoded
    inputs padded to K = 48, 2 x 32 hidden; the gradient sits on the fp16
    rounding model and is as close to the float64 oracle as that model."""
    from helpers import fp16_gradient_model
    cfg, sc, gb, p, cache = _paper_setup(1024, train_precision="fp16", loss_scale=128.0)
    cache.set_params(p)
    g, loss = cache.train_gradient(nvc.Scene.from_synth(sc), dev(gb.pos), seed=5, frame=3)
    pos = O.training_positions(cfg.batch_positions, sc.world_min, sc.world_max, gb.pos, 5, 3)
    y = O.visibility(pos, sc.lights, sc.spheres, sc.boxes, np.float32)
    loss_ref, g_ref = O.gradients(cfg, p, pos, y)
    g_model = fp16_gradient_model(cfg, p, pos, y, 128.0)
    assert abs(host(loss)[0] - loss_ref) <= 2e-3 * abs(loss_ref)
    g = host(g)
    _, _, layers = S.param_layout(cfg)
    parts = [(0, layers[0][0])] + [(off, off + o * i) for off, o, i in layers]
    for lo, hi in [(0, len(g))] + parts:
        assert rel_err(g[lo:hi], g_model[lo:hi]) <= 5e-4, (lo, rel_err(g[lo:hi], g_model[lo:hi]))
        assert rel_err(g[lo:hi], g_ref[lo:hi]) <= 1.1 * rel_err(g_model[lo:hi], g_ref[lo:hi]) + 5e-4
    cache.close()


# ------------------------------------------------- the placement trade-off --

def test_placement_trade_off_on_seen_and_unseen_surfaces(capsys):
    """Section 3.4's comparison, measured: 300 training frames on the left
    half of the 1080p heightfield (the camera's view), then the squared
    error of the predicted visibilities against traced visibility on that
    view and on the right half (surfaces the camera has not seen).
    Screen-space samples fit the seen surfaces better than world-space
    ones; world-space samples carry to the unseen half better than
    screen-space ones; the equal split is better than world-only on the
    seen half and better than screen-only on the unseen half."""
    cfg = S.config_by_name("frame_1080p")
    sc = S.scene_heightfield(seed=1, n_lights=32, n_spheres=32, n_boxes=32)
    scene = nvc.Scene.from_synth(sc)
    seen = S.gbuffer_heightfield(seed=1, width=160, height=320, window=(0.0, 0.0, 5.0, 10.0))
    unseen = S.gbuffer_heightfield(seed=1, width=160, height=320, window=(5.0, 0.0, 5.0, 10.0))
    truth = {}
    for name, gb in (("seen", seen), ("unseen", unseen)):
        v = torch.empty((gb.n, 32), device="cuda")
        nvc.nvc_trace_visibility(scene, dev(gb.pos), v)
        truth[name] = (dev(gb.pos), v)
    B = cfg.batch_positions
    err = {}
    for label, n_world in (("world", B), ("screen", 0), ("split", -1)):
        cache = nvc.VisibilityCache(cfg)
        cache.set_params(S.init_params(cfg, seed=0))
        nvc.nvc_set_training_placement(cache.handle, n_world)
        screen = dev(seen.pos)
        for f in range(300):
            nvc.nvc_train_step(cache.handle, scene, screen, 11, f)
        for name, (pos, v) in truth.items():
            d = cache.infer(pos) - v
            err[(label, name)] = float((d * d).mean())
        cache.close()
    with capsys.disabled():
        print("\nplacement MSE (seen / unseen):",
              {k: round(e, 5) for k, e in err.items()})
    assert err[("screen", "seen")] < err[("world", "seen")]
    assert err[("world", "unseen")] < err[("screen", "unseen")]
    assert err[("split", "seen")] < 0.8 * err[("world", "seen")]
    assert err[("split", "unseen")] < 0.8 * err[("screen", "unseen")]
