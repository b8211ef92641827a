"""The torch.autograd bridge to the hand-written adjoint, against the oracle.

A loss written in torch over ``visibility_logits`` back-propagates through
the library's MLP backward and hash-grid scatter; the gradient equals the
oracle's float64 gradient of the same loss, whatever the order of forward
and backward calls, and a torch optimiser trains the cache through it.
"""
import numpy as np
import pytest
import torch

import nvc_synth as S
from oracle import nvc as O
from helpers import cfg_tiny, rel_err, scaled_params

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import torch.nn.functional as F
    from paper_2506_05930_gb300 import nvc
    from paper_2506_05930_gb300.autograd import visibility_logits


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _batch(cfg, sc, gb, seed, frame):
    pos = O.training_positions(cfg.batch_positions, sc.world_min, sc.world_max, gb.pos,
                               seed, frame)
    return pos, O.visibility(pos, sc.lights, sc.spheres, sc.boxes, np.float32)


@pytest.fixture
def setup():
    cfg = cfg_tiny(loss="bce", leaky_slope=0.01)
    sc, gb = S.scene_unit_cube(seed=0), S.gbuffer_points(0, 64, 64)
    cache = nvc.VisibilityCache(cfg)
    p = scaled_params(cfg, seed=0, table_scale=0.5)
    yield cfg, sc, gb, cache, p
    cache.close()


def test_autograd_gradient_matches_oracle(setup):
    cfg, sc, gb, cache, p = setup
    params = dev(p).requires_grad_(True)
    pos, y = _batch(cfg, sc, gb, 3, 5)
    loss = F.binary_cross_entropy_with_logits(visibility_logits(cache, params, dev(pos)), dev(y))
    loss.backward()
    loss_ref, g_ref = O.gradients(cfg, p, pos, y)
    assert abs(loss.item() - loss_ref) <= 1e-6 * abs(loss_ref)
    assert rel_err(params.grad.cpu().numpy(), g_ref) <= 1e-5


def test_backward_after_a_later_forward_recomputes(setup):
    """Two forwards on the same handle, then the backward of the first: the
    handle's activations belong to the second, so the bridge recomputes."""
    cfg, sc, gb, cache, p = setup
    pos_a, y_a = _batch(cfg, sc, gb, 3, 5)
    pos_b, y_b = _batch(cfg, sc, gb, 4, 6)
    params = dev(p).requires_grad_(True)
    loss_a = F.binary_cross_entropy_with_logits(visibility_logits(cache, params, dev(pos_a)),
                                                dev(y_a))
    loss_b = F.binary_cross_entropy_with_logits(visibility_logits(cache, params, dev(pos_b)),
                                                dev(y_b))
    loss_a.backward()
    _, g_a = O.gradients(cfg, p, pos_a, y_a)
    assert rel_err(params.grad.cpu().numpy(), g_a) <= 1e-5
    params.grad = None
    loss_b.backward()
    _, g_b = O.gradients(cfg, p, pos_b, y_b)
    assert rel_err(params.grad.cpu().numpy(), g_b) <= 1e-5


def test_torch_optimizer_trains_through_the_bridge(setup):
    cfg, sc, gb, cache, p = setup
    params = torch.nn.Parameter(dev(S.init_params(cfg, seed=0)))
    opt = torch.optim.Adam([params], lr=1e-2, betas=(0.9, 0.99), eps=1e-15)
    losses = []
    for f in range(150):
        pos, y = _batch(cfg, sc, gb, 7, f)
        loss = F.binary_cross_entropy_with_logits(visibility_logits(cache, params, dev(pos)),
                                                  dev(y))
        opt.zero_grad()
        loss.backward()
        opt.step()
        losses.append(loss.item())
    assert np.mean(losses[-10:]) < 0.5 * np.mean(losses[:10]), (losses[:3], losses[-3:])


def test_set_params_leaves_the_adam_state(setup):
    cfg, sc, gb, cache, p = setup
    ones = np.ones_like(p)
    cache.set_params(p, ones, 2 * ones, step=5)
    p2 = dev(p * 0.5)
    nvc.nvc_set_params(cache.handle, p2)
    theta, m, v = (t.cpu().numpy() for t in cache.state())
    assert np.array_equal(theta, p2.cpu().numpy())
    assert np.all(m == 1.0) and np.all(v == 2.0)
    assert cache.counters()["step"] == 5
