"""The binding's extent checks, on the CPU: the C entry points take bare
pointers and sizes, so every wrapper compares each tensor's extent with the
call's n, the handle's shapes and the scene's light count, and rejects a
short tensor before the library is called.

The handle here is a registered fake that no call may reach: every case
raises in the wrapper.  A tensor of the right extent gets as far as the
device check (host tensors are not CUDA tensors), which shows that the
extent checks do not reject valid arguments."""
import ctypes
from types import SimpleNamespace

import pytest
import torch

from paper_2506_05930_gb300 import nvc

FAKE = 0x1000
L, ENC, NP, B = 32, 32, 1000, 64
EXTENT = r"holds|must be \[n|rows"


@pytest.fixture
def h():
    nvc._HANDLE_SHAPES[FAKE] = nvc.HandleShapes(n_outputs=L, enc_width=ENC, n_params=NP,
                                                precision=1, batch=B)
    yield ctypes.c_void_p(FAKE)
    nvc._HANDLE_SHAPES.pop(FAKE, None)


def scene(n_lights=8):
    return SimpleNamespace(struct=SimpleNamespace(n_lights=n_lights), ref=None)


def f32(*shape):
    return torch.zeros(shape, dtype=torch.float32)


def i32(*shape):
    return torch.zeros(shape, dtype=torch.int32)


def test_handle_calls_reject_short_outputs(h):
    n = 10
    pos, nrm = f32(n, 3), f32(n, 3)
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_infer(h, pos, f32(n, L - 1))
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_encode(h, pos, f32(n, ENC - 1))
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_sampler_weights(h, scene(), pos, nrm, f32(n - 1, L))
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_shade(h, scene(), pos, nrm, 0, 0, idx=i32(n - 1))
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_wrs_sample(h, scene(), pos, nrm, 0, 0, pdf=f32(n - 1))
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_direct_illum(h, scene(), pos, nrm, f32(n - 1))
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_mlp_forward(h, pos, f32(n * L - 1))
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_mlp_backward(h, pos, f32(n, L), f32(NP - 1))
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_training_batch(h, target=f32(B * L - 1))
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_autotune_infer(h, pos, f32(n, L - 1))


def test_state_calls_reject_short_parameter_arrays(h):
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_set_params(h, f32(NP - 1))
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_set_state(h, f32(NP), adam_m=f32(NP - 1))
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_get_state(h, adam_v=f32(NP - 1))
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_train_gradient(h, scene(), None, 0, 0, f32(NP - 1))


def test_positions_must_be_rows_of_three(h):
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_infer(h, f32(30), f32(10, L))
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_shade(h, scene(), f32(10, 4), f32(10, 3), 0, 0)
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_shade(h, scene(), f32(10, 3), f32(9, 3), 0, 0)
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_train_step(h, scene(), f32(10, 2), 0, 0)


def test_scene_calls_use_the_scene_light_count():
    n, Ls = 10, 8
    pos, nrm = f32(n, 3), f32(n, 3)
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_light_weights(scene(Ls), pos, nrm, f32(n, Ls), f32(n, Ls - 1))
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_trace_visibility(scene(Ls), pos, f32(n * Ls - 1))
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_wrs_from_weights(f32(n, Ls), 0, 0, pdf=f32(n - 1))
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_exact_di(scene(Ls), pos, nrm, f32(n - 1))
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_shade_estimate(scene(Ls), pos, nrm, i32(n), f32(n), estimate=f32(n - 1))
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_training_positions(scene(Ls), None, 16, 0, 0, f32(16 * 3 - 1))
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_temporal_merge(scene(Ls), pos, nrm, i32(n), f32(n), W=f32(n - 1))


def test_clustered_calls_use_the_cluster_count():
    n, k = 10, 4
    cl = SimpleNamespace(struct=SimpleNamespace(k=k), ref=None)
    pos, nrm = f32(n, 3), f32(n, 3)
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_cluster_targets(scene(), cl, pos, 0, 0, f32(n, k - 1))
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_sample_clustered(scene(), cl, f32(n, k - 1), pos, nrm, 0, 0)
    with pytest.raises(ValueError, match=EXTENT):
        nvc.nvc_sample_clustered(scene(), cl, f32(n, k), pos, nrm, 0, 0, light=i32(n - 1))


def test_views_check_their_outputs():
    n = 10
    v = nvc.View(f32(n, 3), f32(n, 3), 0, i32(n), f32(n), f32(n), f32(n - 1))
    with pytest.raises(ValueError, match=EXTENT):
        v.struct()


def test_valid_extents_reach_the_device_check(h):
    n = 10
    pos, nrm = f32(n, 3), f32(n, 3)
    with pytest.raises(ValueError, match="CUDA"):
        nvc.nvc_infer(h, pos, f32(n, L))
    with pytest.raises(ValueError, match="CUDA"):
        nvc.nvc_shade(h, scene(), pos, nrm, 0, 0, idx=i32(n), pdf=f32(n), wsum=f32(n),
                      radiance=f32(n))
    with pytest.raises(ValueError, match="CUDA"):
        nvc.nvc_set_params(h, f32(NP))
    with pytest.raises(ValueError, match="CUDA"):
        nvc.View(pos, nrm, 0, i32(n), f32(n), f32(n), f32(n)).struct()
