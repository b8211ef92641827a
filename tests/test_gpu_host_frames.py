"""nvc_frame_host: frames whose G-buffers and outputs live in page-locked
host memory, uploaded and read back by the library on its own copy streams
while the previous / next frame computes.  Every frame must give what
nvc_frame gives on device copies of the same inputs, frame after frame,
although consecutive frames share the two device slots in turn: bit for bit
without training, and to the last bits with a training step per frame
(its gradients are summed with float atomics, whose order varies)."""
import numpy as np
import pytest
import torch

import nvc_synth as S

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2506_05930_gb300 import nvc, _lib


def _pinned(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).pin_memory()


def _outputs(n, device):
    kw = dict(device=device)
    mk = (lambda *a, **k: torch.empty(*a, **k).pin_memory()) if device == "cpu" else torch.empty
    return dict(idx=mk(n, dtype=torch.int32, **kw), pdf=mk(n, **kw), wsum=mk(n, **kw),
                radiance=mk(n, **kw))


@pytest.mark.parametrize("use_graph,train", [(True, False), (False, False), (True, True)])
def test_host_frames_equal_device_frames(use_graph, train):
    cfg = S.config_by_name("frame_1080p").with_(batch_positions=1024)
    sc = S.scene_heightfield(seed=2, n_lights=32, n_spheres=8, n_boxes=8)
    gbs = [S.gbuffer_heightfield(seed=10 + k, width=123 + 7 * k, height=45) for k in range(3)]
    p = S.init_params(cfg, seed=3)
    dev_cache, host_cache = nvc.VisibilityCache(cfg), nvc.VisibilityCache(cfg)
    dev_cache.set_params(p)
    host_cache.set_params(p)
    scene = nvc.Scene.from_synth(sc)
    n_frames = 5
    tv = 0 if train else nvc.NO_TRAINING
    ref, host_out = [], []
    for f in range(n_frames):
        gb = gbs[f % 3]
        o = _outputs(gb.n, "cuda")
        v = nvc.View(torch.from_numpy(gb.pos).cuda(), torch.from_numpy(gb.nrm).cuda(), 1, **o)
        nvc.nvc_frame(dev_cache.handle, scene, [v], tv, 7, f, use_graph=use_graph)
        ref.append({k: t.cpu() for k, t in o.items()})
    # the host path: all frames issued back to back, one wait at the end
    stream = torch.cuda.current_stream()
    for f in range(n_frames):
        gb = gbs[f % 3]
        o = _outputs(gb.n, "cpu")
        v = nvc.View(_pinned(gb.pos), _pinned(gb.nrm), 1, **o)
        host_out.append((v, o))          # keeps the host tensors alive until the read-back
        nvc.nvc_frame_host(host_cache.handle, scene, [v], tv, 7, f, use_graph=use_graph)
    nvc.nvc_host_frames_wait(host_cache.handle, stream)
    stream.synchronize()
    for f in range(n_frames):
        o = host_out[f][1]
        if not train:
            for k in ("idx", "pdf", "wsum", "radiance"):
                assert torch.equal(o[k], ref[f][k]), (f, k)
        else:
            assert (o["idx"] == ref[f]["idx"]).float().mean() > 0.99, f
            for k in ("pdf", "wsum", "radiance"):
                assert torch.allclose(o[k], ref[f][k], rtol=1e-4, atol=1e-6), (f, k)
        assert (o["idx"] >= 0).float().mean() > 0.5
    dev_cache.close()
    host_cache.close()


def test_host_frame_rejects_missing_inputs():
    cfg = S.config_by_name("tiny_fp32").with_(precision="fp16")
    cache = nvc.VisibilityCache(cfg)
    scene = nvc.Scene.from_synth(S.scene_unit_cube(seed=0))
    arr = (_lib.NvcView * 1)()
    arr[0].n_pixels = 16
    st = nvc.lib.nvc_frame_host(cache.handle, scene.ref, arr, 1, -1, 1, 0, None, 0, None)
    assert st == _lib.NVC_ERR_INVALID_ARG
    assert "NULL" in nvc.nvc_last_error(cache.handle)
    cache.close()


def test_host_frames_several_views_and_an_empty_one():
    """Three views in one host frame, the middle one empty: each non-empty
    view's outputs land in its own host tensors, bit-identical to the
    device path, and the empty view is skipped."""
    cfg = S.config_by_name("frame_1080p").with_(batch_positions=256)
    sc = S.scene_heightfield(seed=6, n_lights=32, n_spheres=4, n_boxes=4)
    gbs = [S.gbuffer_heightfield(seed=20, width=64, height=33),
           S.gbuffer_heightfield(seed=21, width=1, height=1),
           S.gbuffer_heightfield(seed=22, width=77, height=19)]
    p = S.init_params(cfg, seed=5)
    dev_cache, host_cache = nvc.VisibilityCache(cfg), nvc.VisibilityCache(cfg)
    dev_cache.set_params(p)
    host_cache.set_params(p)
    scene = nvc.Scene.from_synth(sc)
    dviews, hviews = [], []
    for k, gb in enumerate(gbs):
        n = 0 if k == 1 else gb.n
        pos, nrm = gb.pos[:n], gb.nrm[:n]
        dviews.append(nvc.View(torch.from_numpy(pos).cuda().reshape(n, 3),
                               torch.from_numpy(nrm).cuda().reshape(n, 3), 10 + k, **_outputs(n, "cuda")))
        hviews.append(nvc.View(_pinned(pos).reshape(n, 3), _pinned(nrm).reshape(n, 3), 10 + k,
                               **_outputs(n, "cpu")))
    nvc.nvc_frame(dev_cache.handle, scene, dviews, nvc.NO_TRAINING, 3, 9, use_graph=True)
    nvc.nvc_frame_host(host_cache.handle, scene, hviews, nvc.NO_TRAINING, 3, 9, use_graph=True)
    stream = torch.cuda.current_stream()
    nvc.nvc_host_frames_wait(host_cache.handle, stream)
    stream.synchronize()
    for dv, hv in zip(dviews, hviews):
        for k in ("idx", "pdf", "wsum", "radiance"):
            assert torch.equal(getattr(hv, k), getattr(dv, k).cpu()), k
    assert (hviews[2].idx >= 0).float().mean() > 0.5
    dev_cache.close()
    host_cache.close()
