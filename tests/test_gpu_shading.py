"""The shading pass (Section 3.1) and the all-lights exact DI (Section 4.4)
through the C ABI, against the CPU oracle.

Both are bit-exact: the shadow-ray decisions use the training targets'
float32 arithmetic, the contributions the sampler's float32 order, and the
estimate, running mean and exact-DI sum each fix their roundings.  At the
1080p workload the accumulated estimates of a trained cache converge to the
exact DI with a smaller error than an untrained cache's: the variance gain
the paper's method exists for.
"""
import numpy as np
import pytest
import torch

import nvc_synth as S
from oracle import nvc as O
from helpers import cfg_tiny, scaled_params

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2506_05930_gb300 import nvc, _lib


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _picks(cache, scene, pos, nrm, seed, frame):
    out = cache.shade(scene, pos, nrm, seed=seed, frame=frame, fused=True)
    return out["idx"], out["pdf"]


def test_shade_estimate_bitexact_on_the_samplers_picks():
    cfg = cfg_tiny(precision="fp16")
    sc, gb = S.scene_unit_cube(seed=0), S.gbuffer_points(0, 64, 64)
    cache = nvc.VisibilityCache(cfg)
    cache.set_params(scaled_params(cfg, seed=2, table_scale=0.5))
    scene = nvc.Scene.from_synth(sc)
    pos, nrm = dev(gb.pos), dev(gb.nrm)
    idx, pdf = _picks(cache, scene, pos, nrm, 3, 1)
    est = torch.full((gb.n,), -1.0, device="cuda")
    nvc.nvc_shade_estimate(scene, pos, nrm, idx, pdf, estimate=est)
    ref = O.shading_estimate(gb.pos, gb.nrm, sc.lights, sc.spheres, sc.boxes, host(idx), host(pdf))
    got = host(est)
    assert np.array_equal(got, ref)
    assert (got > 0).mean() > 0.3 and (got == 0).any()


def test_running_mean_over_frames_bitexact():
    cfg = cfg_tiny(precision="fp16")
    sc, gb = S.scene_unit_cube(seed=1), S.gbuffer_points(1, 32, 32)
    cache = nvc.VisibilityCache(cfg)
    cache.set_params(scaled_params(cfg, seed=4, table_scale=0.5))
    scene = nvc.Scene.from_synth(sc)
    pos, nrm = dev(gb.pos), dev(gb.nrm)
    acc = torch.full((gb.n,), 123.0, device="cuda")      # frame 1 overwrites it
    ref = None
    for k in range(1, 5):
        idx, pdf = _picks(cache, scene, pos, nrm, 9, k)
        nvc.nvc_shade_estimate(scene, pos, nrm, idx, pdf, accum=acc, count=k)
        e = O.shading_estimate(gb.pos, gb.nrm, sc.lights, sc.spheres, sc.boxes, host(idx), host(pdf))
        ref = O.running_mean(ref, e, k)
        assert np.array_equal(host(acc), ref), k


def test_exact_di_bitexact():
    sc = S.scene_heightfield(seed=5, n_lights=32, n_spheres=16, n_boxes=16)
    gb = S.gbuffer_heightfield(seed=5, width=91, height=47)
    scene = nvc.Scene.from_synth(sc)
    di = torch.empty(gb.n, device="cuda")
    nvc.nvc_exact_di(scene, dev(gb.pos), dev(gb.nrm), di)
    V = O.visibility(gb.pos, sc.lights, sc.spheres, sc.boxes, np.float32)
    ref = O.exact_di_f32(V, O.contributions(gb.pos, gb.nrm, sc.lights, np.float32))
    assert np.array_equal(host(di), ref)
    assert (V == 0).mean() > 0.01


def test_exact_di_full_1080p_frame_sampled():
    sc = S.scene_heightfield(seed=1, n_lights=32, n_spheres=32, n_boxes=32)
    gb = S.gbuffer_heightfield(seed=1, width=1920, height=1080)
    scene = nvc.Scene.from_synth(sc)
    di = torch.empty(gb.n, device="cuda")
    nvc.nvc_exact_di(scene, dev(gb.pos), dev(gb.nrm), di)
    pick = np.random.default_rng(0).choice(gb.n, 1500, replace=False)
    V = O.visibility(gb.pos[pick], sc.lights, sc.spheres, sc.boxes, np.float32)
    ref = O.exact_di_f32(V, O.contributions(gb.pos[pick], gb.nrm[pick], sc.lights, np.float32))
    assert np.array_equal(host(di)[pick], ref)


def test_empty_and_invalid_inputs():
    sc = S.scene_unit_cube(seed=0)
    scene = nvc.Scene.from_synth(sc)
    z = torch.empty((0, 3), device="cuda")
    zi = torch.empty(0, dtype=torch.int32, device="cuda")
    ze = torch.empty(0, device="cuda")
    nvc.nvc_shade_estimate(scene, z, z, zi, ze, estimate=ze)
    nvc.nvc_exact_di(scene, z, z, ze)
    p = torch.zeros((4, 3), device="cuda")
    i4 = torch.zeros(4, dtype=torch.int32, device="cuda")
    f4 = torch.zeros(4, device="cuda")
    with pytest.raises(_lib.NVCError):      # neither output
        nvc.nvc_shade_estimate(scene, p, p, i4, f4)
    with pytest.raises(_lib.NVCError):      # a running mean needs count >= 1
        nvc.nvc_shade_estimate(scene, p, p, i4, f4, accum=f4, count=0)


def test_trained_cache_estimates_converge_to_exact_di_with_less_error():
    """The one-sample estimates, accumulated over 32 frames, against the
    exact DI of the same pixels: unbiased for both caches (mean error far
    below the exact DI), and with a trained cache's visibility the error is
    smaller than with the untrained one's -- the variance reduction of
    Section 3.1, measured end to end on the 1080p workload at 480x270."""
    cfg = S.config_by_name("frame_1080p")
    sc = S.scene_heightfield(seed=1, n_lights=32, n_spheres=32, n_boxes=32)
    gb = S.gbuffer_heightfield(seed=1, width=480, height=270)
    scene = nvc.Scene.from_synth(sc)
    pos, nrm = dev(gb.pos), dev(gb.nrm)
    exact = torch.empty(gb.n, device="cuda")
    nvc.nvc_exact_di(scene, pos, nrm, exact)
    trained, untrained = nvc.VisibilityCache(cfg), nvc.VisibilityCache(cfg)
    p0 = S.init_params(cfg, seed=0)
    trained.set_params(p0)
    untrained.set_params(p0)
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    for f in range(300):
        nvc.nvc_train_step(trained.handle, scene, pos, 11, f, loss)
    errs = []
    for cache in (trained, untrained):
        acc = torch.zeros(gb.n, device="cuda")
        for k in range(1, 33):
            idx, pdf = _picks(cache, scene, pos, nrm, 21, 1000 + k)
            nvc.nvc_shade_estimate(scene, pos, nrm, idx, pdf, accum=acc, count=k)
        d = host(acc).astype(np.float64) - host(exact)
        errs.append((np.mean(d * d), np.mean(d)))
    ex = host(exact).astype(np.float64)
    mse_t, bias_t = errs[0]
    mse_u, bias_u = errs[1]
    assert abs(bias_t) < 0.02 * ex.mean() and abs(bias_u) < 0.02 * ex.mean()
    assert mse_t < 0.8 * mse_u, (mse_t, mse_u)
    trained.close()
    untrained.close()
