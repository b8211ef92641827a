"""The cache as ReSTIR's initial-candidate generator (Sections 3.1 and 4.2):
temporal resampling of the cache's reservoir with the previous frame's,
through the C ABI, bit-exact against the oracle, and unbiased over frames."""
import numpy as np
import pytest
import torch

import nvc_synth as S
from oracle import nvc as O
from helpers import cfg_frame, scaled_params

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2506_05930_gb300 import nvc


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _merge(scene, pos, nrm, cl, cW, pl, pW, pM, seed, frame, view=0, offset=0):
    n = pos.shape[0]
    out = dict(light=torch.full((n,), -7, dtype=torch.int32, device="cuda"),
               W=torch.full((n,), -1.0, device="cuda"),
               M=torch.full((n,), -1, dtype=torch.int32, device="cuda"),
               estimate=torch.full((n,), -1.0, device="cuda"))
    nvc.nvc_temporal_merge(scene, pos, nrm, cl, cW, pl, pW, pM, seed=seed, frame=frame, view=view,
                           pixel_offset=offset, **out)
    return {k: host(v) for k, v in out.items()}


def _oracle_estimate(sc, pos, nrm, light, W):
    c32 = O.contributions(pos, nrm, sc.lights, np.float32)
    V = O.visibility(pos, sc.lights, sc.spheres, sc.boxes, np.float32)
    y = np.maximum(light, 0)
    cy = np.take_along_axis(c32, y[:, None], 1)[:, 0]
    vy = np.take_along_axis(V, y[:, None], 1)[:, 0]
    return np.where((light >= 0) & (vy > 0), (cy * W).astype(np.float32), np.float32(0))


def test_temporal_merge_bitexact_on_the_fused_samplers_reservoirs():
    """Current reservoirs from the fused FP16 sampler (y, W = 1 / pdf), a
    previous frame's reservoirs with random lights, weights and confidences
    (0 = disoccluded, some above the cap of 20, some empty): light, W, M and
    the one-ray estimate equal the oracle's bit for bit."""
    cfg = cfg_frame(batch_positions=256)
    sc = S.scene_heightfield(seed=3, n_lights=32, n_spheres=16, n_boxes=16)
    gb = S.gbuffer_heightfield(seed=3, width=61, height=53)
    cache = nvc.VisibilityCache(cfg)
    cache.set_params(scaled_params(cfg, seed=4, table_scale=0.5))
    scene = nvc.Scene.from_synth(sc)
    pos, nrm = dev(gb.pos), dev(gb.nrm)
    out = cache.shade(scene, pos, nrm, seed=9, frame=2, fused=True)
    cl = out["idx"]
    cW = torch.where(out["pdf"] > 0, 1.0 / out["pdf"], torch.zeros_like(out["pdf"]))
    rng = np.random.default_rng(5)
    n = gb.n
    pl = rng.integers(-1, 32, n).astype(np.int32)
    pW = rng.uniform(0.1, 30.0, n).astype(np.float32)
    pM = rng.integers(0, 40, n).astype(np.int32)
    got = _merge(scene, pos, nrm, cl, cW, dev(pl, torch.int32), dev(pW), dev(pM, torch.int32),
                 seed=7, frame=3, view=1, offset=500)
    c32 = O.contributions(gb.pos, gb.nrm, sc.lights, np.float32)
    rl, rW, rM = O.temporal_merge(c32, host(cl), host(cW), pl, pW, pM, 500 + np.arange(n), 7, 3, 1)
    assert np.array_equal(got["light"], rl)
    assert np.array_equal(got["W"], rW)
    assert np.array_equal(got["M"], rM)
    assert np.array_equal(got["estimate"], _oracle_estimate(sc, gb.pos, gb.nrm, rl, rW))
    # both reservoirs win somewhere; disoccluded pixels keep the cache's sample
    assert (rl == host(cl)).mean() > 0.2 and ((rl == pl) & (rl != host(cl))).mean() > 0.1
    dis = pM == 0
    assert np.array_equal(got["light"][dis], host(cl)[dis])
    # without a previous reservoir every pixel is disoccluded
    alone = _merge(scene, pos, nrm, cl, cW, None, None, None, seed=7, frame=3)
    assert np.array_equal(alone["light"], host(cl)) and np.all(alone["M"] == 1)
    cache.close()


def test_temporal_merge_bitexact_on_clustered_reservoirs():
    """The paper's combination: the clustered cache's two-step samples
    (Section 3.6) as ReSTIR's initial candidates on a 300-light scene."""
    sc = S.scene_many_lights(seed=4, n_lights=300, n_groups=24)
    assign, _ = nvc.nvc_kmeans_lights(sc.lights, S.kmeans_init(300, 16, seed=0), 5)
    clusters = nvc.Clusters(assign, 16)
    gb = S.gbuffer_heightfield(seed=4, width=47, height=31)
    scene = nvc.Scene.from_synth(sc)
    pos, nrm = dev(gb.pos), dev(gb.nrm)
    n = gb.n
    vis = np.random.default_rng(2).uniform(0.05, 1.0, (n, 16)).astype(np.float32)
    cl = torch.empty(n, dtype=torch.int32, device="cuda")
    cW = torch.empty(n, device="cuda")
    nvc.nvc_sample_clustered(scene, clusters, dev(vis), pos, nrm, 5, 1, light=cl, weight=cW)
    rng = np.random.default_rng(6)
    pl = rng.integers(-1, 300, n).astype(np.int32)
    pW = rng.uniform(0.1, 300.0, n).astype(np.float32)
    pM = rng.integers(0, 25, n).astype(np.int32)
    got = _merge(scene, pos, nrm, cl, cW, dev(pl, torch.int32), dev(pW), dev(pM, torch.int32),
                 seed=11, frame=4)
    c32 = O.contributions(gb.pos, gb.nrm, sc.lights, np.float32)
    rl, rW, rM = O.temporal_merge(c32, host(cl), host(cW), pl, pW, pM, np.arange(n), 11, 4, 0)
    assert np.array_equal(got["light"], rl) and np.array_equal(got["W"], rW)
    assert np.array_equal(got["M"], rM)
    assert np.array_equal(got["estimate"], _oracle_estimate(sc, gb.pos, gb.nrm, rl, rW))


@pytest.mark.parametrize("disocclude", [0.0, 0.3])
def test_temporal_chain_is_unbiased_against_exact_di(disocclude):
    """Frame after frame, the cache's sample merged with the previous
    frame's output reservoir (a fraction of pixels disoccluded each frame):
    the mean one-ray estimate converges to the all-lights DI (aggregate
    within 2%), as for the cache's sampler alone."""
    cfg = cfg_frame(batch_positions=256)
    sc = S.scene_heightfield(seed=3, n_lights=32, n_spheres=16, n_boxes=16)
    gb = S.gbuffer_heightfield(seed=3, width=64, height=32)
    cache = nvc.VisibilityCache(cfg)
    cache.set_params(scaled_params(cfg, seed=4, table_scale=0.5))
    scene = nvc.Scene.from_synth(sc)
    pos, nrm = dev(gb.pos), dev(gb.nrm)
    n = gb.n
    exact = torch.empty(n, device="cuda")
    nvc.nvc_exact_di(scene, pos, nrm, exact)
    prev = None
    acc = torch.zeros(n, device="cuda", dtype=torch.float64)
    gen = torch.Generator(device="cuda").manual_seed(3)
    frames = 512
    for f in range(frames):
        out = cache.shade(scene, pos, nrm, seed=1, frame=f, fused=True)
        cW = torch.where(out["pdf"] > 0, 1.0 / out["pdf"], torch.zeros_like(out["pdf"]))
        res = dict(light=torch.empty(n, dtype=torch.int32, device="cuda"),
                   W=torch.empty(n, device="cuda"), M=torch.empty(n, dtype=torch.int32, device="cuda"),
                   estimate=torch.empty(n, device="cuda"))
        if prev is not None and disocclude > 0:
            mask = torch.rand(n, device="cuda", generator=gen) < disocclude
            prev["M"] = torch.where(mask, torch.zeros_like(prev["M"]), prev["M"])
        args = (prev["light"], prev["W"], prev["M"]) if prev is not None else (None, None, None)
        nvc.nvc_temporal_merge(scene, pos, nrm, out["idx"], cW, *args, seed=2, frame=f, **res)
        acc += res["estimate"].double()
        prev = res
    mean = host(acc) / frames
    ex = host(exact).astype(np.float64)
    assert abs(mean.sum() - ex.sum()) <= 0.02 * ex.sum()
    assert (host(prev["M"]) > 1).mean() > 0.5
    cache.close()
