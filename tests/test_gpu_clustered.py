"""Clustered cache (Section 3.6) through the C ABI, against the oracle.

The training targets (one uniformly drawn member per cluster) and the
two-step sampler (integer reservoir over the clusters, streaming RIS among
four uniform members) are bit-exact: the same Philox words, the same
float32 roundings in the same order.  Both light-staging variants of the
sampler are covered (lights in shared memory, and a scene too large for it).
End to end, the one-sample estimates are unbiased against the exact DI, a
clustered training step optimises the loss of the oracle's targets, and a
trained clustered cache lowers the estimates' error.
"""
import numpy as np
import pytest
import torch

import nvc_synth as S
from oracle import nvc as O
from helpers import scaled_params

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2506_05930_gb300 import nvc, _lib


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def clustering(sc, k, seed=0, iters=8, empty=None, weights="sum"):
    """k-means clusters of the scene's lights; `empty` names a cluster whose
    members are moved to cluster 0, so the table holds an empty cluster."""
    init = S.kmeans_init(len(sc.lights), k, seed=seed)
    assign, _ = nvc.nvc_kmeans_lights(sc.lights, init, iters)
    if empty is not None:
        assign = np.where(assign == empty, 0, assign).astype(np.int32)
    off, mem = O.cluster_table(assign, k)
    return nvc.Clusters(assign, k, weights=weights), off, mem


def world_points(seed, n, sc):
    rng = np.random.default_rng(seed)
    lo, hi = sc.world_min.astype(np.float64), sc.world_max.astype(np.float64)
    return (lo + rng.random((n, 3)) * (hi - lo)).astype(np.float32)


@pytest.mark.parametrize("k,empty", [(32, None), (7, None), (32, 5)])
def test_cluster_targets_bitexact(k, empty):
    sc = S.scene_many_lights(seed=3, n_lights=300, n_groups=24)
    cl, off, mem = clustering(sc, k, empty=empty)
    pos = world_points(1, 1500, sc)
    scene = nvc.Scene.from_synth(sc)
    tgt = torch.full((len(pos), k), -1.0, device="cuda")
    nvc.nvc_cluster_targets(scene, cl, dev(pos), 77, 4, tgt)
    ref = O.cluster_targets(pos, sc.lights, sc.spheres, sc.boxes, off, mem,
                            np.arange(len(pos)), 77, 4)
    got = host(tgt)
    assert np.array_equal(got, ref.astype(np.float32))
    assert 0.05 < got.mean() < 0.95
    if empty is not None:
        assert (got[:, empty] == 0).all()


def _vis(seed, n, k):
    """Cluster visibilities as a cache feeds them: mostly in (0, 1), some
    below the clamp 0.001, some exact zeros."""
    rng = np.random.default_rng(seed)
    v = rng.random((n, k)).astype(np.float32)
    v[rng.random((n, k)) < 0.1] = 0.0
    v[rng.random((n, k)) < 0.05] = np.float32(2e-4)
    return v


def _estimate_ref(sc, pos, nrm, light, W):
    """V(x) c(x) W for the sampled light, float32, 0 when nothing sampled."""
    est = np.zeros(len(pos), np.float32)
    for p in np.nonzero(light >= 0)[0]:
        l = int(light[p])
        c = O.contributions(pos[p:p + 1], nrm[p:p + 1], sc.lights[l:l + 1], np.float32)[0, 0]
        v = O.visibility(pos[p:p + 1], sc.lights[l:l + 1], sc.spheres, sc.boxes, np.float32)[0, 0]
        est[p] = np.float32(c * W[p]) if v > 0 else np.float32(0.0)
    return est


@pytest.mark.parametrize("n_lights,k,empty,weights",
                         [(300, 32, None, "sum"), (300, 9, 3, "sum"), (15000, 32, None, "sum"),
                          (59000, 32, None, "sum"), (59000, 13, 5, "sum"),
                          (300, 32, None, "visibility"), (300, 9, 3, "visibility"),
                          (15000, 32, 7, "visibility")])
def test_sample_clustered_bitexact(n_lights, k, empty, weights):
    """Light and contribution weight bit-exact against the oracle, for both
    first-step weights.  The 15,000- and 59,000-light cases (the paper's
    many-lights scale) hold more lights than shared memory: the summed
    weights walk them in staged tiles, with clusters spanning tile edges."""
    sc = S.scene_many_lights(seed=4, n_lights=n_lights, n_groups=40)
    cl, off, mem = clustering(sc, k, empty=empty, iters=5, weights=weights)
    w, h = (53, 37) if n_lights < 20000 else (23, 11)    # the oracle's [pixels, lights] arrays
    gb = S.gbuffer_heightfield(seed=4, width=w, height=h)
    scene = nvc.Scene.from_synth(sc)
    vis = _vis(5, gb.n, k)
    light = torch.full((gb.n,), -7, dtype=torch.int32, device="cuda")
    W = torch.full((gb.n,), -1.0, device="cuda")
    est = torch.full((gb.n,), -1.0, device="cuda")
    off_px, seed, frame, view = 1000, 123, 6, 2
    nvc.nvc_sample_clustered(scene, cl, dev(vis), dev(gb.pos), dev(gb.nrm), seed, frame, view,
                             pixel_offset=off_px, light=light, weight=W, estimate=est)
    rl, rW = O.sample_clustered(vis, gb.pos, gb.nrm, sc.lights, off, mem,
                                off_px + np.arange(gb.n), seed, frame, view, weights)
    gl, gW = host(light), host(W)
    assert np.array_equal(gl, rl)
    assert np.array_equal(gW, rW)
    # visibility-only weights also pick clusters whose members all face away
    # (no light then, an unbiased zero estimate)
    assert (gl >= 0).mean() > (0.9 if weights == "sum" else 0.8)
    sub = np.arange(0, gb.n, 7)
    ref_est = _estimate_ref(sc, gb.pos[sub], gb.nrm[sub], rl[sub], rW[sub])
    assert np.array_equal(host(est)[sub], ref_est)
    assert (ref_est > 0).any() and (ref_est[rl[sub] >= 0] == 0).any()


@pytest.mark.parametrize("weights", ["sum", "visibility"])
def test_sample_clustered_is_unbiased_against_exact_di(weights):
    """Averaged over frames, V c W of the two-step sampler converges to the
    all-lights DI of each pixel: the estimator is unbiased for any cluster
    visibilities (here fixed random ones) and either first-step weights."""
    sc = S.scene_many_lights(seed=6, n_lights=512, n_groups=32)
    cl, _, _ = clustering(sc, 32, weights=weights)
    gb = S.gbuffer_heightfield(seed=6, width=64, height=32)
    scene = nvc.Scene.from_synth(sc)
    pos, nrm = dev(gb.pos), dev(gb.nrm)
    vis = dev(np.random.default_rng(8).uniform(0.05, 1.0, (gb.n, 32)))
    exact = torch.empty(gb.n, device="cuda")
    nvc.nvc_exact_di(scene, pos, nrm, exact)
    est = torch.empty(gb.n, device="cuda")
    acc = torch.zeros(gb.n, dtype=torch.float64, device="cuda")
    acc2 = torch.zeros_like(acc)
    F = 2048
    for f in range(F):
        nvc.nvc_sample_clustered(scene, cl, vis, pos, nrm, 9, f, estimate=est)
        e = est.double()
        acc += e
        acc2 += e * e
    mean, ex = host(acc) / F, host(exact).astype(np.float64)
    var = np.maximum(host(acc2) / F - mean * mean, 0.0)
    se = np.sqrt(var / F)
    z = (mean - ex) / np.maximum(se, 1e-12)
    lit = ex > 0
    assert abs(mean[lit].sum() - ex[lit].sum()) < 0.01 * ex[lit].sum()
    assert np.mean(np.abs(z[lit]) < 4.0) > 0.98
    assert (mean[~lit] == 0).all()


def test_clustered_training_step_fits_the_oracles_targets():
    """A clustered step trains on the targets of nvc_cluster_targets (which
    match the oracle bit for bit): its loss is the oracle's float64 BCE on
    them within the FP16 path's tolerance, and its first Adam update,
    -lr m/(sqrt(v) + eps) = -lr sign(g), has the signs of the oracle's
    gradient for those targets, not for other ones."""
    cfg = S.config_by_name("clustered_1080p").with_(batch_positions=4096)
    sc = S.scene_many_lights(seed=7, n_lights=256, n_groups=32)
    gb = S.gbuffer_heightfield(seed=7, width=64, height=48)
    cl, off, mem = clustering(sc, 32)
    scene = nvc.Scene.from_synth(sc)
    cache = nvc.VisibilityCache(cfg)
    p0 = scaled_params(cfg, seed=1, table_scale=8.0)
    cache.set_params(p0)
    screen = dev(gb.pos)
    pos = torch.empty((cfg.batch_positions, 3), device="cuda")
    nvc.nvc_training_positions(scene, screen, cfg.batch_positions, 31, 2, pos)
    tgt = torch.empty((cfg.batch_positions, 32), device="cuda")
    nvc.nvc_cluster_targets(scene, cl, pos, 31, 2, tgt)
    y = host(tgt).astype(np.float64)
    P = host(pos)
    ref_t = O.cluster_targets(P, sc.lights, sc.spheres, sc.boxes, off, mem,
                              np.arange(cfg.batch_positions), 31, 2)
    assert np.array_equal(y, ref_t)
    want, g = O.gradients(cfg, p0, P, y)
    _, g_other = O.gradients(cfg, p0, P, O.visibility(P, sc.lights[:32], sc.spheres,
                                                      sc.boxes, np.float32))
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    nvc.nvc_train_step_clustered(cache.handle, scene, cl, screen, 31, 2, loss)
    assert abs(host(loss)[0] - want) < 2e-3 * want
    step = host(cache.state()[0]).astype(np.float64) - p0
    mlp = slice(cfg.n_levels * cfg.table_size * cfg.n_features, len(p0))
    big = np.abs(g[mlp]) > 1e-2 * np.abs(g[mlp]).max()
    agree = np.mean(np.sign(step[mlp][big]) == -np.sign(g[mlp][big]))
    agree_other = np.mean(np.sign(step[mlp][big]) == -np.sign(g_other[mlp][big]))
    assert agree > 0.97 and agree_other < 0.85, (agree, agree_other)
    cache.close()


def test_trained_clustered_cache_learns_cluster_visibility_and_lowers_error():
    """Online clustered training on the 16-room scene with 1024 lights: the
    loss falls, the network's outputs approach each cluster's average
    visibility, and the two-step estimates accumulated over frames sit
    closer to the exact DI than with the untrained cache -- the purpose of
    Section 3.6 (clusters in other rooms are culled by their visibility)."""
    cfg = S.config_by_name("clustered_1080p").with_(batch_positions=16384)
    sc = S.scene_rooms(seed=1, n_lights=1024)
    gb = S.gbuffer_heightfield(seed=1, width=240, height=136)
    cl, off, mem = clustering(sc, 32, iters=10)
    scene = nvc.Scene.from_synth(sc)
    pos, nrm = dev(gb.pos), dev(gb.nrm)
    trained, untrained = nvc.VisibilityCache(cfg), nvc.VisibilityCache(cfg)
    p0 = S.init_params(cfg, seed=0)
    trained.set_params(p0)
    untrained.set_params(p0)
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    losses = []
    for f in range(300):
        nvc.nvc_train_step_clustered(trained.handle, scene, cl, pos, 11, f, loss)
        if f < 10 or f >= 290:
            losses.append(host(loss)[0])
    assert np.mean(losses[-10:]) < 0.8 * np.mean(losses[:10])
    # average visibility of each cluster at sampled pixels
    pick = np.random.default_rng(0).choice(gb.n, 400, replace=False)
    V = O.visibility(gb.pos[pick], sc.lights, sc.spheres, sc.boxes, np.float32)
    avg = np.stack([V[:, mem[off[y]:off[y + 1]]].mean(1) for y in range(32)], 1)
    err = []
    for cache in (trained, untrained):
        v = host(cache.infer(dev(gb.pos[pick])))
        err.append(np.mean((v - avg) ** 2))
    assert err[0] < 0.5 * err[1], err
    exact = torch.empty(gb.n, device="cuda")
    nvc.nvc_exact_di(scene, pos, nrm, exact)
    ex = host(exact).astype(np.float64)
    cl_vis = nvc.Clusters(nvc.nvc_kmeans_lights(sc.lights, S.kmeans_init(1024, 32, seed=0),
                                                10)[0], 32, weights="visibility")
    mse = {}
    for weights, clw in (("sum", cl), ("visibility", cl_vis)):
        for name, cache in (("trained", trained), ("untrained", untrained)):
            vis = cache.infer(pos)
            est = torch.empty(gb.n, device="cuda")
            acc = torch.zeros(gb.n, dtype=torch.float64, device="cuda")
            for f in range(16):
                nvc.nvc_sample_clustered(scene, clw, vis, pos, nrm, 21, 1000 + f, estimate=est)
                acc += est.double()
            d = host(acc) / 16 - ex
            mse[(weights, name)] = float(np.mean(d * d))
    print("\nclustered estimate MSE after 16 frames:", mse)
    for weights in ("sum", "visibility"):
        assert mse[(weights, "trained")] < 0.6 * mse[(weights, "untrained")], mse
    trained.close()
    untrained.close()


def test_empty_and_invalid_inputs():
    sc = S.scene_many_lights(seed=2, n_lights=64, n_groups=8)
    cl, _, _ = clustering(sc, 8)
    scene = nvc.Scene.from_synth(sc)
    z3 = torch.empty((0, 3), device="cuda")
    zk = torch.empty((0, 8), device="cuda")
    ze = torch.empty(0, device="cuda")
    nvc.nvc_cluster_targets(scene, cl, z3, 1, 1, zk)
    nvc.nvc_sample_clustered(scene, cl, zk, z3, z3, 1, 1, estimate=ze)
    p = torch.zeros((4, 3), device="cuda")
    v = torch.zeros((4, 8), device="cuda")
    with pytest.raises(_lib.NVCError):           # no output
        nvc.nvc_sample_clustered(scene, cl, v, p, p, 1, 1)
    bad = nvc.Clusters(np.zeros(64, np.int32), 8)
    bad.struct.k = 33
    with pytest.raises(_lib.NVCError):           # k above 32
        nvc.nvc_cluster_targets(scene, bad, p, 1, 1, v)
    bad.struct.k = 0
    with pytest.raises(_lib.NVCError):
        nvc.nvc_sample_clustered(scene, bad, v, p, p, 1, 1, estimate=torch.zeros(4, device="cuda"))
    bad.struct.k = 8
    bad.struct.weights = 2
    with pytest.raises(_lib.NVCError):                      # unknown weight mode
        nvc.nvc_sample_clustered(scene, bad, v, p, p, 1, 1, estimate=torch.zeros(4, device="cuda"))
    cache = nvc.VisibilityCache(S.config_by_name("clustered_1080p"))
    with pytest.raises(_lib.NVCError):           # k must equal n_outputs (32)
        nvc.nvc_train_step_clustered(cache.handle, scene, cl, p, 1, 1)
    cache.close()
