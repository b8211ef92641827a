"""The fused tensor-core kernel (encode + tcgen05 MLP + sampler + Neural
DI) against the CPU oracle, through the C ABI.

FP16: visibility within 2e-3 of the float64 oracle; the reservoir pick is
bit-exact on the weights the kernel itself used (read back with
nvc_sampler_weights); the weights, pdf, sum and Neural DI within tolerances
derived from the visibility bound.
"""
import numpy as np
import pytest
import torch

import nvc_synth as S
from oracle import nvc as O
from helpers import cfg_tiny, cfg_frame, scaled_params

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2506_05930_gb300 import nvc


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def make(cfg, seed=0, table_scale=1.0):
    cache = nvc.VisibilityCache(cfg)
    p = scaled_params(cfg, seed=seed, table_scale=table_scale)
    cache.set_params(p)
    return cache, p


FP16_TOL = 2e-3

# The fused kernel's light contribution, c = (I/pi) (n.d) r inv with
# d = l - x, d.d and n.d by fused multiply-adds, r = rsqrtf(d.d) (at most 2
# ulp, 4u relative with u = 2^-24) and inv = r r (1e6 below d.d = 1e-6),
# against the float64 definition: d carries u; d.d 5u; r 4u + 2.5u; inv
# 2 x 6.5u + u = 14u; I rounded with 1/pi 2u and three products 3u: 25.5u
# relative in all.  n.d cancels at grazing angles: its absolute error,
# <= 4u |n| |d|, reaches c as <= 4u S (1 + 26u), S = I / (pi max(d.d, 1e-6))
# the normal-incidence value.  So |c_fused - c| <= 25.5u c + 4.1u S, and as
# c <= S, <= 30u S.  A weight max(v, 0.001) c adds one rounding and the
# visibility's error: |w - w64| <= FP16_TOL c + 31u S.  Neural DI, summed
# by L fused multiply-adds over positive terms, adds (L - 1) u sum v c.
U = 2.0 ** -24
C_TOL = 31 * U


def c_scale(pos, lights):
    """Normal-incidence contribution I / (pi d^2) of every light: the scale
    of the float32 rounding error of a contribution."""
    d2 = np.sum((lights[None, :, :3].astype(np.float64) - pos[:, None, :]) ** 2, -1)
    return lights[None, :, 3] / (np.pi * np.maximum(d2, 1e-6))


def di_bound(c64, cs):
    """Neural DI bound per pixel from the per-light contribution bound:
    visibility error x sum c, contribution error x sum S, summation error."""
    L = c64.shape[1]
    return (FP16_TOL + L * U) * c64.sum(1) + C_TOL * cs.sum(1)


@pytest.mark.parametrize("n", [1, 127, 129, 1000, 4096])
def test_fused_infer_fp16_matches_oracle(n):
    cfg = cfg_tiny(precision="fp16")
    cache, p = make(cfg)
    pos = S.gbuffer_points(3, 64, 64).pos[:n]
    vis = host(cache.infer(dev(pos)))
    ref = O.infer(cfg, p, pos)
    assert np.max(np.abs(vis - ref)) <= FP16_TOL
    assert np.std(ref) > 1e-2


@pytest.mark.parametrize("name,L", [("frame_1080p", 32), ("multiview", 128),
                                    ("precision_4k", 256), ("paper", 32)])
def test_fused_infer_fp16_network_shapes(name, L):
    cfg = S.config_by_name(name).with_(precision="fp16", batch_positions=256)
    assert cfg.n_outputs == L
    cache, p = make(cfg, seed=2, table_scale=0.5)
    lo, hi = np.array(cfg.bounds_min), np.array(cfg.bounds_max)
    pos = np.random.default_rng(1).uniform(lo, hi, (700, 3)).astype(np.float32)
    vis = host(cache.infer(dev(pos)))
    ref = O.infer(cfg, p, pos)
    err = np.abs(vis - ref)
    assert err.max() <= FP16_TOL, err.max()


def test_fused_infer_bf16_error_is_stated():
    cfg = cfg_frame(precision="bf16", batch_positions=256)
    cache, p = make(cfg, seed=2, table_scale=0.5)
    pos = np.random.default_rng(1).uniform(0, 10, (2000, 3)).astype(np.float32)
    err = np.abs(host(cache.infer(dev(pos))) - O.infer(cfg, p, pos))
    # bf16 keeps 8 significand bits: about 8x the fp16 error
    assert err.mean() <= 2e-3 and err.max() <= 2e-2, (err.mean(), err.max())


def _shade_case(cfg, sc, gb, seed=0, table_scale=1.0, offset=0):
    cache, p = make(cfg, seed=seed, table_scale=table_scale)
    scene = nvc.Scene.from_synth(sc)
    pos, nrm = dev(gb.pos), dev(gb.nrm)
    out = cache.shade(scene, pos, nrm, seed=11, frame=4, view=2, pixel_offset=offset, fused=True)
    w = torch.empty((gb.n, cfg.n_outputs), device="cuda")
    nvc.nvc_sampler_weights(cache.handle, scene, pos, nrm, w)
    return cache, p, out, host(w)


@pytest.mark.parametrize("L", [4, 32, 128, 256])
def test_fused_shade_pick_bitexact_on_its_weights(L):
    if L in (4, 128):
        cfg = (cfg_tiny(precision="fp16") if L == 4 else
               S.config_by_name("multiview").with_(precision="fp16", batch_positions=256))
        sc = S.scene_unit_cube(seed=0, n_lights=L)
        gb = S.gbuffer_points(0, 64, 64)
    else:
        base = {32: "frame_1080p", 256: "precision_4k"}[L]
        cfg = S.config_by_name(base).with_(precision="fp16", batch_positions=256)
        sc = S.scene_heightfield(seed=5, n_lights=L, n_spheres=4, n_boxes=4)
        gb = S.gbuffer_heightfield(seed=5, width=61, height=53)
    cache, p, out, w = _shade_case(cfg, sc, gb, offset=77)
    idx, pdf, wsum = O.wrs_select(w, 77 + np.arange(gb.n), 11, 4, 2)
    assert np.array_equal(host(out["idx"]), idx)
    np.testing.assert_allclose(host(out["wsum"]), wsum, rtol=1e-5, atol=1e-30)
    np.testing.assert_allclose(host(out["pdf"]), pdf, rtol=1e-5, atol=1e-30)
    # the weights themselves against the oracle's float64 visibility and contributions
    v64 = O.infer(cfg, p, gb.pos)
    c64 = O.contributions(gb.pos, gb.nrm, sc.lights)
    w64 = np.maximum(v64, 0.001) * c64
    # float32 error of c_i scales with I / (pi d^2) (n.d cancels at grazing angles)
    cs = c_scale(gb.pos, sc.lights)
    assert np.all(np.abs(w - w64) <= FP16_TOL * c64 + C_TOL * cs + 1e-30)
    # Neural DI
    di = host(out["radiance"])
    ref_di = O.neural_di(v64, c64)
    assert np.all(np.abs(di - ref_di) <= di_bound(c64, cs) + 1e-30)


@pytest.mark.parametrize("L", [32, 256])
def test_fused_contribution_within_its_derived_bound(L):
    """The contribution the fused kernel computes (fused multiply-add dot
    products, hardware reciprocal square root), recovered from its exported
    weights w = max(v, 0.001) c as w / max(v, 0.001) with v its own exported
    visibility (one more rounding), against the float64 definition:
    |c - c64| <= 26.5u c64 + 4.1u S, checked as 27u c64 + 5u S."""
    base = {32: "frame_1080p", 256: "precision_4k"}[L]
    cfg = S.config_by_name(base).with_(precision="fp16", batch_positions=256)
    sc = S.scene_heightfield(seed=7, n_lights=L, n_spheres=4, n_boxes=4)
    gb = S.gbuffer_heightfield(seed=7, width=97, height=61)
    cache, p = make(cfg, seed=3, table_scale=0.5)
    scene = nvc.Scene.from_synth(sc)
    pos, nrm = dev(gb.pos), dev(gb.nrm)
    w = torch.empty((gb.n, L), device="cuda")
    nvc.nvc_sampler_weights(cache.handle, scene, pos, nrm, w)
    v = host(cache.infer(pos)).astype(np.float32)
    c_est = host(w).astype(np.float64) / np.maximum(v, np.float32(0.001)).astype(np.float64)
    c64 = O.contributions(gb.pos, gb.nrm, sc.lights)
    cs = c_scale(gb.pos, sc.lights)
    bound = 27 * U * c64 + 5 * U * cs
    err = np.abs(c_est - c64)
    worst = np.unravel_index(np.argmax(err / bound), err.shape)
    assert np.all(err <= bound), (worst, err[worst] / bound[worst])
    cache.close()


def test_fused_shade_shard_invariance_and_zero_size():
    cfg = cfg_tiny(precision="fp16")
    sc = S.scene_unit_cube(seed=0)
    gb = S.gbuffer_points(0, 64, 64)
    cache, p = make(cfg)
    scene = nvc.Scene.from_synth(sc)
    pos, nrm = dev(gb.pos), dev(gb.nrm)
    full = cache.shade(scene, pos, nrm, seed=1, frame=2, fused=True)
    a = cache.shade(scene, pos[:1001], nrm[:1001], seed=1, frame=2, fused=True)
    b = cache.shade(scene, pos[1001:], nrm[1001:], seed=1, frame=2, pixel_offset=1001, fused=True)
    for k in ("idx", "pdf", "wsum", "radiance"):
        assert torch.equal(full[k], torch.cat([a[k], b[k]])), k
    cache.shade(scene, pos[:0], nrm[:0], fused=True)


def test_fused_and_separate_paths_agree():
    cfg = cfg_tiny(precision="fp16")
    sc = S.scene_unit_cube(seed=0)
    gb = S.gbuffer_points(0, 64, 64)
    cache, p = make(cfg)
    scene = nvc.Scene.from_synth(sc)
    pos, nrm = dev(gb.pos), dev(gb.nrm)
    f = cache.shade(scene, pos, nrm, seed=3, frame=1, fused=True)
    u = cache.shade(scene, pos, nrm, seed=3, frame=1, fused=False)
    assert (host(f["idx"]) == host(u["idx"])).mean() > 0.99
    np.testing.assert_allclose(host(f["radiance"]), host(u["radiance"]), rtol=5e-3, atol=1e-4)


def test_fused_full_1080p_frame_sampled():
    """The workload the bench times, in the same launch configuration: all
    2,073,600 pixels in one call; 4096 sampled pixels checked against the
    oracle one by one."""
    cfg = cfg_frame()
    sc = S.scene_heightfield(seed=1, n_lights=32, n_spheres=32, n_boxes=32)
    gb = S.gbuffer_heightfield(seed=1, width=1920, height=1080)
    cache, p = make(cfg, seed=0, table_scale=0.3)
    scene = nvc.Scene.from_synth(sc)
    pos, nrm = dev(gb.pos), dev(gb.nrm)
    out = cache.shade(scene, pos, nrm, seed=9, frame=500, fused=True)
    w = torch.empty((gb.n, 32), device="cuda")
    nvc.nvc_sampler_weights(cache.handle, scene, pos, nrm, w)
    pick = np.random.default_rng(0).choice(gb.n, 4096, replace=False)
    w_s = host(w[torch.from_numpy(pick).cuda()])
    idx, pdf, wsum = O.wrs_select(w_s, pick, 9, 500, 0)
    assert np.array_equal(host(out["idx"])[pick], idx)
    v64 = O.infer(cfg, p, gb.pos[pick])
    vis = host(cache.infer(pos[torch.from_numpy(pick).cuda()]))
    assert np.max(np.abs(vis - v64)) <= FP16_TOL
    c64 = O.contributions(gb.pos[pick], gb.nrm[pick], sc.lights)
    ref_di = O.neural_di(v64, c64)
    di = host(out["radiance"])[pick]
    cs = c_scale(gb.pos[pick], sc.lights)
    assert np.all(np.abs(di - ref_di) <= di_bound(c64, cs) + 1e-30)
    assert (host(out["idx"]) >= 0).mean() > 0.5


PAIR_VARIANT = 5   # two threads per pixel: sums taken as two half-sums


def _assert_resummed(a, b, L):
    """a, b: the same sums of L non-negative float32 terms in two orders.
    Each order is within (L - 1) u of the exact sum (u = 2^-24), so they
    differ by at most 2 (L - 1) u relative; pdf = w / sum adds one more
    rounding."""
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    tol = (2 * (L - 1) + 2) * 2.0 ** -24
    assert np.all(np.abs(a - b) <= tol * np.abs(b) + 1e-37), np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-37))


@pytest.mark.parametrize("cfg_name", ["tiny_fp32", "frame_1080p", "paper"])
def test_every_shade_variant_gives_identical_outputs(cfg_name):
    """The autotuner's variants differ only in how warps share the work:
    each one's picks and visibilities are bit-identical to the monolithic
    kernel's, and so are its sums, except for the two-threads-per-pixel
    variant, which adds two half-sums."""
    cfg = S.config_by_name(cfg_name).with_(precision="fp16", batch_positions=256)
    if cfg_name == "tiny_fp32":
        sc, gb = S.scene_unit_cube(seed=0), S.gbuffer_points(0, 64, 64)
    else:
        sc = S.scene_heightfield(seed=3, n_lights=cfg.n_outputs, n_spheres=8, n_boxes=8)
        gb = S.gbuffer_heightfield(seed=3, width=130, height=77)
    cache, p = make(cfg, seed=1, table_scale=0.5)
    scene = nvc.Scene.from_synth(sc)
    pos, nrm = dev(gb.pos), dev(gb.nrm)
    ref = None
    for v in range(nvc.SHADE_VARIANTS):
        nvc.nvc_set_shade_variant(cache.handle, v)
        out = cache.shade(scene, pos, nrm, seed=5, frame=2, pixel_offset=9, fused=True)
        vis = cache.infer(pos)
        if ref is None:
            ref = (out, vis)
            continue
        assert torch.equal(out["idx"], ref[0]["idx"]), v
        assert torch.equal(vis, ref[1]), v
        for k in ("pdf", "wsum", "radiance"):
            if v == PAIR_VARIANT:
                _assert_resummed(out[k], ref[0][k], cfg.n_outputs)
            else:
                assert torch.equal(out[k], ref[0][k]), (v, k)
    chosen, ms = nvc.nvc_autotune_shade(cache.handle, scene, pos, nrm, reps=2)
    assert 0 <= chosen < nvc.SHADE_VARIANTS and ms[chosen] > 0
    assert ms[chosen] == min(m for m in ms if m > 0)


@pytest.mark.parametrize("L", [4, 48, 128, 201, 256])
def test_two_threads_per_pixel_variant_across_light_counts(L):
    """Variant 5 splits the lights at H = ceil(L/2) rounded up to 16: for
    L = 4 the second thread has no lights, for 48 the first has two 16-light
    chunks; 128, 201 and 256 keep the weights in TMEM between the sampler's
    passes (201: odd, so the paired light table ends in a padding slot and
    the last chunks are ragged), as the monolithic kernel does above 32
    lights.  Its picks equal the monolithic kernel's, its sums agree to
    rounding, and the picks are the oracle's on the kernel's own weights."""
    cfg = S.config_by_name("frame_1080p").with_(n_outputs=L, precision="fp16", batch_positions=256)
    sc = S.scene_heightfield(seed=4, n_lights=L, n_spheres=8, n_boxes=8)
    gb = S.gbuffer_heightfield(seed=4, width=97, height=61)
    cache, p = make(cfg, seed=2, table_scale=0.5)
    scene = nvc.Scene.from_synth(sc)
    pos, nrm = dev(gb.pos), dev(gb.nrm)
    outs = []
    for v in (0, PAIR_VARIANT):
        nvc.nvc_set_shade_variant(cache.handle, v)
        outs.append(cache.shade(scene, pos, nrm, seed=3, frame=1, pixel_offset=5, fused=True))
    ref, out = outs
    assert torch.equal(out["idx"], ref["idx"])
    assert (host(out["idx"]) >= 0).mean() > 0.5
    for k in ("pdf", "wsum", "radiance"):
        _assert_resummed(out[k], ref[k], L)
    w = torch.empty((gb.n, L), device="cuda")
    nvc.nvc_sampler_weights(cache.handle, scene, pos, nrm, w)
    idx, _, _ = O.wrs_select(host(w), 5 + np.arange(gb.n), 3, 1, 0)
    assert np.array_equal(host(out["idx"]), idx)


@pytest.mark.parametrize("L", [32, 256])
def test_e4m3_two_threads_per_pixel_equals_monolithic(L):
    """With E4M3 operands the two-threads-per-pixel kernel (variant 5) runs
    the same scaled encode, MMAs and epilogues as the monolithic kernel:
    visibilities and picks bit for bit, sums to rounding."""
    cfg = S.config_by_name("frame_1080p").with_(n_outputs=L, precision="fp8",
                                                train_precision="fp32", batch_positions=256)
    sc = S.scene_heightfield(seed=6, n_lights=L, n_spheres=8, n_boxes=8)
    gb = S.gbuffer_heightfield(seed=6, width=97, height=61)
    cache, _ = make(cfg, seed=2, table_scale=0.5)
    scene = nvc.Scene.from_synth(sc)
    pos, nrm = dev(gb.pos), dev(gb.nrm)
    nvc.nvc_calibrate(cache.handle, pos[:256])          # at most batch_positions samples
    outs = []
    for v in (0, PAIR_VARIANT):
        nvc.nvc_set_shade_variant(cache.handle, v)
        outs.append((cache.shade(scene, pos, nrm, seed=4, frame=2, pixel_offset=7, fused=True),
                     cache.infer(pos)))
    (ref, vref), (out, vout) = outs
    assert torch.equal(vout, vref)
    assert torch.equal(out["idx"], ref["idx"])
    assert (host(out["idx"]) >= 0).mean() > 0.5
    for k in ("pdf", "wsum", "radiance"):
        _assert_resummed(out[k], ref[k], L)
    with pytest.raises(nvc.NVCError):
        nvc.nvc_set_shade_variant(cache.handle, 7)
    cache.close()


def _views(gbs):
    out = []
    for v, gb in enumerate(gbs):
        n = gb.n
        out.append(nvc.View(dev(gb.pos), dev(gb.nrm), v,
                            torch.empty(n, dtype=torch.int32, device="cuda"),
                            torch.empty(n, device="cuda"), torch.empty(n, device="cuda"),
                            torch.empty(n, device="cuda")))
    return out


def test_multiview_frame_is_one_launch_equal_to_per_view_launches():
    """Views of uneven resolution shaded by one persistent launch give the
    same bits as one launch per view (the tile -> view table only changes
    which CTA takes which tile)."""
    cfg = S.config_by_name("multiview").with_(batch_positions=256)
    sc = S.scene_unit_cube(seed=0, n_lights=128)
    gbs = S.multiview_gbuffers(seed=3, sizes=((160, 90), (192, 108), (256, 144), (384, 216)))
    cache, p = make(cfg, seed=1, table_scale=0.5)
    scene = nvc.Scene.from_synth(sc)
    views = _views(gbs)
    nvc.nvc_stage_times(cache.handle)
    nvc.nvc_frame(cache.handle, scene, views, nvc.NO_TRAINING, seed=7, frame=3, use_graph=False)
    _, launches = nvc.nvc_stage_times(cache.handle)
    assert launches == 2          # all four views in one shading launch + the frame counter
    for v, gb in zip(views, gbs):
        ref = cache.shade(scene, v.pos, v.nrm, seed=7, frame=3, view=v.view_id, fused=True)
        for k in ("idx", "pdf", "wsum", "radiance"):
            assert torch.equal(getattr(v, k), ref[k]), (v.view_id, k)


@pytest.mark.parametrize("variant", [6, 7])
def test_multiview_frame_with_tile_stream_variants(variant):
    """Variants 6 and 7 give each group of a CTA its own stream of tiles,
    which may belong to different views: a four-view, 32-light frame (so
    variant 7 takes its 32-light instantiation) is bit-identical to
    variant 0's."""
    cfg = S.config_by_name("frame_1080p").with_(batch_positions=256)
    sc = S.scene_heightfield(seed=8, n_lights=32, n_spheres=8, n_boxes=8)
    gbs = S.multiview_gbuffers(seed=4, sizes=((160, 90), (97, 33), (256, 144), (64, 64)))
    cache, p = make(cfg, seed=1, table_scale=0.5)
    scene = nvc.Scene.from_synth(sc)
    outs = []
    for v in (0, variant):
        nvc.nvc_set_shade_variant(cache.handle, v)
        views = _views(gbs)
        nvc.nvc_frame(cache.handle, scene, views, nvc.NO_TRAINING, seed=5, frame=2, use_graph=True)
        outs.append(views)
    for a, b in zip(*outs):
        for k in ("idx", "pdf", "wsum", "radiance"):
            assert torch.equal(getattr(a, k), getattr(b, k)), (a.view_id, k)
        assert (host(b.idx) >= 0).mean() > 0.5


def test_multiview_full_workload_in_one_graph_launch_sampled():
    """The batched multi-view workload: 1280x720, 1920x1080, 2560x1440 and
    3840x2160 (14,976,000 pixels) with 128 lights, trained and shaded as
    one graph-replayed frame; 2048 pixels per view checked against the
    oracle."""
    cfg = S.config_by_name("multiview")
    sc = S.scene_unit_cube(seed=0, n_lights=128)
    gbs = S.multiview_gbuffers(seed=0)
    assert sum(g.n for g in gbs) == 14_976_000
    cache, p = make(cfg, seed=2, table_scale=0.5)
    scene = nvc.Scene.from_synth(sc)
    views = _views(gbs)
    nvc.nvc_frame(cache.handle, scene, views, nvc.NO_TRAINING, seed=1, frame=0, use_graph=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    for v, gb in zip(views, gbs):
        pick = rng.choice(gb.n, 2048, replace=False)
        pt = torch.from_numpy(pick).cuda()
        w = torch.empty((2048, 128), device="cuda")
        nvc.nvc_sampler_weights(cache.handle, scene, v.pos[pt].contiguous(), v.nrm[pt].contiguous(), w)
        idx, pdf, wsum = O.wrs_select(host(w), pick, 1, 0, v.view_id)
        assert np.array_equal(host(v.idx)[pick], idx)
        v64 = O.infer(cfg, p, gb.pos[pick])
        c64 = O.contributions(gb.pos[pick], gb.nrm[pick], sc.lights)
        ref_di = O.neural_di(v64, c64)
        cs = c_scale(gb.pos[pick], sc.lights)
        assert np.all(np.abs(host(v.radiance)[pick] - ref_di) <= di_bound(c64, cs))
    # and a training frame over the same views runs and counts
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    nvc.nvc_frame(cache.handle, scene, views, 1, seed=1, frame=1, loss_out=loss, use_graph=True)
    assert cache.counters()["step"] == 1 and np.isfinite(host(loss)[0])


@pytest.mark.parametrize("L", [37, 32])
def test_infer_export_and_its_autotuner(L):
    """Exported visibilities within the fp16 bound of the oracle, with an odd
    light count too (rows alternate between 16-byte and checked scalar
    stores); nvc_autotune_infer keeps the fastest variant and the
    visibilities stay bit-identical."""
    cfg = cfg_frame(precision="fp16", batch_positions=256, n_outputs=L)
    cache, p = make(cfg, seed=2, table_scale=0.5)
    lo, hi = np.array(cfg.bounds_min), np.array(cfg.bounds_max)
    pos = np.random.default_rng(4).uniform(lo, hi, (997, 3)).astype(np.float32)
    ref = O.infer(cfg, p, pos)
    vis0 = host(cache.infer(dev(pos)))
    assert np.max(np.abs(vis0 - ref)) <= FP16_TOL
    chosen, ms = nvc.nvc_autotune_infer(cache.handle, dev(pos),
                                        torch.empty((len(pos), L), device="cuda"), reps=2)
    ran = [m for m in ms if m > 0]
    assert 0 <= chosen < nvc.SHADE_VARIANTS and ms[chosen] == min(ran)
    if L > 32:
        assert all(ms[v] < 0 for v in range(nvc.SHADE_VARIANTS) if v not in (0, PAIR_VARIANT))
    assert np.array_equal(host(cache.infer(dev(pos))), vis0)


def test_fp16_table_copy_follows_the_master():
    """Half-precision table features: inference within the FP16 bound of the
    oracle run on the float16-rounded table; the copy an Adam step refreshes
    equals the copy nvc_set_params writes from the same master (bitwise equal
    visibilities); going back to float32 features reads the master again."""
    cfg = cfg_frame(precision="fp16", batch_positions=512, table_precision="fp16")
    cache, p = make(cfg, seed=2, table_scale=0.5)
    pos_np = np.random.default_rng(3).uniform(0, 10, (3000, 3)).astype(np.float32)
    pos = dev(pos_np)
    assert np.max(np.abs(host(cache.infer(pos)) - O.infer(cfg, p, pos_np))) <= FP16_TOL
    sc = S.scene_heightfield(seed=1, n_lights=32, n_spheres=32, n_boxes=32)
    gb = S.gbuffer_heightfield(seed=1, width=64, height=36)
    cache.train_step(nvc.Scene.from_synth(sc), dev(gb.pos), seed=1, frame=0)
    theta = cache.state()[0]
    vis_trained = host(cache.infer(pos))
    assert np.max(np.abs(vis_trained - O.infer(cfg, host(theta), pos_np))) <= FP16_TOL
    fresh = nvc.VisibilityCache(cfg)
    fresh.set_params(theta)
    assert np.array_equal(host(fresh.infer(pos)), vis_trained)
    # float32 features: the same as a cache that never had the copy
    nvc.nvc_set_table_precision(cache.handle, "fp32")
    plain = nvc.VisibilityCache(cfg.with_(table_precision="fp32"))
    plain.set_params(theta)
    assert np.array_equal(host(cache.infer(pos)), host(plain.infer(pos)))
    assert not np.array_equal(host(plain.infer(pos)), vis_trained)
    for c in (cache, fresh, plain):
        c.close()


@pytest.mark.parametrize("name,L", [("frame_1080p", 32), ("multiview", 128)])
def test_every_point_of_the_tuning_space_shades_identically(name, L):
    """nvc_autotune_shade_plan searches kernel layout (tile streams per CTA,
    levels split across threads, warp specialisation) x resident CTAs per
    SM.  Every point it tries makes the monolithic kernel's picks; all but
    the two-threads-per-pixel layout (whose sums are two half-sums) give
    bit-identical pdf, sum and Neural DI too."""
    cfg = S.config_by_name(name).with_(batch_positions=256)
    cache, p = make(cfg, seed=2, table_scale=0.5)
    if L == 32:
        sc = S.scene_heightfield(seed=8, n_lights=32, n_spheres=8, n_boxes=8)
        gb = S.gbuffer_heightfield(seed=8, width=160, height=97)
    else:
        sc = S.scene_unit_cube(seed=0, n_lights=128)
        gb = S.gbuffer_points(2, 128, 81)
    scene = nvc.Scene.from_synth(sc)
    pos, nrm = dev(gb.pos), dev(gb.nrm)
    chosen, tried = nvc.nvc_autotune_shade_plan(cache.handle, scene, pos, nrm, reps=2)
    points = [pt for pt, _ in tried]
    assert chosen in points and len(set(points)) == len(points)
    variants = {v for v, _ in points}
    assert variants == ({0, 1, 2, 3, 4, 5, 6, 7} if L == 32 else {0, 5})
    assert {c for _, c in points} == {0, 1, 2, 3}
    nvc.nvc_set_shade_plan(cache.handle, 0, 0)
    ref = cache.shade(scene, pos, nrm, seed=3, frame=1, fused=True)
    for v, c in points:
        nvc.nvc_set_shade_plan(cache.handle, v, c)
        out = cache.shade(scene, pos, nrm, seed=3, frame=1, fused=True)
        assert torch.equal(out["idx"], ref["idx"]), (v, c)
        for k in ("pdf", "wsum", "radiance"):
            if v == PAIR_VARIANT:
                np.testing.assert_allclose(host(out[k]), host(ref[k]), rtol=2 * (L - 1) * 2.0 ** -24,
                                           atol=1e-30)
            else:
                assert torch.equal(out[k], ref[k]), (v, c, k)
    cache.close()
