"""The measurement entry points through the C ABI: the phase-profiled fused
shading launch must shade exactly as the plain launch does, and its phase
cycles must account for the tile loop; the gather microbenchmark must load
what it says (its sums are those of rows of the table)."""
import numpy as np
import pytest
import torch

import nvc_synth as S
from helpers import cfg_frame, scaled_params

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2506_05930_gb300 import nvc, _lib


def _frame_case(w=256, h=144):
    cfg = cfg_frame(precision="fp16", batch_positions=256)
    sc = S.scene_heightfield(seed=1, n_lights=32, n_spheres=32, n_boxes=32)
    gb = S.gbuffer_heightfield(seed=1, width=w, height=h)
    cache = nvc.VisibilityCache(cfg)
    cache.set_params(scaled_params(cfg, seed=3, table_scale=0.5))
    return cfg, cache, nvc.Scene.from_synth(sc), torch.from_numpy(gb.pos).cuda(), \
        torch.from_numpy(gb.nrm).cuda()


@pytest.mark.parametrize("variant", [6, 7])
def test_phase_profile_shades_like_the_plain_launch(variant):
    cfg, cache, scene, pos, nrm = _frame_case()
    nvc.nvc_set_shade_variant(cache.handle, variant)
    ref = cache.shade(scene, pos, nrm, seed=5, frame=2, view=0, fused=True)
    n = pos.shape[0]
    out = dict(idx=torch.full((n,), -7, dtype=torch.int32, device="cuda"),
               pdf=torch.full((n,), -1.0, device="cuda"), wsum=torch.full((n,), -1.0, device="cuda"),
               radiance=torch.full((n,), -1.0, device="cuda"))
    cyc = nvc.nvc_shade_phases(cache.handle, scene, pos, nrm, 5, 2, **out)
    torch.cuda.synchronize()
    for k in ref:
        assert torch.equal(out[k], ref[k]), k
    enc, mlp, smp, loop = cyc
    assert min(enc, mlp, smp) > 0
    # the three phases tile each tile's time; the loop adds only its own
    # bookkeeping between tiles
    assert 0.9 * loop <= enc + mlp + smp <= loop
    cache.close()


def test_phase_profile_rejects_other_variants():
    cfg, cache, scene, pos, nrm = _frame_case(64, 32)
    nvc.nvc_set_shade_variant(cache.handle, 0)
    with pytest.raises(_lib.NVCError) as e:
        nvc.nvc_shade_phases(cache.handle, scene, pos, nrm)
    assert e.value.status == _lib.NVC_ERR_UNSUPPORTED
    cache.close()


@pytest.mark.parametrize("row_bytes", [4, 8, 16])
def test_gather_bench_sums_rows_of_the_table(row_bytes):
    # a table whose every float is 1: a thread's sum is exactly the number
    # of floats it loaded, so a wrong row size or a skipped load shows
    n_floats = (1 << 20) // 4
    table = torch.ones(n_floats, device="cuda")
    n_threads, rows = 3000, 64
    sink = torch.zeros(n_threads, device="cuda")
    nvc.nvc_gather_bench(table, row_bytes, n_threads, rows, sink, seed=9)
    torch.cuda.synchronize()
    assert torch.all(sink == rows * row_bytes / 4)
    # rows drawn at random: a table of distinct values gives distinct sums
    table = torch.arange(n_floats, device="cuda", dtype=torch.float32)
    nvc.nvc_gather_bench(table, row_bytes, n_threads, rows, sink, seed=9)
    torch.cuda.synchronize()
    s = sink.cpu().numpy()
    assert len(np.unique(s)) > n_threads // 2
    assert s.min() >= 0 and s.max() <= rows * row_bytes / 4 * n_floats


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_mlp_on_given_features_matches_oracle(precision):
    """The MLP-only launch (the network's throughput apart from the encode):
    sigmoid(MLP(feat)) of given 16-bit operands, within about three times the
    measured FP16/BF16 error of the float64 oracle on the same operands, over
    a ragged last tile;
    both tile-stream layouts give the same bits; a wrong row width is an
    argument error."""
    from oracle import nvc as O
    cfg = cfg_frame(precision=precision, batch_positions=256)
    cache = nvc.VisibilityCache(cfg)
    p = scaled_params(cfg, seed=3, table_scale=0.5)
    cache.set_params(p)
    n, k0 = 5000, 32
    rng = np.random.default_rng(7)
    dtype = torch.float16 if precision == "fp16" else torch.bfloat16
    feat = torch.as_tensor(rng.uniform(-0.6, 0.6, (n, k0)).astype(np.float32)).to("cuda", dtype)
    outs = []
    for variant in (7, 6):
        nvc.nvc_set_shade_variant(cache.handle, variant)
        vis = torch.full((n, cfg.n_outputs), -1.0, device="cuda")
        nvc.nvc_mlp_infer_features(cache.handle, feat, vis)
        outs.append(vis.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    _, Ws = O.split_params(cfg, p)
    logits, _, _ = O.mlp_forward(Ws, feat.float().cpu().numpy().astype(np.float64), cfg.leaky_slope)
    ref = 1.0 / (1.0 + np.exp(-logits))
    # measured on GB300: max 9.2e-5 (FP16), 8.4e-4 (BF16); bounds about 3x that
    tol = 3e-4 if precision == "fp16" else 2.5e-3
    assert np.max(np.abs(outs[0] - ref)) < tol
    with pytest.raises(_lib.NVCError):
        nvc.nvc_mlp_infer_features(cache.handle, feat[:, :16].contiguous(), vis)
    cache.close()
