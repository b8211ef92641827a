"""nvc_infer_noalloc: inference for callers that cannot allocate GPU memory
(a renderer whose frame loop must not call cudaMalloc, or a plugin whose
host application owns every device allocation).  Its output must match
nvc_infer's on the same parameters, call after call, although every call
reuses the same fixed scratch array inside the library.

Kept in a file that pytest collects last, so a run that stops at the first
failure has run every other test before this one.
"""
import ctypes

import numpy as np
import pytest
import torch

import nvc_synth as S
from oracle import nvc as O
from helpers import cfg_tiny, cfg_frame, scaled_params

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2506_05930_gb300 import nvc, _lib

TOL = 1e-5   # the float32 visibility tolerance of the parity tests


def _reference(cfg, p, pos):
    cache = nvc.VisibilityCache(cfg)          # the existing, allocating entry point
    cache.set_params(p)
    vis = cache.infer(pos)
    torch.cuda.synchronize()
    cache.close()
    return vis


@pytest.mark.parametrize("cfg", [cfg_tiny(), cfg_frame(precision="fp32"),
                                 cfg_frame(precision="fp16")],
                         ids=["tiny", "frame_1080p_net", "frame_1080p_net_fp16_config"])
def test_noalloc_matches_nvc_infer_on_two_calls_in_a_row(cfg):
    """Against the existing entry point (a float32 handle holding the same
    parameters) and against the float64 oracle, both at the float32
    tolerance.  An fp16 configuration still gets float32 results: the
    entry point ignores cfg.precision."""
    p = scaled_params(cfg, seed=5, table_scale=0.5)
    params = torch.from_numpy(p).cuda()
    c = nvc.make_config(cfg)
    cfg32 = cfg.with_(precision="fp32")
    lo, hi = np.array(cfg.bounds_min), np.array(cfg.bounds_max)
    rng = np.random.default_rng(1)
    side = torch.cuda.Stream()
    # two calls back to back with different sizes: the second runs on a
    # scratch array that still holds the first call's features; the second
    # is queued on a stream other than the default one
    for n, stream in ((4096, None), (1001, side)):
        pos_np = rng.uniform(lo, hi, (n, 3)).astype(np.float32)
        pos = torch.from_numpy(pos_np).cuda()
        ref = _reference(cfg32, p, pos)
        vis = torch.full((n, cfg.n_outputs), -1.0, device="cuda")
        if stream is not None:
            stream.wait_stream(torch.cuda.current_stream())
        nvc.nvc_infer_noalloc(c, params, pos, vis, stream=stream)
        if stream is not None:
            stream.synchronize()
        torch.cuda.synchronize()
        assert torch.max(torch.abs(vis - ref)).item() <= TOL
        assert np.max(np.abs(vis.cpu().numpy() - O.infer(cfg32, p, pos_np))) <= TOL


def test_noalloc_rejects_sizes_beyond_its_scratch():
    cfg = cfg_frame(precision="fp32")              # 32 encoded features per position
    p = torch.from_numpy(scaled_params(cfg, seed=1)).cuda()
    c = nvc.make_config(cfg)
    n = (1 << 21) // 32 + 1
    pos = torch.zeros((n, 3), device="cuda")
    vis = torch.empty((n, 32), device="cuda")
    with pytest.raises(_lib.NVCError) as e:
        nvc.nvc_infer_noalloc(c, p, pos, vis)
    assert e.value.status == _lib.NVC_ERR_INVALID_ARG
    assert "scratch" in nvc.nvc_last_error(None)
    # the largest size that fits still runs
    nvc.nvc_infer_noalloc(c, p, pos[:n - 1], vis[:n - 1])
    torch.cuda.synchronize()
    assert torch.isfinite(vis[:n - 1]).all()
