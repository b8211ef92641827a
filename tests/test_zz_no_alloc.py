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


@pytest.mark.parametrize("cfg", [cfg_tiny(), cfg_frame(precision="fp32")],
                         ids=["tiny", "frame_1080p_net"])
def test_noalloc_matches_nvc_infer_on_two_calls_in_a_row(cfg):
    p = scaled_params(cfg, seed=5, table_scale=0.5)
    params = torch.from_numpy(p).cuda()
    c = nvc.make_config(cfg)
    lo, hi = np.array(cfg.bounds_min), np.array(cfg.bounds_max)
    rng = np.random.default_rng(1)
    # two calls back to back with different sizes: the second runs on a
    # scratch array that still holds the first call's features
    for n in (4096, 1001):
        pos = torch.from_numpy(rng.uniform(lo, hi, (n, 3)).astype(np.float32)).cuda()
        ref = _reference(cfg, p, pos)
        vis = torch.full((n, cfg.n_outputs), -1.0, device="cuda")
        nvc.nvc_infer_noalloc(c, params, pos, vis)
        torch.cuda.synchronize()
        assert torch.max(torch.abs(vis - ref)).item() <= TOL


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
