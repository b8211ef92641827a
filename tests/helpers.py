"""Shared test helpers: workload construction for the CUDA path and the oracle."""
import numpy as np

import nvc_synth as S


def cfg_tiny(**kw):
    return S.config_by_name("tiny_fp32").with_(**kw)


def cfg_frame(**kw):
    return S.config_by_name("frame_1080p").with_(**kw)


def scaled_params(cfg, seed=0, table_scale=1.0):
    """Initial parameters with table entries scaled up so the encoding and
    the network outputs are far from zero (more telling comparisons)."""
    p = S.init_params(cfg, seed=seed).astype(np.float64)
    n_table = cfg.n_levels * cfg.table_size * cfg.n_features
    p[:n_table] *= table_scale / cfg.table_init
    return p.astype(np.float32)


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
