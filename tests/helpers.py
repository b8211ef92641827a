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


def fp16_gradient_model(cfg, params, pos, y, loss_scale, quantise=True):
    """The training gradient with the roundings the tensor-core path makes:
    encoded features, weights, hidden activations and the scaled deltas
    rounded to fp16, every product and sum in float64.  The distance of
    this model from the float64 oracle is the error fp16 operands cause;
    the CUDA path should sit on the model, not merely near the oracle.
    quantise=False skips the roundings, which must give the oracle's
    gradient (the model's structure is pinned that way)."""
    from oracle import nvc as O

    def q(x):
        x = np.asarray(x, np.float64)
        return x.astype(np.float16).astype(np.float64) if quantise else x

    table, Ws = O.split_params(cfg, params)
    feat, aux = O.encode(cfg, table, pos, with_aux=True)
    h = q(feat.astype(np.float32) if quantise else feat)
    Wq = [q(W) for W in Ws]
    acts = [h]
    for W in Wq[:-1]:
        z = h @ W.T
        h = q(np.where(z > 0, z, cfg.leaky_slope * z))
        acts.append(h)
    z = h @ Wq[-1].T
    s = 1.0 / (1.0 + np.exp(-z))
    n = z.size
    d = q(loss_scale * ((s - y) if cfg.loss == "bce" else 2 * (s - y) * s * (1 - s)))
    dWs = [None] * len(Wq)
    for k in range(len(Wq) - 1, -1, -1):
        dWs[k] = d.T @ acts[k] / n / loss_scale
        g = d @ Wq[k]
        if k > 0:
            d = q(g * np.where(acts[k] > 0, 1.0, cfg.leaky_slope))
        else:
            dfeat = g / n / loss_scale
    return O.join_params(O.encode_backward(cfg, aux, dfeat), dWs)
