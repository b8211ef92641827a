"""Hyper-parameter sets of the workloads (no method arithmetic here).

Each set names the hash-grid, MLP, loss and optimiser settings the CUDA path
and the oracle both run.  Where the paper and a workload's stated setting
differ, the workload's value is used and the paper's value is available as
the ``paper`` set (Section 3.3: 10 levels x 4 features, base resolution 16,
two hidden layers of 32, leaky ReLU 0.01, sigmoid output, L2 loss;
Section 3.4: He init, Adam, learning rate 0.05 -> 0.001 over 200 steps,
4096 world-space + 4096 screen-space training positions per frame).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Tuple


@dataclass(frozen=True)
class NVCConfig:
    name: str
    # multi-resolution hash grid (Section 3.3)
    n_levels: int = 8
    n_features: int = 2
    log2_table_size: int = 14
    base_resolution: int = 4
    growth: float = 1.5
    table_init: float = 1e-4          # table entries ~ U(-a, a)
    # MLP (Section 3.3): input = n_levels * n_features, no biases
    hidden: Tuple[int, ...] = (32, 32)
    n_outputs: int = 4                # one output neuron per light
    leaky_slope: float = 0.0          # 0 = ReLU; the paper uses 0.01
    init: str = "xavier_uniform"      # or "he_normal" (Section 3.4)
    # training (Section 3.4)
    loss: str = "l2"                  # "l2" (paper) or "bce"
    lr: float = 1e-2
    lr_schedule: str = "constant"     # or "paper_ramp"
    lr_end: float = 1e-3
    lr_ramp_steps: int = 200
    beta1: float = 0.9
    beta2: float = 0.99
    eps: float = 1e-15
    loss_scale: float = 1.0
    batch_positions: int = 1024       # half world-space, half screen-space
    # precision of the inference MLP and of the training forward/backward
    precision: str = "fp32"           # fp32 | fp16 | bf16 | fp8
    train_precision: str = "fp32"     # fp32 | fp16
    # hash-table features the fused inference kernels read: the float32
    # master or a half-precision copy of it
    table_precision: str = "fp32"     # fp32 | fp16
    # encoding domain (positions are normalised into [0,1]^3 by these)
    bounds_min: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    bounds_max: Tuple[float, float, float] = (1.0, 1.0, 1.0)

    @property
    def n_inputs(self) -> int:
        return self.n_levels * self.n_features

    @property
    def table_size(self) -> int:
        return 1 << self.log2_table_size

    def with_(self, **kw) -> "NVCConfig":
        return replace(self, **kw)


# Tiny plain FP32 path: 64x64 points in [0,1]^3, 4 lights, 4 spheres,
# 8 levels x 2 features, T = 2^14, base 4, growth 1.5, MLP 16->32->32->4
# ReLU + sigmoid, Xavier init, one Adam step (lr 1e-2) on 1024 positions x
# 4 lights = 4096 shadow-ray samples.
TINY_FP32 = NVCConfig(name="tiny_fp32")

# 1080p inference workload: heightfield + boxes in [0,10]^3, 32 lights,
# 64 occluders, 16 levels x 2 features, T = 2^19, base 16, growth 1.447,
# MLP 32->64->64->64->32 in FP16 with FP32 accumulation, the tensor-core
# inference reading an FP16 copy of the FP32 master table; trained online
# with 8192 positions x 32 lights per frame.
FRAME_1080P = NVCConfig(
    name="frame_1080p", n_levels=16, n_features=2, log2_table_size=19,
    base_resolution=16, growth=1.447, hidden=(64, 64, 64), n_outputs=32,
    leaky_slope=0.01, loss="bce", batch_positions=8192, precision="fp16",
    train_precision="fp16", loss_scale=128.0, table_precision="fp16",
    bounds_min=(0.0, 0.0, 0.0), bounds_max=(10.0, 10.0, 10.0))

# Online training on the tiny scene: 16384 positions x 4 lights = 65,536
# (position, light) samples per frame, BCE, Adam (0.9, 0.99), lr 1e-2,
# FP16 compute with FP32 master weights, static loss scale 128.
ONLINE_TRAIN = TINY_FP32.with_(
    name="online_train", loss="bce", batch_positions=16384,
    precision="fp16", train_precision="fp16", loss_scale=128.0)

# Batched multi-view frame: 128 lights, MLP 32->64->64->64->128, grid as
# the 1080p workload (float32 table features: the 128-light kernels run
# slower on the half-precision copy), unit-cube scene.
MULTIVIEW = FRAME_1080P.with_(
    name="multiview", n_outputs=128, bounds_max=(1.0, 1.0, 1.0), table_precision="fp32")

# Precision sweep at 4K: 256 lights, 256 occluders, T = 2^21, FP16
# hash-table features.
PRECISION_4K = FRAME_1080P.with_(
    name="precision_4k", log2_table_size=21, n_outputs=256)

# Clustered cache on the 1080p workload (Section 3.6): k = 32 cluster
# outputs over the 16-room scene with 1024 lights, 8 levels with base resolution 2 (the
# paper's setting for the smoother cluster visibility; growth 2, not
# stated, gives a finest level of 256), 49,152 training positions per frame
# (the paper's count for its many-lights scene); the rest as frame_1080p.
CLUSTERED_1080P = FRAME_1080P.with_(
    name="clustered_1080p", n_levels=8, base_resolution=2, growth=2.0,
    batch_positions=49152)

# The paper's own settings (Sections 3.3-3.4); T and growth are not stated
# in the paper and take the tiny workload's values.
PAPER = NVCConfig(
    name="paper", n_levels=10, n_features=4, log2_table_size=14,
    base_resolution=16, growth=1.5, hidden=(32, 32), n_outputs=32,
    leaky_slope=0.01, init="he_normal", loss="l2", lr=0.05,
    lr_schedule="paper_ramp", lr_end=1e-3, lr_ramp_steps=200,
    batch_positions=8192, bounds_max=(10.0, 10.0, 10.0))

CONFIGS = {c.name: c for c in
           (TINY_FP32, FRAME_1080P, ONLINE_TRAIN, MULTIVIEW, PRECISION_4K,
            CLUSTERED_1080P, PAPER)}


def config_by_name(name: str) -> NVCConfig:
    return CONFIGS[name]


def param_layout(cfg: NVCConfig):
    """Offsets of the table and of each weight matrix in the flat vector.

    Returns (table_offset, table_numel, [(offset, n_out, n_in), ...]).
    """
    table_numel = cfg.n_levels * cfg.table_size * cfg.n_features
    layers = []
    off = table_numel
    dims = [cfg.n_inputs, *cfg.hidden, cfg.n_outputs]
    for i in range(len(dims) - 1):
        layers.append((off, dims[i + 1], dims[i]))
        off += dims[i + 1] * dims[i]
    return 0, table_numel, layers


def param_count(cfg: NVCConfig) -> int:
    _, tn, layers = param_layout(cfg)
    return tn + sum(o * i for _, o, i in layers)
