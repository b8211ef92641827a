"""Python binding of libnvc: the C entry points under the same names, taking
torch tensors (argument marshalling only; every step runs in the library's
CUDA kernels), plus a small ``VisibilityCache`` convenience class.

torch is used for device memory and streams only.  Tensors must be CUDA,
contiguous and of the stated dtype; the default stream argument is torch's
current stream.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional, Sequence

import torch

from . import _lib
from ._lib import NvcClusters, NvcConfig, NvcCounters, NvcScene, NvcView, NVCError, check

lib = _lib.load()

NO_TRAINING = -2      # nvc_frame train_view: shade only
WORLD_ONLY = -1       # nvc_frame train_view: train on world-space positions only


# ----------------------------------------------------------------- helpers --

def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t: Optional[torch.Tensor], dtype=torch.float32, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


# The C entry points take bare pointers and sizes, so a tensor shorter than
# the extent a call reads or writes would let a kernel run past it.  The
# wrappers check every tensor's extent against the call's n, the handle's
# shapes (recorded here by nvc_create) and the scene's light count before
# anything is launched.
@dataclass(frozen=True)
class HandleShapes:
    n_outputs: int      # L: visibilities per position
    enc_width: int      # levels x features
    n_params: int
    precision: int      # _lib.PRECISIONS value of the inference operands
    batch: int          # training positions per step


_HANDLE_SHAPES: dict = {}


def _shapes(h) -> Optional[HandleShapes]:
    return _HANDLE_SHAPES.get(h.value if isinstance(h, ctypes.c_void_p) else h)


def _rows(t, cols: int, name: str) -> int:
    """n of a [n, cols] tensor (the row count a call is given)."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dim() != 2 or t.shape[1] != cols:
        raise ValueError(f"{name} must be [n, {cols}], got {tuple(t.shape)}")
    return int(t.shape[0])


def _holds(t, count: int, name: str):
    """A tensor the call reads or writes `count` elements of (None passes)."""
    if t is None:
        return
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.numel() < count:
        raise ValueError(f"{name} holds {t.numel()} elements; the call uses {count}")


def _outputs_per_pixel(h) -> Optional[int]:
    s = _shapes(h)
    return None if s is None else s.n_outputs


def _cluster_count(clusters) -> int:
    """k for the extent checks; a k outside 1..32 is left to the library,
    which rejects it."""
    k = int(clusters.struct.k)
    return k if 1 <= k <= 32 else 0


def _pixels(pos, nrm=None, per_pixel=(), name="pos") -> int:
    """n from pos [n, 3]; nrm holds n rows of 3, the per-pixel tensors n
    elements."""
    n = _rows(pos, 3, name)
    if nrm is not None:
        if _rows(nrm, 3, "nrm") < n:
            raise ValueError(f"nrm has {nrm.shape[0]} rows, pos {n}")
    for t, nm in per_pixel:
        _holds(t, n, nm)
    return n


def make_config(cfg=None, **kw) -> NvcConfig:
    """nvc_config from an object/dict with the fields of the workload sets
    (``hidden`` is a tuple of equal widths) plus keyword overrides."""
    src = {}
    if cfg is not None:
        src.update(cfg if isinstance(cfg, dict) else
                   {k: getattr(cfg, k) for k in dir(cfg) if not k.startswith("_")})
    src.update(kw)
    hidden = tuple(src.get("hidden", (32, 32)))
    if len(set(hidden)) != 1:
        raise ValueError("hidden layers must share one width")
    c = NvcConfig()
    c.n_levels = int(src.get("n_levels", 8))
    c.n_features = int(src.get("n_features", 2))
    c.log2_table_size = int(src.get("log2_table_size", 14))
    c.base_resolution = int(src.get("base_resolution", 4))
    c.growth = float(src.get("growth", 1.5))
    c.n_hidden = len(hidden)
    c.hidden_width = int(hidden[0])
    c.n_outputs = int(src.get("n_outputs", 4))
    c.leaky_slope = float(src.get("leaky_slope", 0.0))
    c.precision = _lib.PRECISIONS[src.get("precision", "fp32")]
    c.train_precision = _lib.PRECISIONS[src.get("train_precision", "fp32")]
    c.loss = _lib.LOSSES[src.get("loss", "l2")]
    c.lr_schedule = _lib.LR_SCHEDULES[src.get("lr_schedule", "constant")]
    c.lr = float(src.get("lr", 1e-2))
    c.lr_end = float(src.get("lr_end", 1e-3))
    c.lr_ramp_steps = int(src.get("lr_ramp_steps", 200))
    c.beta1 = float(src.get("beta1", 0.9))
    c.beta2 = float(src.get("beta2", 0.99))
    c.eps = float(src.get("eps", 1e-15))
    c.loss_scale = float(src.get("loss_scale", 1.0))
    c.batch_positions = int(src.get("batch_positions", 1024))
    for d in range(3):
        c.bounds_min[d] = float(src.get("bounds_min", (0, 0, 0))[d])
        c.bounds_max[d] = float(src.get("bounds_max", (1, 1, 1))[d])
    return c


class Scene:
    """Device copies of a scene's lights/occluders and the nvc_scene view."""

    def __init__(self, lights, spheres=None, boxes=None, world_min=(0, 0, 0),
                 world_max=(1, 1, 1), device="cuda"):
        def dev(a, cols):
            t = torch.as_tensor(a if a is not None else torch.zeros((0, cols)),
                                dtype=torch.float32).reshape(-1, cols)
            return t.to(device).contiguous()
        self.lights = dev(lights, 4)
        self.spheres = dev(spheres, 4)
        self.boxes = dev(boxes, 6)
        s = NvcScene()
        s.lights = self.lights.data_ptr()
        s.n_lights = self.lights.shape[0]
        s.spheres = self.spheres.data_ptr() if self.spheres.numel() else None
        s.n_spheres = self.spheres.shape[0]
        s.boxes = self.boxes.data_ptr() if self.boxes.numel() else None
        s.n_boxes = self.boxes.shape[0]
        for d in range(3):
            s.world_min[d] = float(world_min[d])
            s.world_max[d] = float(world_max[d])
        self.struct = s

    @classmethod
    def from_synth(cls, sc, device="cuda"):
        return cls(sc.lights, sc.spheres, sc.boxes, sc.world_min, sc.world_max, device)

    @property
    def ref(self):
        return ctypes.byref(self.struct)


# --------------------------------------------- the C entry points by name --

def nvc_param_count(cfg: NvcConfig) -> int:
    return int(lib.nvc_param_count(ctypes.byref(cfg)))


def nvc_level_resolution(cfg: NvcConfig, level: int) -> int:
    return int(lib.nvc_level_resolution(ctypes.byref(cfg), level))


def nvc_create(cfg: NvcConfig):
    h = ctypes.c_void_p()
    check(lib.nvc_create(ctypes.byref(cfg), ctypes.byref(h)))
    _HANDLE_SHAPES[h.value] = HandleShapes(
        n_outputs=int(cfg.n_outputs), enc_width=int(cfg.n_levels * cfg.n_features),
        n_params=nvc_param_count(cfg), precision=int(cfg.precision),
        batch=int(cfg.batch_positions))
    return h


def nvc_destroy(h):
    _HANDLE_SHAPES.pop(h.value if isinstance(h, ctypes.c_void_p) else h, None)
    lib.nvc_destroy(h)


def nvc_last_error(h=None) -> str:
    return lib.nvc_last_error(h).decode(errors="replace")


def _params_like(h, tensors):
    s = _shapes(h)
    if s is not None:
        for t, name in tensors:
            _holds(t, s.n_params, name)


def nvc_set_state(h, params, adam_m=None, adam_v=None, step=0, stream=None):
    _params_like(h, ((params, "params"), (adam_m, "adam_m"), (adam_v, "adam_v")))
    check(lib.nvc_set_state(h, _ptr(params, name="params"), _ptr(adam_m, name="adam_m"),
                            _ptr(adam_v, name="adam_v"), int(step), _stream(stream)), h)


def nvc_set_params(h, params, stream=None):
    _params_like(h, ((params, "params"),))
    check(lib.nvc_set_params(h, _ptr(params, name="params"), _stream(stream)), h)


def nvc_get_state(h, params=None, adam_m=None, adam_v=None, stream=None):
    _params_like(h, ((params, "params"), (adam_m, "adam_m"), (adam_v, "adam_v")))
    check(lib.nvc_get_state(h, _ptr(params), _ptr(adam_m), _ptr(adam_v), _stream(stream)), h)


def nvc_set_staging(h, max_pixels: int):
    check(lib.nvc_set_staging(h, int(max_pixels)), h)


def nvc_sync_status(h, stream=None) -> dict:
    c = NvcCounters()
    check(lib.nvc_sync_status(h, _stream(stream), ctypes.byref(c)), h)
    return dict(step=c.step, skipped=c.skipped, error_flags=c.error_flags, frames=c.frames)


def nvc_encode(h, pos, feat, stream=None):
    n = _pixels(pos)
    s = _shapes(h)
    if s is not None:
        _holds(feat, n * s.enc_width, "feat")
    check(lib.nvc_encode(h, _ptr(pos, name="pos"), pos.shape[0], _ptr(feat, name="feat"),
                         _stream(stream)), h)


def nvc_mlp_infer_features(h, feat, vis, stream=None):
    """feat: CUDA [n][K0] float16 or bfloat16 tensor (the handle's operand
    type), vis: CUDA [n][L] float32."""
    if not isinstance(feat, torch.Tensor) or not feat.is_cuda or feat.dim() != 2:
        raise ValueError("feat must be a 2-D CUDA tensor")
    if feat.dtype not in (torch.float16, torch.bfloat16) or not feat.is_contiguous():
        raise ValueError("feat must be contiguous float16 or bfloat16")
    if vis.shape[0] != feat.shape[0]:
        raise ValueError("feat and vis must have the same number of rows")
    s = _shapes(h)
    if s is not None:
        _holds(vis, feat.shape[0] * s.n_outputs, "vis")
        want = {_lib.PRECISIONS["fp16"]: torch.float16, _lib.PRECISIONS["bf16"]: torch.bfloat16}
        if s.precision in want and feat.dtype != want[s.precision]:
            raise TypeError(f"feat must be {want[s.precision]} for this handle")
    check(lib.nvc_mlp_infer_features(h, feat.data_ptr(), feat.shape[0], feat.shape[1],
                                     _ptr(vis, name="vis"), _stream(stream)), h)


def nvc_infer(h, pos, vis, stream=None):
    n = _pixels(pos)
    L = _outputs_per_pixel(h)
    if L is not None:
        _holds(vis, n * L, "vis")
    check(lib.nvc_infer(h, _ptr(pos, name="pos"), pos.shape[0], _ptr(vis, name="vis"),
                        _stream(stream)), h)


def nvc_light_weights(scene: Scene, pos, nrm, vis, c, w=None, stream=None):
    n = _pixels(pos, nrm)
    L = scene.struct.n_lights
    for t, name in ((vis, "vis"), (c, "c"), (w, "w")):
        _holds(t, n * L, name)
    check(lib.nvc_light_weights(scene.ref, _ptr(pos), _ptr(nrm), _ptr(vis), pos.shape[0],
                                _ptr(c), _ptr(w), _stream(stream)))


def nvc_wrs_from_weights(w, seed, frame, view=0, pixel_offset=0, idx=None, pdf=None,
                         wsum=None, stream=None):
    if not isinstance(w, torch.Tensor) or w.dim() != 2:
        raise ValueError("w must be a [n, n_lights] tensor")
    for t, name in ((idx, "idx"), (pdf, "pdf"), (wsum, "wsum")):
        _holds(t, w.shape[0], name)
    check(lib.nvc_wrs_from_weights(_ptr(w, name="w"), w.shape[0], w.shape[1], int(seed),
                                   int(frame), int(view), int(pixel_offset),
                                   _ptr(idx, torch.int32, "idx"), _ptr(pdf), _ptr(wsum),
                                   _stream(stream)))


def nvc_wrs_sample(h, scene: Scene, pos, nrm, seed, frame, view=0, pixel_offset=0, idx=None,
                   pdf=None, wsum=None, stream=None):
    _pixels(pos, nrm, ((idx, "idx"), (pdf, "pdf"), (wsum, "wsum")))
    check(lib.nvc_wrs_sample(h, scene.ref, _ptr(pos), _ptr(nrm), pos.shape[0], int(seed),
                             int(frame), int(view), int(pixel_offset),
                             _ptr(idx, torch.int32, "idx"), _ptr(pdf), _ptr(wsum),
                             _stream(stream)), h)


def nvc_direct_illum(h, scene: Scene, pos, nrm, radiance, stream=None):
    _pixels(pos, nrm, ((radiance, "radiance"),))
    check(lib.nvc_direct_illum(h, scene.ref, _ptr(pos), _ptr(nrm), pos.shape[0],
                               _ptr(radiance), _stream(stream)), h)


def nvc_shade(h, scene: Scene, pos, nrm, seed, frame, view=0, pixel_offset=0, idx=None,
              pdf=None, wsum=None, radiance=None, fused=True, stream=None):
    _pixels(pos, nrm, ((idx, "idx"), (pdf, "pdf"), (wsum, "wsum"), (radiance, "radiance")))
    check(lib.nvc_shade(h, scene.ref, _ptr(pos), _ptr(nrm), pos.shape[0], int(seed),
                        int(frame), int(view), int(pixel_offset),
                        _ptr(idx, torch.int32, "idx"), _ptr(pdf), _ptr(wsum), _ptr(radiance),
                        1 if fused else 0, _stream(stream)), h)


def nvc_sampler_weights(h, scene: Scene, pos, nrm, w, stream=None):
    n = _pixels(pos, nrm)
    L = _outputs_per_pixel(h)
    if L is not None:
        _holds(w, n * L, "w")
    check(lib.nvc_sampler_weights(h, scene.ref, _ptr(pos), _ptr(nrm), pos.shape[0], _ptr(w),
                                  _stream(stream)), h)


SHADE_VARIANTS = 8


def nvc_autotune_shade(h, scene: Scene, pos, nrm, idx=None, pdf=None, wsum=None, radiance=None,
                       reps=5, stream=None):
    """Times the fused shading kernel's variants on these pixels and keeps
    the fastest.  Returns (chosen variant, [ms per launch or -1])."""
    _pixels(pos, nrm, ((idx, "idx"), (pdf, "pdf"), (wsum, "wsum"), (radiance, "radiance")))
    chosen = ctypes.c_int32()
    ms = (ctypes.c_double * SHADE_VARIANTS)()
    check(lib.nvc_autotune_shade(h, scene.ref, _ptr(pos), _ptr(nrm), pos.shape[0],
                                 _ptr(idx, torch.int32, "idx"), _ptr(pdf), _ptr(wsum),
                                 _ptr(radiance), int(reps), ctypes.byref(chosen), ms,
                                 _stream(stream)), h)
    return int(chosen.value), list(ms)


def nvc_autotune_infer(h, pos, vis, reps=5, stream=None):
    """Times nvc_infer under each fused-kernel variant (vis is scratch) and
    keeps the fastest for this handle's nvc_infer.  Returns (chosen variant,
    [ms per call or -1])."""
    n = _pixels(pos)
    L = _outputs_per_pixel(h)
    if L is not None:
        _holds(vis, n * L, "vis")
    chosen = ctypes.c_int32()
    ms = (ctypes.c_double * SHADE_VARIANTS)()
    check(lib.nvc_autotune_infer(h, _ptr(pos, name="pos"), pos.shape[0], _ptr(vis, name="vis"),
                                 int(reps), ctypes.byref(chosen), ms, _stream(stream)), h)
    return int(chosen.value), list(ms)


def nvc_calibrate(h, pos, stream=None):
    """Per-tensor E4M3 activation scales from a float32 pass over pos."""
    _pixels(pos)
    check(lib.nvc_calibrate(h, _ptr(pos, name="pos"), pos.shape[0], _stream(stream)), h)


def nvc_set_table_precision(h, precision: str, stream=None):
    """"fp16": the fused inference kernels read a half-precision copy of the
    hash table, refreshed after every parameter change; "fp32": the master."""
    check(lib.nvc_set_table_precision(h, _lib.PRECISIONS[precision], _stream(stream)), h)


def nvc_set_shade_plan(h, variant: int, ctas_per_sm: int = 0):
    check(lib.nvc_set_shade_plan(h, ctypes.byref(_lib.NvcShadePlan(int(variant), int(ctas_per_sm)))), h)


def nvc_autotune_shade_plan(h, scene: Scene, pos, nrm, idx=None, pdf=None, wsum=None,
                            radiance=None, reps=5, stream=None):
    """Times every point (variant, CTAs per SM) of the fused shading
    kernel's tuning space on these pixels and keeps the fastest.  Returns
    ((variant, ctas_per_sm) chosen, [((variant, ctas_per_sm), ms), ...])."""
    _pixels(pos, nrm, ((idx, "idx"), (pdf, "pdf"), (wsum, "wsum"), (radiance, "radiance")))
    cap = 64
    chosen = _lib.NvcShadePlan()
    pts = (_lib.NvcShadePlan * cap)()
    ms = (ctypes.c_double * cap)()
    n = ctypes.c_int32()
    check(lib.nvc_autotune_shade_plan(h, scene.ref, _ptr(pos), _ptr(nrm), pos.shape[0],
                                      _ptr(idx, torch.int32, "idx"), _ptr(pdf), _ptr(wsum),
                                      _ptr(radiance), int(reps), ctypes.byref(chosen), pts, ms, cap,
                                      ctypes.byref(n), _stream(stream)), h)
    tried = [((pts[i].variant, pts[i].ctas_per_sm), ms[i]) for i in range(min(n.value, cap))]
    return (chosen.variant, chosen.ctas_per_sm), tried


def nvc_set_shade_variant(h, variant: int):
    check(lib.nvc_set_shade_variant(h, int(variant)), h)


def nvc_shade_phases(h, scene: Scene, pos, nrm, seed=0, frame=0, idx=None, pdf=None, wsum=None,
                     radiance=None, stream=None):
    """One instrumented fused shading launch (variants 6 and 7): returns the
    summed SM cycles of [encode, MLP, sampler, whole tile loop]."""
    _pixels(pos, nrm, ((idx, "idx"), (pdf, "pdf"), (wsum, "wsum"), (radiance, "radiance")))
    cyc = (ctypes.c_double * 4)()
    check(lib.nvc_shade_phases(h, scene.ref, _ptr(pos, name="pos"), _ptr(nrm, name="nrm"),
                               pos.shape[0], int(seed), int(frame),
                               _ptr(idx, torch.int32, "idx"), _ptr(pdf), _ptr(wsum),
                               _ptr(radiance), cyc, _stream(stream)), h)
    return list(cyc)


def nvc_gather_bench(table, row_bytes, n_threads, rows_per_thread, sink, seed=0, stream=None):
    """Queues the random-row gather microbenchmark over `table` (a CUDA
    tensor of a power-of-two byte size); the caller times it."""
    if not isinstance(table, torch.Tensor) or not table.is_cuda or not table.is_contiguous():
        raise ValueError("table must be a contiguous CUDA tensor")
    if sink.numel() < n_threads:
        raise ValueError("sink must hold n_threads floats")
    check(lib.nvc_gather_bench(table.data_ptr(), table.numel() * table.element_size(),
                               int(row_bytes), int(n_threads), int(rows_per_thread), int(seed),
                               _ptr(sink, name="sink"), _stream(stream)))


def nvc_trace_visibility(scene: Scene, pos, vis, stream=None):
    n = _pixels(pos)
    _holds(vis, n * scene.struct.n_lights, "vis")
    check(lib.nvc_trace_visibility(scene.ref, _ptr(pos), pos.shape[0], _ptr(vis),
                                   _stream(stream)))


def nvc_training_positions(scene: Scene, screen_pos, batch, seed, frame, pos, stream=None):
    n_screen = 0 if screen_pos is None else _rows(screen_pos, 3, "screen_pos")
    _holds(pos, int(batch) * 3, "pos")
    check(lib.nvc_training_positions(scene.ref, _ptr(screen_pos), n_screen, int(batch),
                                     int(seed), int(frame), _ptr(pos), _stream(stream)))


def nvc_training_positions_split(scene: Scene, screen_pos, batch, n_world, seed, frame, pos,
                                 stream=None):
    n_screen = 0 if screen_pos is None else _rows(screen_pos, 3, "screen_pos")
    _holds(pos, int(batch) * 3, "pos")
    check(lib.nvc_training_positions_split(scene.ref, _ptr(screen_pos), n_screen, int(batch),
                                           int(n_world), int(seed), int(frame), _ptr(pos),
                                           _stream(stream)))


def nvc_set_training_data_fused(h, fused: bool):
    """FP16 training makes its positions and shadow-ray targets inside the
    tensor-core training kernel (True) or in a launch of their own (False)."""
    check(lib.nvc_set_training_data_fused(h, 1 if fused else 0), h)


def nvc_training_batch(h, pos=None, target=None, stream=None):
    """Copies the last training step's positions [B, 3] and targets [B, L] out."""
    s = _shapes(h)
    if s is not None:
        _holds(pos, s.batch * 3, "pos")
        _holds(target, s.batch * s.n_outputs, "target")
    check(lib.nvc_training_batch(h, _ptr(pos, name="pos"), _ptr(target, name="target"),
                                 _stream(stream)), h)


def nvc_set_training_placement(h, n_world: int):
    check(lib.nvc_set_training_placement(h, int(n_world)), h)


def nvc_train_step(h, scene: Scene, screen_pos, seed, frame, loss_out=None, stream=None):
    n_screen = 0 if screen_pos is None else _rows(screen_pos, 3, "screen_pos")
    check(lib.nvc_train_step(h, scene.ref, _ptr(screen_pos), n_screen, int(seed), int(frame),
                             _ptr(loss_out, torch.float64, "loss_out"), _stream(stream)), h)


def nvc_train_gradient(h, scene: Scene, screen_pos, seed, frame, grad, loss_out=None,
                       stream=None):
    n_screen = 0 if screen_pos is None else _rows(screen_pos, 3, "screen_pos")
    _params_like(h, ((grad, "grad"),))
    check(lib.nvc_train_gradient(h, scene.ref, _ptr(screen_pos), n_screen, int(seed),
                                 int(frame), _ptr(grad), _ptr(loss_out, torch.float64),
                                 _stream(stream)), h)


def nvc_mlp_forward(h, pos, logits, stream=None):
    n = _pixels(pos)
    L = _outputs_per_pixel(h)
    if L is not None:
        _holds(logits, n * L, "logits")
    check(lib.nvc_mlp_forward(h, _ptr(pos), pos.shape[0], _ptr(logits), _stream(stream)), h)


def nvc_mlp_backward(h, pos, dlogits, grad, stream=None):
    n = _pixels(pos)
    L = _outputs_per_pixel(h)
    if L is not None:
        _holds(dlogits, n * L, "dlogits")
    _params_like(h, ((grad, "grad"),))
    check(lib.nvc_mlp_backward(h, _ptr(pos), pos.shape[0], _ptr(dlogits), _ptr(grad),
                               _stream(stream)), h)


@dataclass
class View:
    """One view of a frame and its output tensors."""
    pos: torch.Tensor
    nrm: torch.Tensor
    view_id: int = 0
    idx: Optional[torch.Tensor] = None
    pdf: Optional[torch.Tensor] = None
    wsum: Optional[torch.Tensor] = None
    radiance: Optional[torch.Tensor] = None

    def check_extents(self):
        _pixels(self.pos, self.nrm, ((self.idx, "idx"), (self.pdf, "pdf"), (self.wsum, "wsum"),
                                     (self.radiance, "radiance")))

    def struct(self) -> NvcView:
        self.check_extents()
        v = NvcView()
        v.pos = _ptr(self.pos)
        v.nrm = _ptr(self.nrm)
        v.n_pixels = self.pos.shape[0]
        v.view_id = self.view_id
        v.idx = _ptr(self.idx, torch.int32, "idx")
        v.pdf = _ptr(self.pdf)
        v.wsum = _ptr(self.wsum)
        v.radiance = _ptr(self.radiance)
        return v


def nvc_frame(h, scene: Scene, views: Sequence[View], train_view, seed, frame, loss_out=None,
              use_graph=True, stream=None):
    arr = (NvcView * max(1, len(views)))(*[v.struct() for v in views])
    check(lib.nvc_frame(h, scene.ref, arr, len(views), WORLD_ONLY if train_view is None else train_view,
                        int(seed), int(frame), _ptr(loss_out, torch.float64, "loss_out"),
                        1 if use_graph else 0, _stream(stream)), h)


def _host_ptr(t: Optional[torch.Tensor], dtype=torch.float32, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.is_cuda:
        raise ValueError(f"{name} must be a host tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _host_view(v: "View") -> NvcView:
    v.check_extents()
    s = NvcView()
    s.pos = _host_ptr(v.pos, name="pos")
    s.nrm = _host_ptr(v.nrm, name="nrm")
    s.n_pixels = v.pos.shape[0]
    s.view_id = int(v.view_id)
    s.idx = _host_ptr(v.idx, torch.int32, "idx")
    s.pdf = _host_ptr(v.pdf, name="pdf")
    s.wsum = _host_ptr(v.wsum, name="wsum")
    s.radiance = _host_ptr(v.radiance, name="radiance")
    return s


def nvc_frame_host(h, scene: Scene, views: Sequence[View], train_view, seed, frame, loss_out=None,
                   use_graph=True, stream=None):
    """nvc_frame with every view's tensors in (pinned) host memory; returns
    at once, the read-back completes in stream order after
    nvc_host_frames_wait."""
    arr = (NvcView * max(1, len(views)))(*[_host_view(v) for v in views])
    check(lib.nvc_frame_host(h, scene.ref, arr, len(views),
                             WORLD_ONLY if train_view is None else train_view, int(seed), int(frame),
                             _ptr(loss_out, torch.float64, "loss_out"), 1 if use_graph else 0,
                             _stream(stream)), h)


def nvc_host_frames_wait(h, stream=None):
    check(lib.nvc_host_frames_wait(h, _stream(stream)), h)


def nvc_shade_estimate(scene: Scene, pos, nrm, idx, pdf, estimate=None, accum=None, count=1,
                       stream=None):
    """V c / pdf for each pixel's sampled light (one shadow ray), and/or its
    running mean over `count` frames into `accum`."""
    _pixels(pos, nrm, ((idx, "idx"), (pdf, "pdf"), (estimate, "estimate"), (accum, "accum")))
    check(lib.nvc_shade_estimate(scene.ref, _ptr(pos, name="pos"), _ptr(nrm, name="nrm"),
                                 pos.shape[0], _ptr(idx, torch.int32, "idx"), _ptr(pdf, name="pdf"),
                                 _ptr(estimate, name="estimate"), _ptr(accum, name="accum"),
                                 int(count), _stream(stream)))


def nvc_exact_di(scene: Scene, pos, nrm, di, stream=None):
    """Sum over all lights of V_i c_i, one shadow ray per (pixel, light)."""
    _pixels(pos, nrm, ((di, "di"),))
    check(lib.nvc_exact_di(scene.ref, _ptr(pos, name="pos"), _ptr(nrm, name="nrm"), pos.shape[0],
                           _ptr(di, name="di"), _stream(stream)))


def nvc_kmeans_lights(lights, init, iters):
    """Lloyd's k-means of the light positions (host, float64) from the seed
    lights `init`; returns (assign int32 [n], centroids float64 [k, 3])."""
    import numpy as np
    L = np.ascontiguousarray(np.asarray(lights, np.float32).reshape(-1, 4))
    init = np.ascontiguousarray(np.asarray(init, np.int32))
    assign = np.empty(L.shape[0], np.int32)
    cent = np.empty((init.shape[0], 3), np.float64)
    check(lib.nvc_kmeans_lights(L.ctypes.data, L.shape[0], init.ctypes.data, init.shape[0],
                                int(iters), assign.ctypes.data, cent.ctypes.data))
    return assign, cent


class Clusters:
    """Device CSR table of a light clustering and its nvc_clusters view;
    `weights` names the sampler's first-step weights ("sum" or
    "visibility", NVC_CLUSTER_WEIGHT_*)."""

    def __init__(self, assign, k, device="cuda", weights="sum"):
        import numpy as np
        assign = np.asarray(assign, np.int64)
        order = np.argsort(assign, kind="stable")
        counts = np.bincount(assign, minlength=k)
        self.offsets = torch.as_tensor(np.concatenate([[0], np.cumsum(counts)]), dtype=torch.int32).to(device)
        self.members = torch.as_tensor(order, dtype=torch.int32).to(device)
        c = NvcClusters()
        c.k = int(k)
        c.offsets = self.offsets.data_ptr()
        c.members = self.members.data_ptr()
        c.weights = _lib.CLUSTER_WEIGHTS[weights]
        self.struct = c

    @property
    def ref(self):
        return ctypes.byref(self.struct)


def nvc_train_step_clustered(h, scene: Scene, clusters: Clusters, screen_pos, seed, frame,
                             loss_out=None, stream=None):
    n_screen = 0 if screen_pos is None else _rows(screen_pos, 3, "screen_pos")
    check(lib.nvc_train_step_clustered(h, scene.ref, clusters.ref, _ptr(screen_pos), n_screen,
                                       int(seed), int(frame), _ptr(loss_out, torch.float64, "loss_out"),
                                       _stream(stream)), h)


def nvc_cluster_targets(scene: Scene, clusters: Clusters, pos, seed, frame, target, stream=None):
    n = _pixels(pos)
    _holds(target, n * _cluster_count(clusters), "target")
    check(lib.nvc_cluster_targets(scene.ref, clusters.ref, _ptr(pos, name="pos"), pos.shape[0],
                                  int(seed), int(frame), _ptr(target, name="target"), _stream(stream)))


def nvc_sample_clustered(scene: Scene, clusters: Clusters, vis, pos, nrm, seed, frame, view=0,
                         pixel_offset=0, light=None, weight=None, estimate=None, stream=None):
    n = _pixels(pos, nrm, ((light, "light"), (weight, "weight"), (estimate, "estimate")))
    _holds(vis, n * _cluster_count(clusters), "vis")
    check(lib.nvc_sample_clustered(scene.ref, clusters.ref, _ptr(vis, name="vis"),
                                   _ptr(pos, name="pos"), _ptr(nrm, name="nrm"), pos.shape[0],
                                   int(pixel_offset), int(seed), int(frame), int(view),
                                   _ptr(light, torch.int32, "light"), _ptr(weight, name="weight"),
                                   _ptr(estimate, name="estimate"), _stream(stream)))


def nvc_temporal_merge(scene: Scene, pos, nrm, cur_light, cur_W, prev_light=None, prev_W=None,
                       prev_M=None, seed=0, frame=0, view=0, pixel_offset=0, light=None, W=None,
                       M=None, estimate=None, stream=None):
    """Temporal resampling of the frame's cache reservoir (cur_light, cur_W)
    with the previous frame's (prev_light, prev_W, prev_M; None: every pixel
    disoccluded) into (light, W, M) and the one-shadow-ray estimate."""
    _pixels(pos, nrm, ((cur_light, "cur_light"), (cur_W, "cur_W"), (prev_light, "prev_light"),
                       (prev_W, "prev_W"), (prev_M, "prev_M"), (light, "light"), (W, "W"),
                       (M, "M"), (estimate, "estimate")))
    check(lib.nvc_temporal_merge(scene.ref, _ptr(pos, name="pos"), _ptr(nrm, name="nrm"),
                                 pos.shape[0], int(pixel_offset), int(seed), int(frame), int(view),
                                 _ptr(cur_light, torch.int32, "cur_light"), _ptr(cur_W, name="cur_W"),
                                 _ptr(prev_light, torch.int32, "prev_light"),
                                 _ptr(prev_W, name="prev_W"), _ptr(prev_M, torch.int32, "prev_M"),
                                 _ptr(light, torch.int32, "light"), _ptr(W, name="W"),
                                 _ptr(M, torch.int32, "M"), _ptr(estimate, name="estimate"),
                                 _stream(stream)))


def nvc_infer_noalloc(cfg: NvcConfig, params, pos, vis, stream=None):
    """nvc_infer for callers that cannot allocate GPU memory: parameters come
    from the caller, the library's fixed scratch array holds the encoded
    features (at most 2^21 floats per call).

    The C entry point cannot see tensor sizes, so the shapes are checked
    here against the configuration before anything is launched: params must
    hold exactly nvc_param_count(cfg) floats, pos be [n, 3] and vis
    [n, n_outputs], all three on one CUDA device; the call is made with that
    device current, so the library uses that device's scratch array."""
    n_params = nvc_param_count(cfg)
    if n_params < 0:
        raise NVCError(_lib.NVC_ERR_INVALID_ARG, "invalid configuration")
    for t, name in ((params, "params"), (pos, "pos"), (vis, "vis")):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch.Tensor")
    if params.numel() != n_params:
        raise ValueError(f"params holds {params.numel()} floats, the configuration needs {n_params}")
    if pos.dim() != 2 or pos.shape[1] != 3:
        raise ValueError(f"pos must be [n, 3], got {tuple(pos.shape)}")
    if tuple(vis.shape) != (pos.shape[0], cfg.n_outputs):
        raise ValueError(f"vis must be [{pos.shape[0]}, {cfg.n_outputs}], got {tuple(vis.shape)}")
    if not (params.device == pos.device == vis.device):
        raise ValueError("params, pos and vis must be on one device")
    pp, px, pv = _ptr(params, name="params"), _ptr(pos, name="pos"), _ptr(vis, name="vis")
    with torch.cuda.device(params.device):
        check(lib.nvc_infer_noalloc(ctypes.byref(cfg), pp, px, pos.shape[0], pv, _stream(stream)))


def nvc_set_profiling(h, enable: bool):
    check(lib.nvc_set_profiling(h, 1 if enable else 0), h)


def nvc_stage_times(h):
    ms = (ctypes.c_double * 4)()
    n = ctypes.c_int64()
    check(lib.nvc_stage_times(h, ms, 4, ctypes.byref(n)), h)
    return list(ms), int(n.value)


# ------------------------------------------------------ convenience class --

class VisibilityCache:
    """Owns one nvc handle; methods allocate outputs with torch."""

    def __init__(self, cfg=None, **kw):
        self.cfg = make_config(cfg, **kw)
        self.n_params = nvc_param_count(self.cfg)
        if self.n_params < 0:
            raise NVCError(_lib.NVC_ERR_INVALID_ARG, "invalid configuration")
        self.handle = nvc_create(self.cfg)
        self.L = self.cfg.n_outputs
        self.din = self.cfg.n_levels * self.cfg.n_features
        # a half-precision feature copy serves the tensor-core inference only
        table_precision = kw.get("table_precision", getattr(cfg, "table_precision", "fp32"))
        if table_precision != "fp32" and self.cfg.precision != _lib.PRECISIONS["fp32"]:
            nvc_set_table_precision(self.handle, table_precision)

    def close(self):
        if self.handle is not None:
            nvc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params, m=None, v=None, step=0):
        p = torch.as_tensor(params, dtype=torch.float32).cuda().contiguous()
        if p.numel() != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {p.numel()}")
        mm = None if m is None else torch.as_tensor(m, dtype=torch.float32).cuda().contiguous()
        vv = None if v is None else torch.as_tensor(v, dtype=torch.float32).cuda().contiguous()
        nvc_set_state(self.handle, p, mm, vv, step)

    def state(self):
        p = torch.empty(self.n_params, device="cuda")
        m = torch.empty_like(p)
        v = torch.empty_like(p)
        nvc_get_state(self.handle, p, m, v)
        return p, m, v

    def encode(self, pos):
        feat = torch.empty((pos.shape[0], self.din), device="cuda")
        nvc_encode(self.handle, pos, feat)
        return feat

    def infer(self, pos):
        vis = torch.empty((pos.shape[0], self.L), device="cuda")
        nvc_infer(self.handle, pos, vis)
        return vis

    def shade(self, scene, pos, nrm, seed=0, frame=0, view=0, pixel_offset=0, fused=True):
        n = pos.shape[0]
        out = dict(idx=torch.empty(n, dtype=torch.int32, device="cuda"),
                   pdf=torch.empty(n, device="cuda"), wsum=torch.empty(n, device="cuda"),
                   radiance=torch.empty(n, device="cuda"))
        nvc_shade(self.handle, scene, pos, nrm, seed, frame, view, pixel_offset, fused=fused, **out)
        return out

    def train_step(self, scene, screen_pos, seed, frame):
        loss = torch.empty(1, dtype=torch.float64, device="cuda")
        nvc_train_step(self.handle, scene, screen_pos, seed, frame, loss)
        return loss

    def train_gradient(self, scene, screen_pos, seed, frame):
        g = torch.empty(self.n_params, device="cuda")
        loss = torch.empty(1, dtype=torch.float64, device="cuda")
        nvc_train_gradient(self.handle, scene, screen_pos, seed, frame, g, loss)
        return g, loss

    def counters(self):
        return nvc_sync_status(self.handle)
