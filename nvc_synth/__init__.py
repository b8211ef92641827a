"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This package holds no arithmetic of the visibility-cache method itself: it
only draws scenes (point lights, sphere/box occluders), G-buffers (shading
positions and normals) and initial parameter vectors from seeded numpy
generators, and names the hyper-parameter sets the workloads run.  Both the
CUDA library and the CPU oracle are fed the same float32 arrays from here.

Conventions (identical for every consumer):
  * lights   float32 [L, 4]  : x, y, z, intensity (scalar, monochrome)
  * spheres  float32 [S, 4]  : cx, cy, cz, radius
  * boxes    float32 [Bx, 6] : lo x, lo y, lo z, hi x, hi y, hi z
  * G-buffer float32 [P, 3] positions and [P, 3] unit normals, row-major
    pixels (row i, column j -> pixel i*W + j)
  * parameter vector float32, laid out as
        [hash table: levels x T x F (level-major, F contiguous per entry)]
        [W_1: width x n_in] [W_2: width x width] ... [W_out: L x width]
    every weight matrix row-major [out][in]; no biases (the MLP has none).
"""
from .configs import (NVCConfig, CONFIGS, config_by_name, param_layout,
                      param_count)
from .scenes import (Scene, GBuffer, scene_unit_cube, scene_heightfield,
                     scene_many_lights, scene_rooms, kmeans_init, gbuffer_points, gbuffer_heightfield, gbuffer_camera_path,
                     init_params, multiview_gbuffers)

__all__ = [
    "NVCConfig", "CONFIGS", "config_by_name", "param_layout", "param_count",
    "Scene", "GBuffer", "scene_unit_cube", "scene_heightfield",
    "scene_many_lights", "scene_rooms", "kmeans_init",
    "gbuffer_points", "gbuffer_heightfield", "gbuffer_camera_path",
    "init_params", "multiview_gbuffers",
]
