"""The C ABI library builds, loads and exports every symbol include/nvc.h
declares; host-side argument checks answer without a GPU."""
import ctypes
import os
import re

import pytest

import nvc_synth as S
from oracle import nvc as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_05930_gb300.build import build
    build()
    from paper_2506_05930_gb300 import _lib
    return _lib.load()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(nvc_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("nvc_encode", "nvc_infer", "nvc_train_step", "nvc_wrs_sample",
                     "nvc_direct_illum", "nvc_create", "nvc_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2506_05930_gb300 import _lib
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.PROTOTYPES, f"binding lacks a prototype for {name}"


def _cfg(name="frame_1080p", **kw):
    import paper_2506_05930_gb300.nvc as nvc
    return nvc.make_config(S.config_by_name(name).with_(**kw))


def test_param_count_and_level_resolutions_match_the_layout(lib):
    import paper_2506_05930_gb300.nvc as nvc
    for name in ("tiny_fp32", "frame_1080p", "multiview", "precision_4k", "clustered_1080p",
                 "paper"):
        c = S.config_by_name(name)
        cc = nvc.make_config(c)
        assert nvc.nvc_param_count(cc) == S.param_count(c)
        assert [nvc.nvc_level_resolution(cc, l) for l in range(c.n_levels)] == \
            O.level_resolutions(c.base_resolution, c.growth, c.n_levels)
    assert nvc.nvc_level_resolution(_cfg(), 99) == -1


@pytest.mark.parametrize("field,value", [
    ("n_levels", 0), ("n_levels", 33), ("n_features", 3), ("log2_table_size", 30),
    ("hidden_width", 24), ("n_outputs", 257), ("leaky_slope", -0.5), ("loss_scale", 0.0),
    ("batch_positions", 0), ("growth", 0.5), ("precision", 9), ("beta1", 1.0)])
def test_invalid_configs_rejected_without_a_gpu(lib, field, value):
    import paper_2506_05930_gb300.nvc as nvc
    c = _cfg()
    setattr(c, field, value)
    assert nvc.nvc_param_count(c) == -1
    h = ctypes.c_void_p()
    assert lib.nvc_create(ctypes.byref(c), ctypes.byref(h)) == 1   # NVC_ERR_INVALID_ARG
    assert h.value is None
    assert len(nvc.nvc_last_error(None)) > 0


def test_null_arguments_rejected_without_a_gpu(lib):
    from paper_2506_05930_gb300 import _lib
    assert lib.nvc_encode(None, None, 10, None, None) == 1
    assert lib.nvc_wrs_from_weights(None, 10, 4, 0, 0, 0, 0, None, None, None, None) == 1
    assert lib.nvc_wrs_from_weights(None, 10, 0, 0, 0, 0, 0, None, None, None, None) == 1
    assert lib.nvc_trace_visibility(None, None, 1, None, None) == 1
    sc = _lib.NvcScene()
    assert lib.nvc_trace_visibility(ctypes.byref(sc), None, 1, None, None) == 1
    # zero-size work is a no-op that touches nothing
    assert lib.nvc_wrs_from_weights(None, 0, 4, 0, 0, 0, 0, None, None, None, None) == 0
    lib.nvc_destroy(None)


def test_host_kmeans_matches_the_oracle_bit_for_bit(lib):
    """nvc_kmeans_lights runs on the host: assignments and float64 centroids
    equal the oracle's Lloyd iterations exactly, on the many-lights scene."""
    import numpy as np
    import paper_2506_05930_gb300.nvc as nvc
    sc = S.scene_many_lights(seed=1, n_lights=1024)
    init = S.kmeans_init(1024, 32, seed=0)
    for iters in (0, 1, 10):
        a, c = nvc.nvc_kmeans_lights(sc.lights, init, iters)
        ra, rc = O.kmeans_lights(sc.lights, init, iters)
        assert np.array_equal(a, ra), iters
        assert np.array_equal(c, rc), iters
    assert len(np.unique(a)) > 24


def test_host_kmeans_rejects_bad_arguments(lib):
    import numpy as np
    import paper_2506_05930_gb300.nvc as nvc
    from paper_2506_05930_gb300 import _lib
    L = S.scene_many_lights(seed=2, n_lights=40).lights
    with pytest.raises(_lib.NVCError):
        nvc.nvc_kmeans_lights(L, np.array([0, 40], np.int32), 3)      # index out of range
    with pytest.raises(_lib.NVCError):
        nvc.nvc_kmeans_lights(L, np.arange(41, dtype=np.int32), 3)    # k > n_lights
    with pytest.raises(_lib.NVCError):
        nvc.nvc_kmeans_lights(L, np.arange(4, dtype=np.int32), -1)


def test_new_entry_points_reject_null_arguments_without_a_gpu(lib):
    """The clustered, placement, parameter and autotuning entry points answer
    argument errors on the host, before any CUDA call."""
    from paper_2506_05930_gb300 import _lib
    E = _lib.NVC_ERR_INVALID_ARG
    assert lib.nvc_set_training_placement(None, 0) == E
    assert lib.nvc_set_params(None, None, None) == E
    assert lib.nvc_autotune_infer(None, None, 10, None, 1, None, None, None) == E
    assert lib.nvc_training_positions_split(None, None, 0, 10, 5, 0, 0, None, None) == E
    assert lib.nvc_train_step_clustered(None, None, None, None, 0, 0, 0, None, None) == E
    assert lib.nvc_cluster_targets(None, None, None, 1, 0, 0, None, None) == E
    assert lib.nvc_sample_clustered(None, None, None, None, None, 1, 0, 0, 0, 0, None, None, None,
                                    None) == E
    # a scene with lights but no cluster table, and a table with a bad weight mode
    sc = _lib.NvcScene()
    sc.n_lights = 4
    sc.lights = 16                      # never dereferenced: the table check fails first
    assert lib.nvc_cluster_targets(ctypes.byref(sc), None, None, 1, 0, 0, None, None) == E
    cl = _lib.NvcClusters()
    cl.k, cl.offsets, cl.members, cl.weights = 4, 16, 16, 7
    assert lib.nvc_sample_clustered(ctypes.byref(sc), ctypes.byref(cl), None, None, None, 1, 0, 0,
                                    0, 0, None, None, None, None) == E
    cl.weights, cl.k = 0, 33
    assert lib.nvc_cluster_targets(ctypes.byref(sc), ctypes.byref(cl), None, 1, 0, 0, None,
                                   None) == E


def test_measurement_entry_points_reject_bad_arguments_without_a_gpu(lib):
    """The gather microbenchmark and the phase profile check their arguments
    on the host: nothing is launched for a bad row size, a table whose row
    count is not a power of two, a row count per thread that is not a
    multiple of 8, or a missing handle."""
    from paper_2506_05930_gb300 import _lib
    E = _lib.NVC_ERR_INVALID_ARG
    fake = 1 << 20            # an aligned address that is never dereferenced
    assert lib.nvc_gather_bench(fake, 1 << 20, 12, 100, 8, 0, fake, None) == E
    assert lib.nvc_gather_bench(fake, 3 << 20, 8, 100, 8, 0, fake, None) == E
    assert lib.nvc_gather_bench(fake, 1 << 20, 8, 100, 12, 0, fake, None) == E
    assert lib.nvc_gather_bench(fake, 1 << 20, 8, 0, 8, 0, fake, None) == E
    assert lib.nvc_gather_bench(fake + 4, 1 << 20, 8, 100, 8, 0, fake, None) == E
    assert lib.nvc_gather_bench(None, 1 << 20, 8, 100, 8, 0, fake, None) == E
    cyc = (ctypes.c_double * 4)()
    assert lib.nvc_shade_phases(None, None, None, None, 10, 0, 0, None, None, None, None, cyc,
                                None) == E
    assert lib.nvc_set_training_data_fused(None, 1) == E
    assert lib.nvc_training_batch(None, None, None, None) == E
    assert lib.nvc_set_table_precision(None, 1, None) == E
    assert lib.nvc_temporal_merge(None, None, None, 10, 0, 0, 0, 0, None, None, None, None, None,
                                  None, None, None, None, None) == E
    sc = _lib.NvcScene()
    sc.n_lights, sc.lights = 4, fake
    # a previous reservoir given in part
    assert lib.nvc_temporal_merge(ctypes.byref(sc), fake, fake, 10, 0, 0, 0, 0, fake, fake, fake,
                                  None, None, fake, None, None, None, None) == E


def test_noalloc_wrapper_checks_shapes_before_launching(lib):
    """nvc_infer_noalloc cannot see tensor sizes, so the binding checks them
    against the configuration first: a short parameter vector, a position
    array of the wrong width or an output of the wrong shape is refused with
    ValueError before any pointer reaches the library (CPU tensors here, so
    a launch could not even be attempted)."""
    import torch
    import paper_2506_05930_gb300.nvc as nvc
    cfg = S.config_by_name("tiny_fp32")
    c = nvc.make_config(cfg)
    n_params = nvc.nvc_param_count(c)
    good = dict(params=torch.zeros(n_params), pos=torch.zeros((8, 3)),
                vis=torch.zeros((8, cfg.n_outputs)))
    for key, bad in (("params", torch.zeros(n_params - 1)), ("pos", torch.zeros((8, 2))),
                     ("vis", torch.zeros((8, cfg.n_outputs + 1))), ("vis", torch.zeros((7, 4)))):
        args = dict(good, **{key: bad})
        with pytest.raises(ValueError):
            nvc.nvc_infer_noalloc(c, args["params"], args["pos"], args["vis"])
    # right shapes but host tensors: refused as not CUDA, still before the call
    with pytest.raises(ValueError):
        nvc.nvc_infer_noalloc(c, good["params"], good["pos"], good["vis"])


def test_shade_plan_entry_points_reject_bad_arguments_without_a_gpu(lib):
    from paper_2506_05930_gb300 import _lib
    E = _lib.NVC_ERR_INVALID_ARG
    plan = _lib.NvcShadePlan(0, 0)
    assert lib.nvc_set_shade_plan(None, ctypes.byref(plan)) == E
    assert lib.nvc_autotune_shade_plan(None, None, None, None, 10, None, None, None, None, 1, None,
                                       None, None, 0, None, None) == E
