"""Pins of the oracle's float32 decisions against definitions outside it.

Where floating point decides an integer the oracle takes the decision in
float32, the precision the kernels use: the binary shadow-ray visibility
(Section 3.4) and the float32 light contributions that the integer
reservoir quantises (Section 3.1).  These tests pin those float32 forms to
the definitions themselves, independently of the oracle's own arithmetic:

* visibility against exact rational geometry (every input's float32 value
  converted exactly to a fraction, the segment and occluder tests of the
  definition evaluated without rounding) wherever the exact answer is not
  within a thin margin of a surface, over random heightfield and box
  scenes and the hard cases: directions with negative components, segments
  parallel to an axis, points on box faces, zero-length segments;
* visibility against dense marching along the segment (a different method
  again), in float64 and float32;
* float32 contributions against the float64 form within an error bound
  derived from the operations, at grazing angles and tiny distances too.
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import nvc_synth as S
from oracle import nvc as O

T0 = Fr(O.SEG_T0)
T1 = Fr(O.SEG_T1)


def _fr3(v):
    return [Fr(float(c)) for c in v]


def exact_visibility(x, l, spheres, boxes):
    """The shadow-ray definition in exact rational arithmetic.

    Segment x + t (l - x), t in [1e-4, 1 - 1e-4]; a sphere (c, r) blocks it
    when the segment's closest point to c is strictly closer than r; a box
    blocks it when the segment meets the closed box.  Returns (visible,
    margin): margin is the smallest relative distance of any test from its
    decision boundary, so that an answer whose margin exceeds the rounding
    error of a float32 evaluation is the answer float32 must give."""
    X, L = _fr3(x), _fr3(l)
    D = [L[a] - X[a] for a in range(3)]
    dd = sum(d * d for d in D)
    scale = max([abs(v) for v in X + L] + [Fr(1)])
    visible, margin = True, math.inf
    for s in spheres:
        C, r = _fr3(s[:3]), Fr(float(s[3]))
        if dd == 0:
            tc = T0
        else:
            tc = sum((C[a] - X[a]) * D[a] for a in range(3)) / dd
            tc = min(max(tc, T0), T1)
        E = [C[a] - X[a] - tc * D[a] for a in range(3)]
        d2 = sum(e * e for e in E)
        if d2 < r * r:
            visible = False
        # |dist - r| relative to the scene's coordinate scale
        gap = abs(math.sqrt(float(d2)) - float(r)) / float(scale)
        margin = min(margin, gap)
    for b in boxes:
        lo, hi = _fr3(b[:3]), _fr3(b[3:])
        tmin, tmax, miss = T0, T1, False
        for a in range(3):
            if D[a] == 0:
                if X[a] < lo[a] or X[a] > hi[a]:
                    miss = True
                margin = min(margin, float(min(abs(X[a] - lo[a]), abs(X[a] - hi[a])) / scale))
                continue
            ta, tb = (lo[a] - X[a]) / D[a], (hi[a] - X[a]) / D[a]
            tmin, tmax = max(tmin, min(ta, tb)), min(tmax, max(ta, tb))
        if not miss:
            if tmin <= tmax:
                visible = False
            margin = min(margin, float(abs(tmax - tmin) / max(Fr(1), abs(tmin), abs(tmax))))
    return visible, margin


def _hard_cases(rng, sc, n):
    """(position, light) pairs of the kinds a float32 slip would show in:
    negative direction components, axis-parallel segments, points on box
    faces (leaving and entering), zero-length segments."""
    pairs = []
    lights = sc.lights[:, :3].astype(np.float32)
    for k in range(n):
        kind = k % 6
        l = lights[rng.integers(len(lights))]
        if kind == 0:                               # light below and behind: every component negative
            x = (l + rng.uniform(0.5, 4.0, 3)).astype(np.float32)
        elif kind == 1:                             # parallel to z (x, y shared)
            x = np.array([l[0], l[1], rng.uniform(0, 10)], np.float32)
        elif kind == 2:                             # parallel to x (y, z shared)
            x = np.array([rng.uniform(0, 10), l[1], l[2]], np.float32)
        elif kind in (3, 4):                        # on a face of a box, light anywhere
            b = sc.boxes[rng.integers(len(sc.boxes))].astype(np.float32)
            a = rng.integers(3)
            x = rng.uniform(b[:3], b[3:]).astype(np.float32)
            x[a] = b[a] if kind == 3 else b[3 + a]
        else:                                       # zero-length segment: the light at the point
            x = l.copy() if rng.uniform() < 0.5 else rng.uniform(0, 10, 3).astype(np.float32)
            l = x.copy()
        pairs.append((x, l.astype(np.float32)))
    return pairs


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_visibility_matches_exact_rational_geometry(dtype):
    rng = np.random.default_rng(21)
    sc = S.scene_heightfield(seed=3, n_lights=6, n_spheres=12, n_boxes=12)
    pos = rng.uniform(0, 10, (40, 3)).astype(np.float32)
    pairs = [(p, l[:3].astype(np.float32)) for p in pos for l in sc.lights]
    pairs += _hard_cases(rng, sc, 300)
    kinds = np.zeros(6, int)
    checked = 0
    for k, (x, l) in enumerate(pairs):
        light = np.concatenate([l, [1.0]])[None]
        v = O.visibility(x[None], light, sc.spheres, sc.boxes, dtype)[0, 0]
        ve, margin = exact_visibility(x, l, sc.spheres, sc.boxes)
        if margin < 2e-5:
            continue
        checked += 1
        if k >= 240:
            kinds[(k - 240) % 6] += 1
        assert v == (1.0 if ve else 0.0), (x, l, ve, margin)
    assert checked >= 500
    assert np.all(kinds >= 30), kinds            # every hard-case kind is represented


def test_visibility_exact_on_box_faces_and_points():
    """The closed-box and t-range readings decide these exactly: a segment
    leaving a box face is not blocked by that box (it starts at t = 1e-4);
    one entering it is; a zero-length segment is blocked exactly when its
    point lies in an occluder (a closed box or strictly inside a sphere)."""
    box = np.array([[1.0, 1.0, 1.0, 2.0, 2.0, 2.0]])
    nos = np.zeros((0, 4))
    for dt in (np.float64, np.float32):
        V = lambda x, l, sph=nos, bx=box: O.visibility(np.array([x], float),
                                                        np.array([l + [1.0]]), sph, bx, dt)[0, 0]
        assert V([1.0, 1.5, 1.5], [0.0, 1.5, 1.5]) == 1.0     # leaves through the x = lo face
        assert V([1.0, 1.5, 1.5], [3.0, 1.5, 1.5]) == 0.0     # enters through it
        assert V([2.0, 1.2, 1.7], [5.0, -3.0, 9.0]) == 1.0    # leaves the x = hi face obliquely
        assert V([2.0, 1.2, 1.7], [0.5, 1.4, 1.6]) == 0.0     # crosses the box
        assert V([1.5, 1.5, 1.5], [1.5, 1.5, 1.5]) == 0.0     # point inside, zero length
        assert V([2.0, 2.0, 2.0], [2.0, 2.0, 2.0]) == 0.0     # on the closed corner
        assert V([2.5, 1.5, 1.5], [2.5, 1.5, 1.5]) == 1.0     # outside, zero length
        sph = np.array([[0.0, 0.0, 0.0, 1.0]])
        assert V([0.5, 0.0, 0.0], [0.5, 0.0, 0.0], sph, np.zeros((0, 6))) == 0.0
        assert V([1.0, 0.0, 0.0], [1.0, 0.0, 0.0], sph, np.zeros((0, 6))) == 1.0  # on the sphere: strict


def _march_clearance(x, l, spheres, boxes, ts):
    P = x + ts[:, None] * (l - x)
    clear = np.inf
    for s in spheres.astype(float):
        clear = min(clear, np.min(np.linalg.norm(P - s[:3], axis=1) - s[3]))
    for b in boxes.astype(float):
        lo, hi = b[:3], b[3:]
        out = np.maximum(np.maximum(lo - P, P - hi), 0)
        inside_depth = np.min(np.minimum(P - lo, hi - P), axis=1)
        sd = np.where(np.all((P >= lo) & (P <= hi), 1), -inside_depth,
                      np.linalg.norm(out, axis=1))
        clear = min(clear, np.min(sd))
    return clear


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_visibility_f32_and_f64_match_dense_marching(dtype):
    """Dense marching (20001 points per segment, signed distance to every
    occluder) on float32-representable inputs, random pairs plus the hard
    cases; pairs whose clearance is within 2e-3 of a surface are left to the
    exact test above.  The float32 and float64 decisions must both equal the
    marcher's, so they agree with each other everywhere outside the band."""
    rng = np.random.default_rng(8)
    sc = S.scene_heightfield(seed=3, n_lights=6, n_spheres=10, n_boxes=10)
    pos = rng.uniform(0, 10, (45, 3)).astype(np.float32)
    pairs = [(p, l[:3].astype(np.float32)) for p in pos for l in sc.lights]
    pairs += [(x, l) for x, l in _hard_cases(rng, sc, 120)]
    ts = np.linspace(O.SEG_T0, O.SEG_T1, 20001)
    checked = 0
    for x, l in pairs:
        light = np.concatenate([l, [1.0]])[None]
        v = O.visibility(x[None], light, sc.spheres, sc.boxes, dtype)[0, 0]
        clear = _march_clearance(x.astype(float), l.astype(float), sc.spheres, sc.boxes, ts)
        if abs(clear) < 2e-3:
            continue
        checked += 1
        assert v == (1.0 if clear > 0 else 0.0), (x, l, clear)
    assert checked > 300


# ------------------------------------------------------------ contributions --

U32 = 2.0 ** -24


def _contribution_cases(rng, n):
    pos = rng.uniform(-5, 5, (n, 3)).astype(np.float32)
    lights = np.empty((n, 4), np.float32)
    lights[:, 3] = rng.uniform(0.5, 100, n)
    kind = np.arange(n) % 4
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    dist = np.where(kind == 2, rng.uniform(1e-5, 2e-3, n), rng.uniform(0.01, 20, n))
    lights[:, :3] = (pos + d * dist[:, None]).astype(np.float32)
    nrm = rng.normal(size=(n, 3))
    # grazing: the normal nearly perpendicular to the direction, either side
    dd = (lights[:, :3].astype(float) - pos)
    dd /= np.linalg.norm(dd, axis=1, keepdims=True)
    perp = nrm - np.sum(nrm * dd, 1, keepdims=True) * dd
    perp /= np.linalg.norm(perp, axis=1, keepdims=True)
    eps = rng.choice([-1, 1], n) * 10.0 ** rng.uniform(-8, -2, n)
    graze = perp + eps[:, None] * dd
    nrm = np.where((kind == 1)[:, None], graze, nrm)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return pos, nrm.astype(np.float32), lights


def test_contributions_f32_within_derived_bound_of_f64():
    """float32 c_i against the float64 form on the same float32 inputs.

    Error bound, u = 2^-24, every step a correctly rounded float32
    operation (d = l - x, d.d and n.d summed x, y then z, sqrt, max,
    products, one division):
      * d_a carries relative error u; d.d, a sum of positive terms,
        <= 5u; sqrt(d.d) <= 3.5u; the denominator sqrt(d.d) max(d.d, 1e-6)
        <= 9.5u; I (1/pi), with 1/pi rounded, <= 2u; the numerator product
        and the division add u each: relative <= 13.5u overall;
      * n.d can cancel: its absolute error is <= 4u sum_a |n_a d_a|
        <= 4u |n| |d|, which reaches c as an absolute error of at most
        4u S (1 + 14u) with S = I / (pi max(|d|^2, 1e-6)) for a unit normal;
      * the n.d > 0 test can flip only where |n.d| is inside that error, so
        the flipped contribution is itself below 4u S.
    So |c32 - c64| <= 14u c64 + 5u S, checked on random, grazing and
    very close lights."""
    rng = np.random.default_rng(4)
    pos, nrm, lights = _contribution_cases(rng, 4000)
    c64 = np.array([O.contributions(pos[i:i + 1], nrm[i:i + 1], lights[i:i + 1])[0, 0]
                    for i in range(len(pos))])
    c32 = np.array([O.contributions(pos[i:i + 1], nrm[i:i + 1], lights[i:i + 1], np.float32)[0, 0]
                    for i in range(len(pos))], np.float64)
    d2 = np.sum((lights[:, :3].astype(float) - pos) ** 2, 1)
    Sc = lights[:, 3].astype(float) / (math.pi * np.maximum(d2, 1e-6))
    err = np.abs(c32 - c64)
    bound = 14 * U32 * c64 + 5 * U32 * Sc
    assert np.all(err <= bound), np.max(err / bound)
    # the cases are telling: grazing ones sit far below S, some change sign
    # across the float32 rounding, and close lights hit the 1e-6 clamp
    graze = (np.arange(len(pos)) % 4) == 1
    assert np.median(c64[graze] / Sc[graze]) < 1e-3
    assert np.any(d2 < 1e-6)
    # the bound is tight enough to catch plausible slips: n.d without its
    # z term, the direction reversed (x - l), or the 1/pi factor dropped
    d = lights[:, :3].astype(float) - pos
    I = lights[:, 3].astype(float)
    den = np.sqrt(d2) * np.maximum(d2, 1e-6)
    for ndl, k in ((nrm[:, 0] * d[:, 0] + nrm[:, 1] * d[:, 1], 1 / math.pi),
                   (-np.sum(nrm * d, 1), 1 / math.pi), (np.sum(nrm * d, 1), 1.0)):
        wrong = np.where(ndl > 0, I * k * ndl / den, 0.0)
        assert np.any(np.abs(wrong - c64) > bound)


def test_contributions_at_grazing_angles_stay_nonnegative_and_small():
    rng = np.random.default_rng(5)
    pos, nrm, lights = _contribution_cases(rng, 2000)
    c32 = O.contributions(pos, nrm, lights, np.float32)
    diag = np.einsum("ii->i", c32)
    assert np.all(diag >= 0) and np.all(np.isfinite(diag))


# ------------------------------------------------- the fp16 gradient model --

def _gradient_case(name, loss, batch):
    cfg = S.config_by_name(name).with_(train_precision="fp16", loss=loss, loss_scale=128.0,
                                       leaky_slope=0.01, batch_positions=batch)
    if name == "tiny_fp32":
        sc, gb = S.scene_unit_cube(seed=0), S.gbuffer_points(0, 64, 64)
    else:
        sc = S.scene_heightfield(seed=1, n_lights=32, n_spheres=32, n_boxes=32)
        gb = S.gbuffer_heightfield(seed=1, width=96, height=54)
    from helpers import scaled_params
    p = scaled_params(cfg, seed=2, table_scale=0.5)
    pos = O.training_positions(batch, sc.world_min, sc.world_max, gb.pos, 5, 3)
    y = O.visibility(pos, sc.lights, sc.spheres, sc.boxes, np.float32)
    return cfg, p, pos, y


def test_fp16_gradient_model_without_rounding_is_the_oracle_gradient():
    """The rounding model the FP16 training test measures the kernel
    against: with its fp16 roundings switched off it must reproduce the
    oracle's float64 gradient, so it carries no dropped term or transposed
    product of its own."""
    from helpers import fp16_gradient_model, rel_err
    for name, loss, batch in (("tiny_fp32", "bce", 256), ("tiny_fp32", "l2", 250),
                              ("frame_1080p", "bce", 128)):
        cfg, p, pos, y = _gradient_case(name, loss, batch)
        _, g_ref = O.gradients(cfg, p, pos, y)
        g = fp16_gradient_model(cfg, p, pos, y, 128.0, quantise=False)
        assert rel_err(g, g_ref) <= 1e-12, (name, loss)


def test_fp16_operand_rounding_alone_sets_the_training_gradient_error():
    """The FP16 training bound is a reading: rounding the operands to fp16
    (features, weights, activations, scaled deltas; everything else exact)
    moves the gradient of the 1080p network 3.2e-3 from the float64 oracle
    on the whole-vector norm and 2e-2 on the table's part -- above the 2e-3
    budget -- while the tiny network stays inside it (1.2e-3).  So FP16
    training is bounded on the tiny network by 2e-3 on the norm and on the
    1080p network by the rounding model's own distance."""
    from helpers import fp16_gradient_model, rel_err
    dist = {}
    for name, loss, batch in (("tiny_fp32", "bce", 1024), ("frame_1080p", "bce", 1024)):
        cfg, p, pos, y = _gradient_case(name, loss, batch)
        _, g_ref = O.gradients(cfg, p, pos, y)
        dist[name] = rel_err(fp16_gradient_model(cfg, p, pos, y, 128.0), g_ref)
    assert dist["tiny_fp32"] < 2e-3 < dist["frame_1080p"], dist


# ------------------------------------------------- FP16 hash-table features --

def test_fp16_table_features_are_the_rounded_table_used_exactly():
    """A cache with half-precision table features infers from every table
    entry rounded to the nearest float16 (ties to even), then exactly: the
    same result as the float32-feature oracle run on a table already holding
    those rounded values, and a different one from the unrounded table."""
    from helpers import scaled_params
    cfg = S.config_by_name("tiny_fp32").with_(precision="fp16", table_precision="fp16")
    p = scaled_params(cfg, seed=4, table_scale=0.3)
    tn = cfg.n_levels * cfg.table_size * cfg.n_features
    q = p.copy()
    q[:tn] = p[:tn].astype(np.float16).astype(np.float32)
    # float16 rounding of float32 values: ties go to the even neighbour
    assert np.float32(1 + 2 ** -11).astype(np.float16) == np.float16(1.0)
    assert np.float32(1 + 3 * 2 ** -11).astype(np.float16) == np.float16(1 + 2 ** -9)
    pos = np.random.default_rng(0).uniform(0, 1, (500, 3))
    v16 = O.infer(cfg, p, pos)
    assert np.array_equal(v16, O.infer(cfg.with_(table_precision="fp32"), q, pos))
    v32 = O.infer(cfg.with_(table_precision="fp32"), p, pos)
    assert 0 < np.max(np.abs(v16 - v32)) < 1e-2
    # float32 inference reads the float32 master whatever the copy's precision
    assert np.array_equal(O.infer(cfg.with_(precision="fp32"), p, pos), v32)
