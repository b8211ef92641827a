"""Pins of the CPU oracle to facts outside itself (closed forms, library
routines, brute force, hand-worked values, invariants).  CPU only."""
import math
import os
from decimal import Decimal, getcontext

import numpy as np
import pytest
import scipy.interpolate
import scipy.stats

from oracle import nvc as O
from oracle import philox as PH
import nvc_synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox --

def test_philox_round_structure_matches_numpy_philox4x64():
    """numpy's Philox bit generator (an independent implementation of
    Philox-4x64-10) pins the round function, word permutation and key
    schedule; numpy increments its counter before the first block."""
    rng = np.random.default_rng(5)
    cases = [([0, 0, 0, 0], [0, 0]),
             ([2**64 - 1, 0, 0, 0], [1, 2]),       # carry into word 1
             ([5, 7, 9, 11], [123, 456])]
    for _ in range(5):
        cases.append((list(map(int, rng.integers(0, 2**63, 4))),
                      list(map(int, rng.integers(0, 2**63, 2)))))
    for ctr, key in cases:
        bg = np.random.Philox(counter=np.array(ctr, dtype=np.uint64),
                             key=np.array(key, dtype=np.uint64))
        got = [int(v) for v in bg.random_raw(4)]
        c = ctr[0] + (ctr[1] << 64) + (ctr[2] << 128) + (ctr[3] << 192) + 1
        c1 = [(c >> (64 * i)) & (2**64 - 1) for i in range(4)]
        want = PH.philox_generic(c1, key, width=64, mult=PH.M4x64, weyl=PH.W64)
        assert got == list(want)


def test_philox_weyl_constants_closed_form():
    """Key increments = fractional parts of the golden ratio and sqrt(3)."""
    getcontext().prec = 80
    phi_frac = (Decimal(5).sqrt() - 1) / 2
    s3_frac = Decimal(3).sqrt() - 1
    for bits, W in ((32, PH.W32), (64, PH.W64)):
        assert W[0] == int(phi_frac * (2**bits))
        assert W[1] == int(s3_frac * (2**bits))


def test_philox4x32_vectorised_matches_generic():
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2**32, (64, 4), dtype=np.uint64).astype(np.uint32)
    key = (0xDEADBEEF, 0x01234567)
    vec = PH.philox4x32(ctr, key)
    for i in range(64):
        assert tuple(int(v) for v in vec[i]) == PH.philox_generic(ctr[i], key)


def test_philox_uniformity_chi2():
    r = PH.stream_words(np.arange(1 << 16), 3, 1, PH.TAG_WRS, 16, seed=42)
    u = PH.uniform24(r).ravel()
    assert u.min() >= 0.0 and u.max() < 1.0
    hist = np.bincount((u * 256).astype(np.int64), minlength=256)
    assert scipy.stats.chisquare(hist).pvalue > 1e-4
    # consecutive words of one stream are uncorrelated
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 0.01


def test_uniform24_exact():
    r = np.array([0, 0xFF, 0x100, 0xFFFFFFFF], np.uint32)
    assert list(PH.uniform24(r)) == [0.0, 0.0, 2.0**-24, 1.0 - 2.0**-24]


# ------------------------------------------------------------------- hash --

def test_hash_hand_worked_vectors():
    rows = np.loadtxt(os.path.join(GOLDEN, "hash_vectors.txt"), dtype=np.int64)
    for x, y, z, _, _, h, h14, h19 in rows:
        assert O.hash_index(x, y, z, 1 << 14) == h14
        assert O.hash_index(x, y, z, 1 << 19) == h19
        assert O.hash_index(x, y, z, 1 << 32) == h


def test_hash_axis_properties():
    x = np.arange(1000)
    # the x axis carries prime 1: identity below T
    assert np.array_equal(O.hash_index(x, 0, 0, 1 << 14), x)
    # XOR-separable over the axes
    y, z = x * 7 + 3, x * 13 + 5
    T = 1 << 19
    assert np.array_equal(O.hash_index(x, y, z, T),
                          O.hash_index(x, 0, 0, T) ^ O.hash_index(0, y, 0, T)
                          ^ O.hash_index(0, 0, z, T))


# ----------------------------------------------------------------- encode --

def _cfg(**kw):
    base = dict(name="t", n_levels=4, n_features=2, log2_table_size=14,
                base_resolution=4, growth=2.0, hidden=(8,), n_outputs=3)
    base.update(kw)
    return S.NVCConfig(**base)


def test_level_resolutions():
    assert O.level_resolutions(4, 2.0, 4) == [4, 8, 16, 32]
    assert O.level_resolutions(4, 1.5, 8) == [4, 6, 9, 13, 20, 30, 45, 68]
    assert O.level_resolutions(16, 1.447, 3) == [16, 23, 33]


def test_encode_grid_vertices_return_stored_entries():
    """At power-of-two resolutions vertex k / N_l is exact in float32 and
    the encoding returns the stored row bit-for-bit."""
    cfg = _cfg()
    rng = np.random.default_rng(0)
    table = rng.standard_normal((4, 1 << 14, 2))
    for l, n_l in enumerate([4, 8, 16, 32]):
        k = rng.integers(0, n_l + 1, (200, 3))
        k[0] = (n_l, n_l, n_l)          # the far corner (x_hat = 1)
        k[1] = (0, 0, 0)
        pos = (k / n_l).astype(np.float32)
        feat = O.encode(cfg, table, pos)
        rows = O.hash_index(k[:, 0], k[:, 1], k[:, 2], 1 << 14)
        assert np.array_equal(feat[:, 2 * l:2 * l + 2], table[l, rows])


def _collision_free_level(n_l, T):
    v = np.stack(np.meshgrid(*[np.arange(n_l + 1)] * 3, indexing="ij"), -1).reshape(-1, 3)
    rows = O.hash_index(v[:, 0], v[:, 1], v[:, 2], T)
    return v, rows, len(np.unique(rows)) == len(rows)


def test_encode_reproduces_affine_functions():
    """Trilinear interpolation is exact on affine functions of position: a
    wrong corner weight (f vs 1-f) or offset breaks this."""
    cfg = _cfg(n_levels=1, base_resolution=5, growth=1.0)
    T = 1 << 14
    v, rows, ok = _collision_free_level(5, T)
    assert ok
    a, b = np.array([0.3, -1.7, 2.9]), 0.25
    table = np.zeros((1, T, 2))
    table[0, rows, 0] = (v / 5.0) @ a + b
    table[0, rows, 1] = 1.0
    # dyadic positions: x_hat * N_l is exact in float32, so the blend is
    # evaluated at the query itself
    pos = (np.random.default_rng(1).integers(0, 1025, (500, 3)) / 1024.0).astype(np.float32)
    feat = O.encode(cfg, table, pos)
    np.testing.assert_allclose(feat[:, 0], pos.astype(np.float64) @ a + b, atol=1e-12)
    np.testing.assert_allclose(feat[:, 1], 1.0, atol=1e-14)   # partition of unity


def test_encode_matches_scipy_trilinear_interpolator():
    cfg = _cfg(n_levels=1, base_resolution=7, growth=1.0, n_features=1)
    T = 1 << 14
    v, rows, ok = _collision_free_level(7, T)
    assert ok
    vals = np.random.default_rng(2).standard_normal(len(v))
    table = np.zeros((1, T, 1))
    table[0, rows, 0] = vals
    grid = np.zeros((8, 8, 8))
    grid[v[:, 0], v[:, 1], v[:, 2]] = vals
    ax = np.arange(8) / 7.0
    interp = scipy.interpolate.RegularGridInterpolator((ax, ax, ax), grid)
    pos = (np.random.default_rng(3).integers(0, 4097, (400, 3)) / 4096.0).astype(np.float32)
    np.testing.assert_allclose(O.encode(cfg, table, pos)[:, 0],
                               interp(pos.astype(np.float64)), atol=1e-12)


def test_encode_clamps_outside_bounds_and_normalises():
    cfg = _cfg(bounds_min=(-2.0, 0.0, 1.0), bounds_max=(2.0, 4.0, 3.0))
    table = np.random.default_rng(4).standard_normal((4, 1 << 14, 2))
    inside = np.array([[-2.0, 0.0, 1.0], [2.0, 4.0, 3.0], [0.0, 2.0, 2.0]], np.float32)
    outside = np.array([[-9.0, -1.0, 0.0], [5.0, 8.0, 9.0], [0.0, 2.0, 2.0]], np.float32)
    np.testing.assert_array_equal(O.encode(cfg, table, inside), O.encode(cfg, table, outside))
    unit = _cfg()
    np.testing.assert_array_equal(
        O.encode(cfg, table, inside),
        O.encode(unit, table, np.array([[0, 0, 0], [1, 1, 1], [.5, .5, .5]], np.float32)))


def test_encode_backward_is_the_adjoint():
    """<encode(table), g> == <table, encode_backward(g)> (linear in table)."""
    cfg = _cfg(log2_table_size=8)          # small T: many collisions
    rng = np.random.default_rng(5)
    table = rng.standard_normal((4, 256, 2))
    pos = rng.uniform(0, 1, (300, 3)).astype(np.float32)
    feat, aux = O.encode(cfg, table, pos, with_aux=True)
    g = rng.standard_normal(feat.shape)
    lhs = np.sum(feat * g)
    rhs = np.sum(table * O.encode_backward(cfg, aux, g))
    assert abs(lhs - rhs) < 1e-9 * max(1.0, abs(lhs))


# -------------------------------------------------------------------- MLP --

def test_mlp_hand_computed():
    # 2 -> 2 -> 1, slope 0.25: x = (1, 1); z = (-1, 1.5); h = (-0.25, 1.5)
    W1 = np.array([[1.0, -2.0], [0.5, 1.0]])
    Wo = np.array([[1.0, -1.0]])
    out, acts, zs = O.mlp_forward([W1, Wo], np.array([[1.0, 1.0]]), 0.25)
    assert out[0, 0] == -1.75
    assert list(acts[1][0]) == [-0.25, 1.5]
    # 3 -> 2 -> 2 -> 2 ReLU: x = (2, 0, -1)
    A = np.array([[1.0, 0.5, 2.0], [-1.0, 1.0, 0.0]])   # z = (0, -2) -> (0, 0)
    B = np.array([[1.0, 1.0], [2.0, -1.0]])
    C = np.array([[3.0, 0.0], [0.0, 1.0]])
    out, _, _ = O.mlp_forward([A, B, C], np.array([[2.0, 0.0, -1.0]]), 0.0)
    assert list(out[0]) == [0.0, 0.0]
    out, _, _ = O.mlp_forward([A, B, C], np.array([[2.0, 4.0, 0.0]]), 0.0)
    # z1 = (4, 2); z2 = (6, 6); out = (18, 6)
    assert list(out[0]) == [18.0, 6.0]
    assert O.sigmoid(0.0) == 0.5
    np.testing.assert_allclose(O.sigmoid(np.log(3.0)), 0.75)


# ------------------------------------------------------- loss / backward --

@pytest.mark.parametrize("loss,slope", [("bce", 0.01), ("l2", 0.0), ("bce", 0.0)])
def test_gradients_match_central_finite_differences(loss, slope):
    """Analytic gradient vs central differences (h = 1e-3, float64) on 128
    parameters with nonzero gradient, relative error <= 1e-6."""
    cfg = _cfg(n_levels=3, log2_table_size=10, hidden=(16, 16), n_outputs=4,
               leaky_slope=slope, loss=loss, table_init=4.0, growth=1.5)
    p = S.init_params(cfg, seed=3).astype(np.float64)
    rng = np.random.default_rng(6)
    pos = rng.uniform(0, 1, (256, 3)).astype(np.float32)
    y = (rng.uniform(0, 1, (256, 4)) < 0.5).astype(np.float64)
    table, Ws = O.split_params(cfg, p)
    _, _, zs = O.mlp_forward(Ws, O.encode(cfg, table, pos), slope)
    # keep the samples away from the activation kinks, which a 1e-3 step
    # could cross
    keep = np.all([np.min(np.abs(z), axis=1) > 1e-2 for z in zs], axis=0)
    pos, y = pos[keep], y[keep]
    assert len(pos) >= 8
    _, g = O.gradients(cfg, p, pos, y)
    cand = np.flatnonzero(np.abs(g) > 1e-4 * np.abs(g).max())
    pick = rng.choice(cand, 128, replace=False)
    h = 1e-3
    worst = 0.0
    for i in pick:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (O.gradients(cfg, pp, pos, y)[0] - O.gradients(cfg, pm, pos, y)[0]) / (2 * h)
        worst = max(worst, abs(fd - g[i]) / max(abs(fd), abs(g[i])))
    assert worst <= 1e-6, worst


def test_bce_and_l2_closed_forms():
    z = np.array([[-3.0, 0.0, 2.0]])
    y = np.array([[1.0, 0.0, 1.0]])
    s = 1 / (1 + np.exp(-z))
    lb, gb = O.loss_and_grad("bce", z, y)
    np.testing.assert_allclose(lb, np.mean(-y * np.log(s) - (1 - y) * np.log(1 - s)))
    np.testing.assert_allclose(gb, (s - y) / 3)
    l2, g2 = O.loss_and_grad("l2", z, y)
    np.testing.assert_allclose(l2, np.mean((s - y) ** 2))
    # large logits: BCE stays finite
    lb, _ = O.loss_and_grad("bce", np.array([[800.0, -800.0]]), np.array([[0.0, 1.0]]))
    np.testing.assert_allclose(lb, 800.0)


# ------------------------------------------------------------------- Adam --

def test_adam_first_step_closed_form():
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    th = np.array([1.0, 1.0, 1.0, 1.0])
    t1, m, v = O.adam_update(th, g, np.zeros(4), np.zeros(4), 1, 0.01, 0.9, 0.99, 1e-15)
    # m_hat = g, v_hat = g^2: step = -lr * g / (|g| + eps)
    np.testing.assert_allclose(t1, th - 0.01 * g / (np.abs(g) + 1e-15), rtol=0, atol=1e-15)
    # a constant gradient keeps m_hat = g, v_hat = g^2 on step 2 as well
    t2, _, _ = O.adam_update(t1, g, m, v, 2, 0.01, 0.9, 0.99, 1e-15)
    np.testing.assert_allclose(t2, t1 - 0.01 * np.sign(g), atol=1e-12)


def test_adam_matches_torch_optim():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    th0 = rng.standard_normal(50)
    grads = [rng.standard_normal(50) * 10 ** rng.uniform(-3, 1) for _ in range(6)]
    p = torch.tensor(th0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=0.02, betas=(0.9, 0.99), eps=1e-15)
    th, m, v = th0.copy(), np.zeros(50), np.zeros(50)
    for t, g in enumerate(grads, 1):
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        th, m, v = O.adam_update(th, g, m, v, t, 0.02, 0.9, 0.99, 1e-15)
    np.testing.assert_allclose(th, p.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_learning_rate_schedules():
    paper = S.config_by_name("paper")
    assert O.learning_rate(paper, 1) == 0.05
    assert abs(O.learning_rate(paper, 101) - 0.0255) < 1e-15
    assert abs(O.learning_rate(paper, 201) - 0.001) < 1e-15
    assert abs(O.learning_rate(paper, 5000) - 0.001) < 1e-15
    assert O.learning_rate(S.config_by_name("tiny_fp32"), 77) == 0.01


# ------------------------------------------------------------- visibility --

LIGHT = np.array([[0.0, 0.0, 10.0, 1.0]])
ORIGIN = np.array([[0.0, 0.0, 0.0]])
NOBOX = np.zeros((0, 6))
NOSPH = np.zeros((0, 4))


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_visibility_sphere_special_cases(dt):
    V = lambda pos, sph: O.visibility(pos, LIGHT, np.array(sph, float).reshape(-1, 4), NOBOX, dt)[0, 0]
    assert V(ORIGIN, []) == 1.0
    assert V(ORIGIN, [0, 0, 5, 1]) == 0.0                 # on the axis
    assert V(ORIGIN, [1.5, 0, 5, 1]) == 1.0               # beside it
    assert V(ORIGIN, [0, 0, 12, 1]) == 1.0                # beyond the light
    assert V(ORIGIN, [0, 0, -3, 1]) == 1.0                # behind the point
    assert V(ORIGIN, [0.2, 0, 0.1, 0.5]) == 0.0           # point inside
    assert V(ORIGIN, [0, 0.1, 10, 0.5]) == 0.0            # light inside
    if dt == np.float64:
        assert V(ORIGIN, [1 + 1e-6, 0, 5, 1]) == 1.0      # just tangent
        assert V(ORIGIN, [1 - 1e-6, 0, 5, 1]) == 0.0      # just inside


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_visibility_box_special_cases(dt):
    V = lambda pos, box: O.visibility(np.array(pos, float).reshape(1, 3), LIGHT, NOSPH,
                                      np.array(box, float).reshape(-1, 6), dt)[0, 0]
    assert V([0, 0, 0], [-1, -1, 4, 1, 1, 6]) == 0.0      # axis-aligned through
    assert V([0, 0, 0], [0.5, -1, 4, 2, 1, 6]) == 1.0     # parallel, outside in x
    assert V([0, 0, 0], [0.0, -1, 4, 2, 1, 6]) == 0.0     # touching face: closed
    assert V([0, 0, 0], [-1, -1, -1, 1, 1, 1]) == 0.0     # point inside
    assert V([0, 0, 0], [-1, -1, 11, 1, 1, 12]) == 1.0    # beyond the light
    assert V([3, 0, 0], [1, -1, 4, 2, 1, 6]) == 0.0       # oblique ray through
    assert V([3, 0, 0], [-1, -1, 4, 1, 1, 6]) == 1.0      # oblique ray passes by
    assert V([3, 0, 0], [2.5, 0.5, 1, 3, 1, 2]) == 1.0    # oblique ray misses


def test_visibility_matches_dense_segment_sampling():
    """Brute force: march 20001 points along each segment and test each
    against every occluder; configurations whose minimum clearance is
    within 2e-3 of a surface are skipped as ambiguous for the marcher."""
    rng = np.random.default_rng(8)
    sc = S.scene_heightfield(seed=3, n_lights=6, n_spheres=10, n_boxes=10)
    pos = rng.uniform(0, 10, (60, 3))
    V = O.visibility(pos, sc.lights, sc.spheres, sc.boxes, np.float64)
    ts = np.linspace(O.SEG_T0, O.SEG_T1, 20001)
    checked = 0
    for a in range(len(pos)):
        for i in range(len(sc.lights)):
            P = pos[a] + ts[:, None] * (sc.lights[i, :3].astype(float) - pos[a])
            clear = np.inf
            for s in sc.spheres.astype(float):
                clear = min(clear, np.min(np.linalg.norm(P - s[:3], axis=1) - s[3]))
            for b in sc.boxes.astype(float):
                lo, hi = b[:3], b[3:]
                out = np.maximum(np.maximum(lo - P, P - hi), 0)
                inside_depth = np.min(np.minimum(P - lo, hi - P), axis=1)
                sd = np.where(np.all((P >= lo) & (P <= hi), 1), -inside_depth,
                              np.linalg.norm(out, axis=1))
                clear = min(clear, np.min(sd))
            if abs(clear) < 2e-3:
                continue
            checked += 1
            assert V[a, i] == (1.0 if clear > 0 else 0.0)
    assert checked > 300


# -------------------------------------------------- contributions and WRS --

def test_contribution_closed_forms():
    L = np.array([[0.0, 0.0, 2.0, 8.0], [2.0, 0.0, 2 * math.sqrt(3.0), 4.0],
                  [0.0, 0.0, -1.0, 5.0]])
    c = O.contributions(np.zeros((1, 3)), np.array([[0.0, 0.0, 1.0]]), L)[0]
    np.testing.assert_allclose(c, [8 / (math.pi * 4), 4 * math.cos(math.pi / 6) / (math.pi * 16), 0.0])
    c32 = O.contributions(np.zeros((1, 3)), np.array([[0.0, 0.0, 1.0]]), L, np.float32)[0]
    np.testing.assert_allclose(c32, c, rtol=1e-6)
    # light on the point: zero-length direction gives 0 (no NaN)
    c0 = O.contributions(np.zeros((1, 3)), np.array([[0.0, 0.0, 1.0]]),
                         np.array([[0.0, 0.0, 0.0, 1.0]]), np.float32)
    assert c0[0, 0] == 0.0


def test_fp32_constants():
    assert O.INV_PI_F32 == np.float32(1 / math.pi)
    assert O.VIS_CLAMP_F32.view(np.uint32) == 0x3A83126F


def test_quantize_weights_range_and_ratio():
    rng = np.random.default_rng(9)
    w = (rng.uniform(0, 1, (1000, 32)) * 10.0 ** rng.uniform(-30, 30, (1000, 1))).astype(np.float32)
    w[:, 5] = 0
    q = O.quantize_weights(w)
    assert np.all(q[:, 5] == 0)
    assert np.all((q.max(1) >= 2**23) & (q.max(1) < 2**24))
    pos = w > 0
    assert np.all(q[pos] >= 1)
    law = O.selection_law(w)
    ref = w / w.astype(np.float64).sum(1, keepdims=True)
    big = ref > 1e-4
    np.testing.assert_allclose(law[big], ref[big], rtol=2e-3)
    np.testing.assert_allclose(law[ref > 1e-2], ref[ref > 1e-2], rtol=1e-5)


@pytest.mark.parametrize("weights", [
    [1.0, 2.0, 3.0, 4.0],
    [0.0, 5.0, 0.0, 1e-3, 2.0, 0.0, 7.0, 0.5],
    [1e-30, 3e-30, 2e-30, 0.0],
])
def test_wrs_frequencies_chi2(weights):
    """Selection frequencies of the streaming reservoir match w_i / sum w."""
    w = np.tile(np.array(weights, np.float32), (200_000, 1))
    idx, pdf, wsum = O.wrs_select(w, np.arange(len(w)), seed=11, frame=0, view=0)
    w64 = np.array(weights, np.float32).astype(np.float64)
    p = w64 / w64.sum()
    counts = np.bincount(idx, minlength=len(weights))
    assert np.all(counts[p == 0] == 0)
    nz = p > 0
    stat = scipy.stats.chisquare(counts[nz], p[nz] * len(w))
    assert stat.pvalue > 1e-4
    np.testing.assert_allclose(pdf, p[idx], rtol=1e-12)


def test_wrs_degenerate_rows():
    w = np.array([[0, 0, 0], [0, 2, 0], [1, 0, 0]], np.float32)
    idx, pdf, wsum = O.wrs_select(w, np.arange(3), seed=0, frame=0, view=0)
    assert list(idx) == [-1, 1, 0]
    assert list(pdf) == [0.0, 1.0, 1.0]
    assert list(wsum) == [0.0, 2.0, 1.0]


def test_estimator_unbiased_with_clamp_and_biased_without():
    """E[V c / p] = exact DI when every light with c > 0 has p > 0: the
    sample mean over many frames is within 4 sigma of sum V c."""
    sc = S.scene_unit_cube(seed=0)
    gb = S.gbuffer_points(1, 8, 8)
    V = O.visibility(gb.pos, sc.lights, sc.spheres, sc.boxes)
    c32 = O.contributions(gb.pos, gb.nrm, sc.lights, np.float32)
    vis_pred = np.where(V > 0, 0.9, 0.0).astype(np.float32)   # a confident cache
    vis_pred[:, 0] = 0.0                                       # ... wrong on light 0
    w = O.light_weights_f32(vis_pred, c32)
    p = O.selection_law(w)
    E, var = O.estimator_moments(V, c32, p)
    np.testing.assert_allclose(E, O.exact_di(V, c32), rtol=1e-12)
    frames = 4000
    acc = np.zeros(len(gb.pos))
    ids = np.arange(len(gb.pos))
    for f in range(frames):
        idx, pdf, _ = O.wrs_select(w, ids, seed=3, frame=f, view=0)
        ok = idx >= 0
        j = np.maximum(idx, 0)
        acc += np.where(ok, V[ids, j] * c32[ids, j] / np.where(ok, p[ids, j], 1), 0)
    mean = acc / frames
    sigma = np.sqrt(np.maximum(var, 0) / frames)
    assert np.all(np.abs(mean - E) <= 4 * sigma + 1e-9)
    # without the clamp, light 0 can never be picked: biased low
    p_noclamp = O.selection_law(vis_pred * c32)
    E_nc, _ = O.estimator_moments(V, c32, p_noclamp)
    lost = V[:, 0] * c32[:, 0]
    np.testing.assert_allclose(E - E_nc, lost, atol=1e-9)
    assert lost.sum() > 0


# ------------------------------------------------------- training samples --

def test_training_positions_split_and_ranges():
    sc = S.scene_heightfield(seed=1, n_lights=4, n_spheres=2, n_boxes=2)
    gb = S.gbuffer_points(2, 16, 16, lo=(1, 2, 3), hi=(2, 3, 4))
    pos = O.training_positions(64, sc.world_min, sc.world_max, gb.pos, 5, 9)
    assert pos.dtype == np.float32 and pos.shape == (64, 3)
    assert np.all((pos[:32] >= 0) & (pos[:32] < 10))
    rows = {tuple(r) for r in gb.pos}
    assert all(tuple(r) in rows for r in pos[32:])
    assert not np.array_equal(pos, O.training_positions(64, sc.world_min, sc.world_max, gb.pos, 5, 10))
    allw = O.training_positions(64, sc.world_min, sc.world_max, None, 5, 9)
    np.testing.assert_array_equal(allw[:32], pos[:32])


def test_training_positions_placement_options():
    """The placements of Section 3.4: world space only, screen space only,
    and any split.  World rows are a prefix of one stream (row j of every
    split is the same point), screen rows index their own stream from 0
    (row n_world + s of every split is the same G-buffer point), so a split
    that reused the world index for the screen stream, or the other way
    round, would fail; the default is ceil(batch / 2) world rows."""
    sc = S.scene_heightfield(seed=1, n_lights=4, n_spheres=2, n_boxes=2)
    gb = S.gbuffer_points(2, 16, 16, lo=(1, 2, 3), hi=(2, 3, 4))
    rows = {tuple(r) for r in gb.pos}
    B = 65
    args = (sc.world_min, sc.world_max, gb.pos, 5, 9)
    world = O.training_positions(B, *args, n_world=B)
    screen = O.training_positions(B, *args, n_world=0)
    assert np.all((world >= 0) & (world < 10)) and not any(tuple(r) in rows for r in world)
    assert all(tuple(r) in rows for r in screen)
    np.testing.assert_array_equal(world, O.training_positions(B, sc.world_min, sc.world_max,
                                                              None, 5, 9))
    for nw in (1, 17, 33, 64):
        split = O.training_positions(B, *args, n_world=nw)
        np.testing.assert_array_equal(split[:nw], world[:nw])
        np.testing.assert_array_equal(split[nw:], screen[:B - nw])
    np.testing.assert_array_equal(O.training_positions(B, *args),
                                  O.training_positions(B, *args, n_world=33))


# ------------------------------------------------------------ learned part --

def test_oracle_training_converges_to_brute_force_visibility_and_gains():
    """Online training on the tiny scene: the cache's prediction approaches
    brute-force ray-cast visibility, and sampling with it lowers the
    estimator variance below sampling without a cache (v = 1)."""
    cfg = S.config_by_name("tiny_fp32").with_(loss="bce", leaky_slope=0.01, batch_positions=512)
    sc = S.scene_unit_cube(seed=0)
    st = O.TrainState.fresh(S.init_params(cfg, seed=0))
    test_pts = S.gbuffer_points(77, 32, 32)
    Vt = O.visibility(test_pts.pos, sc.lights, sc.spheres, sc.boxes, np.float32)
    mae0 = np.mean(np.abs(O.infer(cfg, st.params, test_pts.pos) - Vt))
    maes = []
    for f in range(300):
        view = S.gbuffer_points(1000 + f, 16, 16)
        O.train_step(cfg, st, sc, view.pos, seed=1, frame=f)
        if f % 50 == 49:
            maes.append(np.mean(np.abs(O.infer(cfg, st.params, test_pts.pos) - Vt)))
    assert st.step == 300 and st.skipped == 0
    assert maes[-1] < 0.5 * mae0 and maes[-1] < 0.12, (mae0, maes)
    c = O.contributions(test_pts.pos, test_pts.nrm, sc.lights, np.float32)
    vis = O.infer(cfg, st.params, test_pts.pos).astype(np.float32)
    _, var_cache = O.estimator_moments(Vt, c, O.selection_law(O.light_weights_f32(vis, c)))
    _, var_none = O.estimator_moments(Vt, c, O.selection_law(O.light_weights_f32(np.ones_like(vis), c)))
    assert var_cache.mean() < 0.8 * var_none.mean()


# -------------------------------------------------------------------- fp8 --

def test_e4m3_rounding_matches_torch_float8():
    """The oracle's E4M3 rounding against torch's float8_e4m3fn conversion
    (a library implementation of the same OCP format)."""
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8")
    from oracle import fp8
    rng = np.random.default_rng(12)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.uniform(-4, 3, 20000),
                        [0.0, 448.0, -448.0, 2.0 ** -9, 2.0 ** -10, 1.0625, 1.1875, 240.0, 232.0]])
    x = x[np.abs(x) <= 448.0].astype(np.float32)
    want = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(fp8.round_e4m3(x), want)
    # saturation above the largest finite value
    assert fp8.round_e4m3(np.array([1e4, -600.0])).tolist() == [448.0, -448.0]


# ------------------------------------------------ shading pass, exact DI --

def test_shading_estimate_is_unbiased_over_the_selection_law():
    """Averaged over the sampler's choice, V_s c_s / p_s is sum_i V_i c_i
    (Eq. 1; Section 3.1's estimator): sum_i p_i e(i, p_i) must equal the
    exact DI, which pins both the visibility factor and the division."""
    sc = S.scene_unit_cube(seed=2)
    gb = S.gbuffer_points(3, 16, 16)
    V = O.visibility(gb.pos, sc.lights, sc.spheres, sc.boxes, np.float32)
    c32 = O.contributions(gb.pos, gb.nrm, sc.lights, np.float32)
    w = O.light_weights_f32(np.full(c32.shape, 0.5, np.float32), c32)
    law = O.selection_law(w)                                  # [n, L], sums to 1 or 0
    mean = np.zeros(gb.n)
    for i in range(c32.shape[1]):
        pdf = law[:, i].astype(np.float32)
        e = O.shading_estimate(gb.pos, gb.nrm, sc.lights, sc.spheres, sc.boxes,
                               np.full(gb.n, i), pdf)
        mean += law[:, i] * e.astype(np.float64)
    exact = O.exact_di(V, O.contributions(gb.pos, gb.nrm, sc.lights))
    assert (exact > 0).mean() > 0.3
    assert ((V == 0) & (c32 > 0)).any()     # a dropped visibility factor would show
    np.testing.assert_allclose(mean, exact, rtol=2e-6, atol=1e-12)


def test_shading_estimate_special_cases():
    """No pick or no probability gives 0; a light behind a sphere gives 0;
    an unblocked light gives c / p in float32."""
    pos = np.array([[0.0, 0.0, 0.0]] * 4, np.float32)
    nrm = np.array([[0.0, 0.0, 1.0]] * 4, np.float32)
    lights = np.array([[0.0, 0.0, 2.0, 3.0],          # above, behind the sphere
                       [1.5, 0.0, 1.0, 2.0]], np.float32)   # off to the side, clear
    spheres = np.array([[0.0, 0.0, 1.0, 0.2]], np.float32)
    boxes = np.zeros((0, 6), np.float32)
    idx = np.array([0, 1, -1, 1])
    pdf = np.array([0.5, 0.25, 0.5, 0.0], np.float32)
    e = O.shading_estimate(pos, nrm, lights, spheres, boxes, idx, pdf)
    c = O.contributions(pos[:1], nrm[:1], lights, np.float32)[0]
    assert c[0] > 0 and c[1] > 0
    assert e[0] == 0.0                                   # blocked
    assert e[1] == np.float32(c[1] / np.float32(0.25))   # c / p, one rounding
    assert e[2] == 0.0 and e[3] == 0.0                   # no pick, no probability


def test_running_mean_is_the_mean_of_the_frames():
    rng = np.random.default_rng(4)
    frames = rng.uniform(0, 3, (50, 64)).astype(np.float32)
    a = None
    for k in range(1, 51):
        a = O.running_mean(a, frames[k - 1], k)
        if k == 1:
            assert np.array_equal(a, frames[0])
    np.testing.assert_allclose(a, frames.astype(np.float64).mean(0), rtol=2e-6)
    const = np.full(8, 1.75, np.float32)
    b = None
    for k in range(1, 20):
        b = O.running_mean(b, const, k)
    assert np.array_equal(b, const)


def test_exact_di_float32_sum_matches_the_float64_sum():
    sc = S.scene_heightfield(seed=3, n_lights=32, n_spheres=8, n_boxes=8)
    gb = S.gbuffer_heightfield(seed=3, width=40, height=30)
    V = O.visibility(gb.pos, sc.lights, sc.spheres, sc.boxes, np.float32)
    c32 = O.contributions(gb.pos, gb.nrm, sc.lights, np.float32)
    c64 = O.contributions(gb.pos, gb.nrm, sc.lights)
    np.testing.assert_allclose(O.exact_di_f32(V, c32), O.exact_di(V, c64), rtol=2e-6, atol=1e-12)
    assert (V == 0).mean() > 0.01        # some rays are blocked


# ------------------------------------------------------- clustered NVC --

def test_kmeans_separates_distant_groups_and_never_increases_its_objective():
    rng = np.random.default_rng(7)
    groups = [np.array([0.0, 0.0, 0.0]), np.array([10.0, 0.0, 0.0]), np.array([0.0, 10.0, 5.0])]
    P = np.concatenate([g + rng.normal(0, 0.3, (20, 3)) for g in groups])
    lights = np.concatenate([P, np.ones((60, 1))], 1)
    a, C = O.kmeans_lights(lights, [0, 1, 2], 10)        # all three seeds in group 0
    labels = [set(a[20 * g:20 * g + 20].tolist()) for g in range(3)]
    assert all(len(l) == 1 for l in labels) and len(set.union(*labels)) == 3
    for y in range(3):
        np.testing.assert_allclose(C[y], P[a == y].mean(0), rtol=0, atol=1e-12)

    def sse(a, C):
        return sum(((P[a == y] - C[y]) ** 2).sum() for y in range(len(C)))

    big = np.concatenate([rng.uniform(0, 10, (200, 3)), np.ones((200, 1))], 1)
    P = big[:, :3]
    init = rng.permutation(200)[:16]
    prev = np.inf
    for it in range(1, 8):
        a, C = O.kmeans_lights(big, init, it)
        cur = sse(a, C)
        assert cur <= prev + 1e-9
        prev = cur


def test_cluster_targets_are_the_visibility_of_a_member_light():
    sc = S.scene_heightfield(seed=2, n_lights=48, n_spheres=8, n_boxes=8)
    rng = np.random.default_rng(1)
    a, _ = O.kmeans_lights(sc.lights, rng.permutation(48)[:6], 8)
    off, mem = O.cluster_table(a, 6)
    gb = S.gbuffer_heightfield(seed=2, width=12, height=9)
    V = O.visibility(gb.pos, sc.lights, sc.spheres, sc.boxes, np.float32)
    T = O.cluster_targets(gb.pos, sc.lights, sc.spheres, sc.boxes, off, mem,
                          np.arange(gb.n), 5, 3)
    for y in range(6):
        vm = V[:, mem[off[y]:off[y + 1]]]                    # members' visibilities
        assert np.all((T[:, y][:, None] == vm).any(axis=1))
    # over many frames a target averages to the cluster's mean visibility
    y = int(np.argmax(np.diff(off)))
    acc = np.zeros(gb.n)
    F = 300
    for f in range(F):
        acc += O.cluster_targets(gb.pos, sc.lights, sc.spheres, sc.boxes, off, mem,
                                 np.arange(gb.n), 5, f)[:, y]
    mean_v = V[:, mem[off[y]:off[y + 1]]].mean(1)
    sd = np.sqrt(np.maximum(mean_v * (1 - mean_v), 1e-12) / F)
    assert np.all(np.abs(acc / F - mean_v) <= 5 * sd + 1e-12)


@pytest.mark.parametrize("mode", ["sum", "visibility"])
def test_clustered_estimate_is_unbiased_by_exact_enumeration(mode):
    """E[V(x) c(x) W] over the cluster law, every uniform candidate tuple
    and the pick law on it equals sum_x V_x c_x: the source pdf, the RIS
    weight and both reservoirs agree (Section 3.6), for either choice of
    the first step's cluster weights."""
    import itertools
    sc = S.scene_heightfield(seed=9, n_lights=6, n_spheres=6, n_boxes=6)
    assign = np.array([0, 1, 1, 2, 2, 2])
    off, mem = O.cluster_table(assign, 3)
    gb = S.gbuffer_heightfield(seed=9, width=6, height=4)
    V = O.visibility(gb.pos, sc.lights, sc.spheres, sc.boxes, np.float32)
    c32 = O.contributions(gb.pos, gb.nrm, sc.lights, np.float32)
    vis = np.random.default_rng(3).uniform(0.1, 0.9, (gb.n, 3)).astype(np.float32)
    w = O.cluster_weights(vis, c32, off, mem, mode)
    if mode == "sum":
        np.testing.assert_array_equal(
            w, O.light_weights_f32(vis, O.cluster_contributions(c32, off, mem)))
    else:
        np.testing.assert_array_equal(w, np.maximum(vis, np.float32(0.001)))
    law = O.selection_law(w)
    M = O.RIS_CANDIDATES
    checked = 0
    for p in range(gb.n):
        wsum = np.float32(0)
        for t in range(3):
            wsum = np.float32(wsum + w[p, t])
        E = 0.0
        for y in range(3):
            if law[p, y] == 0:
                continue
            ms = mem[off[y]:off[y + 1]]
            for tup in itertools.product(ms, repeat=M):
                cc = c32[p, list(tup)].astype(np.float32)
                if not (cc > 0).any():
                    continue
                pick = O.selection_law(cc[None, :])[0]
                for j in range(M):
                    if pick[j] == 0:
                        continue
                    W = float(O.ris_weight(cc, np.int64(j), w[p, y], wsum, len(ms)))
                    x = tup[j]
                    E += law[p, y] * len(ms) ** -M * pick[j] * V[p, x] * float(c32[p, x]) * W
        exact = float((V[p] * c32[p].astype(np.float64)).sum())
        if exact > 0:
            checked += 1
        np.testing.assert_allclose(E, exact, rtol=2e-5, atol=1e-12)
    assert checked >= 8
    assert (V == 0).any()


@pytest.mark.parametrize("mode", ["sum", "visibility"])
def test_sample_clustered_mean_estimate_converges_to_exact_di(mode):
    sc = S.scene_heightfield(seed=4, n_lights=24, n_spheres=8, n_boxes=8)
    rng = np.random.default_rng(2)
    a, _ = O.kmeans_lights(sc.lights, rng.permutation(24)[:5], 6)
    off, mem = O.cluster_table(a, 5)
    gb = S.gbuffer_heightfield(seed=4, width=8, height=6)
    V = O.visibility(gb.pos, sc.lights, sc.spheres, sc.boxes, np.float32)
    c32 = O.contributions(gb.pos, gb.nrm, sc.lights, np.float32)
    vis = rng.uniform(0.2, 0.9, (gb.n, 5)).astype(np.float32)
    F = 400
    est = np.zeros((F, gb.n))
    for f in range(F):
        light, W = O.sample_clustered(vis, gb.pos, gb.nrm, sc.lights, off, mem,
                                      np.arange(gb.n), 3, f, 0, mode)
        ok = light >= 0
        x = np.maximum(light, 0)
        est[f] = np.where(ok, V[np.arange(gb.n), x] * c32[np.arange(gb.n), x] * W, 0.0)
    exact = (V * c32.astype(np.float64)).sum(1)
    se = est.std(0) / np.sqrt(F)
    assert np.all(np.abs(est.mean(0) - exact) <= 5 * se + 1e-9 * exact + 1e-12)
    assert (exact > 0).mean() > 0.5


def test_visibility_weights_with_equal_visibilities_pick_clusters_uniformly():
    """With every cluster's visibility equal, the visibility-only first step
    (Section 3.6) picks each non-empty cluster with probability 1/(number of
    non-empty clusters) and never an empty one, whatever the contributions;
    the summed-contribution weights do not (they follow the contributions)."""
    sc = S.scene_heightfield(seed=2, n_lights=12, n_spheres=2, n_boxes=2)
    assign = np.array([0, 0, 1, 1, 1, 3, 3, 3, 3, 4, 4, 4])      # cluster 2 empty
    off, mem = O.cluster_table(assign, 5)
    gb = S.gbuffer_heightfield(seed=2, width=5, height=4)
    c32 = O.contributions(gb.pos, gb.nrm, sc.lights, np.float32)
    vis = np.full((gb.n, 5), 0.37, np.float32)
    law = O.selection_law(O.cluster_weights(vis, c32, off, mem, "visibility"))
    want = np.array([0.25, 0.25, 0.0, 0.25, 0.25])
    np.testing.assert_allclose(law, np.broadcast_to(want, law.shape), atol=1e-6)
    law_sum = O.selection_law(O.cluster_weights(vis, c32, off, mem, "sum"))
    assert np.abs(law_sum - want).max() > 0.05
    assert np.all(law_sum[:, 2] == 0.0)


def test_ris_weight_closed_forms():
    """W = (sum_j c_j / M) / (p(x) c(x)), p(x) = (w_y / w_sum) / m_y
    (Section 3.6).  Equal candidates give W = 1 / p(x); a pick whose
    contribution is twice the others' halves W against picking one of the
    others; and W scales with m_y and w_sum / w_y as 1/p does.  A swapped
    argument (w_sum for w_y, or the mean for c(x)) breaks these."""
    c = np.array([0.5, 0.5, 0.5, 0.5], np.float32)
    for w_y, w_sum, m_y in ((0.25, 1.0, 8), (3.0, 4.0, 1), (0.125, 0.5, 64)):
        W = float(O.ris_weight(c, np.int64(2), w_y, w_sum, m_y))
        assert W == pytest.approx(m_y * w_sum / w_y, rel=1e-6)
    c2 = np.array([1.0, 0.5, 0.5, 0.5], np.float32)
    W0 = float(O.ris_weight(c2, np.int64(0), 0.5, 1.0, 4))
    W1 = float(O.ris_weight(c2, np.int64(1), 0.5, 1.0, 4))
    assert W1 == pytest.approx(2 * W0, rel=1e-6)
    # mean 0.625, p = 0.125: W0 = 0.625 / (0.125 * 1.0)
    assert W0 == pytest.approx(5.0, rel=1e-6)


# ------------------------------------------- temporal resampling (ReSTIR) --

def _merge_expectation(c32, V, v32, prev_M, drop_inverse_M=False):
    """E[f(y) W] of one pixel's temporal merge, enumerated exactly over the
    current reservoir's light i, the previous reservoir's light j (both from
    the cache's sampler, independent) and the integer reservoir's pick."""
    w = O.light_weights_f32(v32[None], c32[None])[0]
    P = O.selection_law(w[None])[0]
    wsum = np.float32(np.sum(w.astype(np.float64)))
    L = len(c32)
    E = 0.0
    for i in range(L):
        if P[i] == 0:
            continue
        Wi = np.float32(1.0) / np.float32(w[i] / wsum)
        for j in range(L):
            if P[j] == 0 and prev_M > 0:
                continue
            Wj = np.float32(1.0) / np.float32(w[j] / wsum) if P[j] > 0 else np.float32(0)
            pj = P[j] if prev_M > 0 else (1.0 if j == 0 else 0.0)
            if pj == 0:
                continue
            args = (c32[None], np.array([i]), np.array([Wi]), np.array([j]), np.array([Wj]),
                    np.array([prev_M]), np.array([0]))
            # r = 0 keeps the last candidate with q > 0; r = 2^32 - 1 the first
            wc = np.float32(np.float32(1.0) * c32[i]) * Wi
            wp = np.float32(np.float32(min(prev_M, 20)) * c32[j]) * Wj if prev_M > 0 else np.float32(0)
            q = O.quantize_weights(np.array([[wc, wp]], np.float32))[0].astype(np.float64)
            for pick_last, prob in ((True, q[1] / q.sum()), (False, q[0] / q.sum())):
                if prob == 0:
                    continue
                import oracle.philox as ph
                old = ph.stream_words
                ph.stream_words = lambda ids, f, v, tag, m, s: np.full(
                    (len(ids), m), 0 if pick_last else (1 << 32) - 1, np.uint64)
                try:
                    y, W, M = O.temporal_merge(*args[:6], args[6], 0, 0, 0)
                finally:
                    ph.stream_words = old
                Wy = float(W[0]) * (float(M[0]) if drop_inverse_M else 1.0)
                E += P[i] * pj * prob * (V[y[0]] * float(c32[y[0]]) * Wy if y[0] >= 0 else 0.0)
    return E


@pytest.mark.parametrize("prev_M", [0, 1, 3, 40])
def test_temporal_merge_is_unbiased_by_exact_enumeration(prev_M):
    """Temporal resampling of the cache's reservoirs (Sections 3.1, 4.2):
    with the current and the previous frame's reservoir both unbiased for
    the pixel, E[V(y) c(y) W] over every (current light, previous light,
    pick) equals the all-lights DI sum V_i c_i, whatever the previous
    reservoir's confidence M (0 = disoccluded, clamped at 20); dropping the
    1/M normalisation, or the previous reservoir's weight, breaks it."""
    rng = np.random.default_rng(11 + prev_M)
    c32 = rng.uniform(0.1, 3.0, 6).astype(np.float32)
    c32[2] = 0.0                                   # a back-facing light
    V = np.array([1, 0, 1, 1, 0, 1], np.float64)   # two blocked lights
    v32 = np.array([0.9, 0.05, 0.5, 0.8, 0.0, 0.3], np.float32)
    exact = float(np.sum(V * c32.astype(np.float64)))
    E = _merge_expectation(c32, V, v32, prev_M)
    assert abs(E - exact) <= 1e-5 * exact, (E, exact)
    if prev_M > 0:
        wrong = _merge_expectation(c32, V, v32, prev_M, drop_inverse_M=True)
        assert abs(wrong - exact) > 0.5 * exact


def test_temporal_merge_special_cases():
    """A disoccluded pixel keeps the cache's sample with its weight; a pixel
    without any sample stays empty; the confidence adds up and is clamped."""
    c32 = np.array([[1.0, 2.0, 0.0]], np.float32)
    ids = np.array([7])
    y, W, M = O.temporal_merge(c32, [1], [np.float32(1.5)], [0], [np.float32(2.0)], [0], ids, 3, 1, 0)
    assert y[0] == 1 and W[0] == np.float32(1.5) and M[0] == 1
    y, W, M = O.temporal_merge(c32, [-1], [np.float32(0)], [-1], [np.float32(0)], [5], ids, 3, 1, 0)
    assert y[0] == -1 and W[0] == 0 and M[0] == 6
    y, W, M = O.temporal_merge(c32, [0], [np.float32(1)], [1], [np.float32(1)], [100], ids, 3, 1, 0)
    assert M[0] == 21 and y[0] in (0, 1) and W[0] > 0
