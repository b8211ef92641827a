"""Plain CPU oracle of the neural visibility cache hot path (Bokshansky &
Meister, "Neural Visibility Cache for Real-Time Light Sampling", JCGT 2025).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
bench's CPU-baseline / reference legs; the CUDA product path never imports,
links or runs anything here, and this module imports nothing from it.

Everything is float64 numpy, written step by step in the paper's order:
  encode (multi-resolution hash grid, Sections 3.1/3.3) -> MLP with leaky
  ReLU hidden layers and a sigmoid output (Section 3.3) -> clamp to 0.001
  (Section 3.1, bias figure) -> light weight = BRDF*cos * radiance *
  visibility (Section 3.1) -> weighted reservoir sampling of one light
  (Section 3.1) / Neural DI sum (Section 3.2); training: random world- and
  screen-space positions, one binary shadow ray per (position, light)
  (Section 3.4), loss, backpropagation, Adam (Section 3.4).

Where floating point decides an integer, the decision is taken in the
kernel's precision (float32, separate correctly-rounded operations, no
fused multiply-add): the grid cell of a position, the binary visibility of a
shadow ray (``dtype=np.float32``), and the float32 light weights that the
integer reservoir test quantises.  Everything downstream of those decisions
is float64.

Readings of points the paper leaves open (each is listed with its reason in
the design notes):
  * level resolution N_l = floor(N_min * b^l); vertex k of level l sits at
    k / N_l; the cell is c = min(floor(x * N_l), N_l - 1);
  * every level is hashed: idx = (x*1 ^ y*2654435761 ^ z*805459861) mod 2^32
    & (T - 1); entry idx holds F consecutive features; output level-major;
  * the MLP has no biases; hidden activation derivative is 1 for z > 0 and
    the slope otherwise;
  * BRDF*cos is the Lambertian (albedo 1) clamped cosine over pi: LTC with
    the identity transform; radiance of a point light falls off as 1/d^2
    with d^2 clamped to at least 1e-6;
  * the reservoir decision runs on integer weights (see ``wrs_select``).

Parity pins for every function live in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import philox as _ph

PRIMES = (1, 2654435761, 805459861)
VIS_CLAMP_F32 = np.float32(0.001)                  # Section 3.1 clamp
INV_PI_F32 = np.array([0x3EA2F983], np.uint32).view(np.float32)[0]
D2_MIN_F32 = np.float32(1e-6)
SEG_T0 = 1e-4                                      # shadow segment t range
SEG_T1 = 1.0 - 1e-4


# ----------------------------------------------------------------------------
# Multi-resolution hash-grid encoding (Sections 3.1 and 3.3)
# ----------------------------------------------------------------------------

def level_resolutions(base_resolution: int, growth: float, n_levels: int):
    """N_l = floor(N_min * b^l) for l = 0..n_levels-1, computed in float64."""
    return [int(math.floor(base_resolution * growth ** l))
            for l in range(n_levels)]


def normalize_f32(pos, bmin, bmax) -> np.ndarray:
    """x_hat = clamp((x - bmin) / (bmax - bmin), 0, 1) in float32."""
    p = np.asarray(pos, np.float32)
    lo = np.asarray(bmin, np.float32)
    ext = np.asarray(bmax, np.float32) - lo
    return np.clip((p - lo) / ext, np.float32(0), np.float32(1))


def grid_cell(xh32: np.ndarray, n_l: int):
    """Cell corner c and fraction f of x_hat at resolution N_l (float32)."""
    p = xh32 * np.float32(n_l)
    c = np.minimum(np.floor(p).astype(np.int64), n_l - 1)
    f = p - c.astype(np.float32)                     # exact in float32
    return c, f


def hash_index(cx, cy, cz, table_size: int) -> np.ndarray:
    """Spatial hash of an integer vertex: XOR of coordinate * prime, mod T."""
    m = (1 << 64) - 1
    h = ((np.asarray(cx, np.uint64) * np.uint64(PRIMES[0]))
         ^ (np.asarray(cy, np.uint64) * np.uint64(PRIMES[1]))
         ^ (np.asarray(cz, np.uint64) * np.uint64(PRIMES[2])))
    return (h & np.uint64(0xFFFFFFFF) & np.uint64(table_size - 1)).astype(np.int64)


def corner_offsets():
    """The 8 cell corners; bit 0 -> x, bit 1 -> y, bit 2 -> z."""
    return [((d >> 0) & 1, (d >> 1) & 1, (d >> 2) & 1) for d in range(8)]


@dataclass
class EncodeAux:
    idx: np.ndarray   # int64 [n, levels, 8] table row of each corner
    w: np.ndarray     # float64 [n, levels, 8] trilinear weight of each corner


def encode(cfg, table: np.ndarray, pos: np.ndarray, with_aux: bool = False):
    """Hash-grid features of each position, float64 [n, levels * F].

    table: [levels, T, F] (any float dtype; promoted to float64).
    Per level: cell c and fraction f of x_hat * N_l; each of the 8 corners
    c + delta is hashed to a table row; the feature vector is the trilinear
    blend sum_delta w_delta * table[row], w_delta = prod_d (f_d if delta_d
    else 1 - f_d).
    """
    L, F, T = cfg.n_levels, cfg.n_features, cfg.table_size
    tab = np.asarray(table, np.float64).reshape(L, T, F)
    xh = normalize_f32(pos, cfg.bounds_min, cfg.bounds_max)
    n = xh.shape[0]
    feat = np.zeros((n, L * F), np.float64)
    aux_idx = np.zeros((n, L, 8), np.int64)
    aux_w = np.zeros((n, L, 8), np.float64)
    for l, n_l in enumerate(level_resolutions(cfg.base_resolution, cfg.growth, L)):
        c, f32 = grid_cell(xh, n_l)
        f = f32.astype(np.float64)
        for d, (dx, dy, dz) in enumerate(corner_offsets()):
            idx = hash_index(c[:, 0] + dx, c[:, 1] + dy, c[:, 2] + dz, T)
            w = ((f[:, 0] if dx else 1.0 - f[:, 0])
                 * (f[:, 1] if dy else 1.0 - f[:, 1])
                 * (f[:, 2] if dz else 1.0 - f[:, 2]))
            feat[:, l * F:(l + 1) * F] += w[:, None] * tab[l, idx, :]
            aux_idx[:, l, d] = idx
            aux_w[:, l, d] = w
    if with_aux:
        return feat, EncodeAux(aux_idx, aux_w)
    return feat


def encode_backward(cfg, aux: EncodeAux, dfeat: np.ndarray) -> np.ndarray:
    """d loss / d table, [levels, T, F]: each corner row receives
    w_delta * dfeat of its level (the encoding is linear in the table)."""
    L, F, T = cfg.n_levels, cfg.n_features, cfg.table_size
    g = np.zeros((L, T, F), np.float64)
    for l in range(L):
        dl = dfeat[:, l * F:(l + 1) * F]
        for d in range(8):
            np.add.at(g[l], aux.idx[:, l, d], aux.w[:, l, d][:, None] * dl)
    return g


# ----------------------------------------------------------------------------
# MLP (Section 3.3)
# ----------------------------------------------------------------------------

def split_params(cfg, params: np.ndarray):
    """(table [levels, T, F], [W_1, ..., W_out]) views of the flat vector."""
    p = np.asarray(params, np.float64)
    L, F, T = cfg.n_levels, cfg.n_features, cfg.table_size
    tn = L * T * F
    table = p[:tn].reshape(L, T, F)
    dims = [cfg.n_inputs, *cfg.hidden, cfg.n_outputs]
    Ws, off = [], tn
    for i in range(len(dims) - 1):
        Ws.append(p[off:off + dims[i + 1] * dims[i]].reshape(dims[i + 1], dims[i]))
        off += dims[i + 1] * dims[i]
    return table, Ws


def join_params(table: np.ndarray, Ws) -> np.ndarray:
    return np.concatenate([np.ravel(table)] + [np.ravel(W) for W in Ws])


def leaky_relu(z, slope):
    return np.where(z > 0, z, slope * z)


def mlp_forward(Ws, feat: np.ndarray, slope: float):
    """Logits [n, L] and the per-layer inputs/pre-activations for backprop.

    Hidden layers: z = h W^T, h' = leaky_relu(z); output layer: logits =
    h W_out^T (the sigmoid is applied by ``sigmoid``).
    """
    acts = [np.asarray(feat, np.float64)]
    zs = []
    h = acts[0]
    for W in Ws[:-1]:
        z = h @ W.T
        zs.append(z)
        h = leaky_relu(z, slope)
        acts.append(h)
    return h @ Ws[-1].T, acts, zs


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-np.asarray(x, np.float64)))


def inference_table(cfg, table: np.ndarray) -> np.ndarray:
    """The feature table inference reads: the float32 master itself, or, for
    a cache whose tensor-core inference reads half-precision features (the
    1080p and 4K workloads' FP16 feature copy), every entry rounded to the
    nearest float16 (ties to even) and then used exactly.  Float32 inference
    always reads the master."""
    if getattr(cfg, "table_precision", "fp32") == "fp16" and cfg.precision != "fp32":
        return np.asarray(table, np.float64).astype(np.float16).astype(np.float64)
    return table


def infer(cfg, params: np.ndarray, pos: np.ndarray) -> np.ndarray:
    """Predicted visibility of every light, float64 [n, L]."""
    table, Ws = split_params(cfg, params)
    logits, _, _ = mlp_forward(Ws, encode(cfg, inference_table(cfg, table), pos), cfg.leaky_slope)
    return sigmoid(logits)


# ----------------------------------------------------------------------------
# Light weights, WRS and Neural DI (Sections 3.1 and 3.2)
# ----------------------------------------------------------------------------

def contributions(pos, nrm, lights, dtype=np.float64) -> np.ndarray:
    """Unshadowed contribution c_i of every point light, [n, L].

    Lambertian BRDF (albedo 1) times the clamped cosine, times the light's
    intensity over the squared distance (the integrand of Eq. 1 without
    visibility, for a point light): with d = l_i - x,
        c_i = I_i * max(0, n.d / |d|) / pi / max(|d|^2, 1e-6)
            = ((I_i / pi) * (n.d)) / (|d| * max(|d|^2, 1e-6))   for n.d > 0.
    With dtype=float32 the second form is evaluated operation by operation,
    each rounded to float32, which is the order the light weights use.
    """
    t = np.dtype(dtype)
    P = np.asarray(pos, t)[:, None, :]
    N = np.asarray(nrm, t)[:, None, :]
    Lp = np.asarray(lights, t)[None, :, :3]
    I = np.asarray(lights, t)[None, :, 3]
    d = Lp - P
    d2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
    ndl = (N[..., 0] * d[..., 0] + N[..., 1] * d[..., 1]) + N[..., 2] * d[..., 2]
    inv_pi = INV_PI_F32 if t == np.float32 else 1.0 / math.pi
    d2min = D2_MIN_F32 if t == np.float32 else 1e-6
    num = (I * t.type(inv_pi)) * ndl
    den = np.sqrt(d2) * np.maximum(d2, t.type(d2min))
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(ndl > 0, num / np.where(ndl > 0, den, t.type(1)), t.type(0))


def light_weights_f32(vis, c32) -> np.ndarray:
    """float32 WRS weights w_i = max(v_i, 0.001) * c_i (Section 3.1 clamp).

    vis is the float32 visibility the sampler is fed; c32 from
    ``contributions(..., dtype=np.float32)``.
    """
    v = np.asarray(vis, np.float32)
    return np.maximum(v, VIS_CLAMP_F32) * np.asarray(c32, np.float32)


def quantize_weights(w32: np.ndarray):
    """Integer reservoir weights q_i (uint64) of float32 weights w_i >= 0.

    With e = floor(log2(max_i w_i)), q_i = max(1, floor(w_i * 2^(23 - e)))
    for w_i > 0 and 0 otherwise: a power-of-two rescaling (exact) followed
    by truncation, so q_i < 2^24 and q_i / sum q = w_i / sum w up to 2^-23
    relative.  All-zero rows give all-zero q.
    """
    w = np.asarray(w32, np.float32).astype(np.float64)
    wmax = w.max(axis=1, keepdims=True)
    _, e = np.frexp(np.where(wmax > 0, wmax, 1.0))
    e = e - 1                                       # ilogb
    scaled = np.ldexp(w, (23 - e).astype(np.int64))
    q = np.where(w > 0, np.maximum(1.0, np.floor(scaled)), 0.0)
    return q.astype(np.uint64)


def wrs_select(w32: np.ndarray, pixel_ids: np.ndarray, seed: int, frame: int,
               view: int):
    """Weighted reservoir sampling of one light per pixel (Section 3.1).

    Streams over the lights in index order keeping a running integer weight
    sum Q_i = sum_{j<=i} q_j; candidate i replaces the reservoir when its
    uniform r_i (32-bit Philox word i of the pixel's stream) satisfies
    r_i * Q_i < q_i * 2^32, i.e. with probability q_i / Q_i.  The selected
    light is then i with probability q_i / Q_L.

    Returns (idx int32 [n] or -1 when all weights are 0, pdf = w_sel / sum w
    float64, wsum = sum w float64).
    """
    w32 = np.asarray(w32, np.float32)
    n, L = w32.shape
    q = quantize_weights(w32)
    r = _ph.stream_words(pixel_ids, frame, view, _ph.TAG_WRS, L, seed).astype(np.uint64)
    sel = np.full(n, -1, np.int64)
    Q = np.zeros(n, np.uint64)
    two32 = np.uint64(1 << 32)
    for i in range(L):
        Q = Q + q[:, i]
        take = (q[:, i] > 0) & (r[:, i] * Q < q[:, i] * two32)
        sel = np.where(take, i, sel)
    w64 = w32.astype(np.float64)
    wsum = w64.sum(axis=1)
    pdf = np.where(sel >= 0, w64[np.arange(n), np.maximum(sel, 0)]
                   / np.where(wsum > 0, wsum, 1.0), 0.0)
    return sel.astype(np.int32), pdf, wsum


def selection_law(w32: np.ndarray) -> np.ndarray:
    """Probabilities q_i / Q_L with which ``wrs_select`` picks each light."""
    q = quantize_weights(w32).astype(np.float64)
    s = q.sum(axis=1, keepdims=True)
    return np.where(s > 0, q / np.where(s > 0, s, 1.0), 0.0)


def neural_di(vis, c) -> np.ndarray:
    """Neural direct illumination (Section 3.2): sum_i v_i * c_i, with the
    raw sigmoid visibility (no clamp) and no shadow rays."""
    return np.sum(np.asarray(vis, np.float64) * np.asarray(c, np.float64), axis=1)


def exact_di(V, c) -> np.ndarray:
    """Direct illumination with true binary visibility: sum_i V_i c_i (the
    reflection integral, Eq. 1, for point lights)."""
    return np.sum(np.asarray(V, np.float64) * np.asarray(c, np.float64), axis=1)


def estimator_moments(V, c, p):
    """Mean and variance of the one-sample estimator V_s c_s / p_s of Eq. 1.

    E = sum_{p_i > 0} V_i c_i ; Var = sum_{p_i > 0} (V_i c_i)^2 / p_i - E^2.
    Unbiased (E = exact DI) exactly when p_i > 0 wherever V_i c_i > 0, which
    the 0.001 clamp guarantees for every light with c_i > 0.
    """
    f = np.asarray(V, np.float64) * np.asarray(c, np.float64)
    p = np.asarray(p, np.float64)
    pos = p > 0
    E = np.sum(np.where(pos, f, 0.0), axis=1)
    M2 = np.sum(np.where(pos, f * f / np.where(pos, p, 1.0), 0.0), axis=1)
    return E, M2 - E * E


# ----------------------------------------------------------------------------
# Training data (Section 3.4)
# ----------------------------------------------------------------------------

def training_positions(batch: int, world_min, world_max, screen_pos,
                       seed: int, frame: int, n_world: Optional[int] = None) -> np.ndarray:
    """float32 [batch, 3]: world-space then screen-space training positions
    (Section 3.4 compares the two placements and their combination).

    The first n_world positions (by default ceil(batch / 2), the paper's
    equal split; all of them when no screen positions are given) are uniform
    in the scene bounds: x = lo + u * (hi - lo) with u = 24-bit uniforms of
    stream (j, frame, 0, world); position n_world + s picks G-buffer pixel
    floor(r * P / 2^32), r = word 0 of stream (s, frame, 0, screen).
    """
    have_screen = screen_pos is not None and len(screen_pos) > 0
    if not have_screen:
        n_world = batch
    elif n_world is None:
        n_world = batch - batch // 2
    n_world = min(max(int(n_world), 0), batch)
    n_screen = batch - n_world
    lo = np.asarray(world_min, np.float32)
    ext = np.asarray(world_max, np.float32) - lo
    out = np.empty((batch, 3), np.float32)
    if n_world:
        r = _ph.stream_words(np.arange(n_world), frame, 0, _ph.TAG_WORLD, 3, seed)
        out[:n_world] = lo + _ph.uniform24(r) * ext
    if n_screen:
        P = len(screen_pos)
        r = _ph.stream_words(np.arange(n_screen), frame, 0, _ph.TAG_SCREEN, 1, seed)
        pix = ((r[:, 0].astype(np.uint64) * np.uint64(P)) >> np.uint64(32)).astype(np.int64)
        out[n_world:] = np.asarray(screen_pos, np.float32)[pix]
    return out


def _dot3(a, b):
    return (a[..., 0] * b[..., 0] + a[..., 1] * b[..., 1]) + a[..., 2] * b[..., 2]


def visibility(pos, lights, spheres, boxes, dtype=np.float64) -> np.ndarray:
    """Binary visibility V [n, L] of each light from each position.

    A point light is visible when the segment x + t (l - x), t in
    [1e-4, 1 - 1e-4], meets no occluder: a sphere blocks it when the
    segment's closest point lies strictly inside (|c - q|^2 < r^2); a box
    blocks it when the segment overlaps the closed box (slab test).  The
    arithmetic runs in ``dtype`` with float32 giving the kernel's decision;
    the reciprocals 1/|d|^2 and 1/d_a are formed once per (position, light)
    and multiply the per-occluder numerators.
    """
    t = np.dtype(dtype).type
    X = np.asarray(pos, t)[:, None, :]
    Lp = np.asarray(lights, t)[None, :, :3]
    D = Lp - X                                    # [n, L, 3]
    dd = _dot3(D, D)
    occ = np.zeros(dd.shape, bool)
    t0, t1 = t(SEG_T0), t(SEG_T1)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv_dd = np.where(dd > 0, t(1) / np.where(dd > 0, dd, t(1)), t(0))
        inv_d = np.where(D != 0, t(1) / np.where(D != 0, D, t(1)), t(0))
    for s in np.asarray(spheres, t).reshape(-1, 4):
        C, r = s[:3], s[3]
        O = C - X
        tc = _dot3(O, D) * inv_dd         # dd = 0: the segment is a point, t -> t0
        tc = np.minimum(np.maximum(tc, t0), t1)
        Q = X + tc[..., None] * D
        E = C - Q
        occ |= _dot3(E, E) < r * r
    for b in np.asarray(boxes, t).reshape(-1, 6):
        lo, hi = b[:3], b[3:]
        tmin = np.full(dd.shape, t0, t)
        tmax = np.full(dd.shape, t1, t)
        miss = np.zeros(dd.shape, bool)
        for a in range(3):
            xa = np.broadcast_to(X[..., a], dd.shape)
            da = D[..., a]
            par = da == 0
            miss |= par & ((xa < lo[a]) | (xa > hi[a]))
            ta = (lo[a] - xa) * inv_d[..., a]
            tb = (hi[a] - xa) * inv_d[..., a]
            tn = np.where(par, t0, np.minimum(ta, tb))
            tf = np.where(par, t1, np.maximum(ta, tb))
            tmin = np.maximum(tmin, tn)
            tmax = np.minimum(tmax, tf)
        occ |= (~miss) & (tmin <= tmax)
    return (~occ).astype(np.float64)


# ----------------------------------------------------------------------------
# The shading pass (Section 3.1) and exact direct illumination (Section 4.4)
# ----------------------------------------------------------------------------

def shading_estimate(pos, nrm, lights, spheres, boxes, idx, pdf) -> np.ndarray:
    """One-sample estimate of Eq. 1 for each pixel's sampled light (the
    shading pass after light sampling, Section 3.1): one shadow ray towards
    light s = idx[p], and

        e[p] = V_s c_s / pdf[p]

    with V_s the float32 shadow-ray decision of ``visibility`` and c_s the
    float32 contribution of ``contributions``; the division rounds once to
    float32.  Pixels with idx < 0 or pdf <= 0 give 0.  Averaged over the
    sampler's choice (probability pdf of light s), e has mean sum_i V_i c_i:
    the estimator is unbiased wherever every light with c_i > 0 can be
    picked."""
    pos = np.asarray(pos, np.float32)
    nrm = np.asarray(nrm, np.float32)
    idx = np.asarray(idx, np.int64)
    pdf = np.asarray(pdf, np.float32)
    est = np.zeros(len(pos), np.float32)
    sel = np.nonzero((idx >= 0) & (pdf > 0))[0]
    if len(sel) == 0:
        return est
    rows = np.arange(len(sel))
    V = visibility(pos[sel], lights, spheres, boxes, np.float32)[rows, idx[sel]]
    c = contributions(pos[sel], nrm[sel], lights, np.float32)[rows, idx[sel]]
    ok = (V > 0) & (c > 0)
    est[sel] = np.where(ok, c.astype(np.float32) / np.where(ok, pdf[sel], np.float32(1)),
                        np.float32(0)).astype(np.float32)
    return est


def running_mean(accum, est, count: int) -> np.ndarray:
    """Temporal accumulation of the per-frame estimates: the mean of the
    first k frames, updated in place of the mean of k - 1 as
    a <- a + (e - a) / k (each operation rounded to float32; a = e for
    k = 1)."""
    e = np.asarray(est, np.float32)
    if count <= 1:
        return e.copy()
    a = np.asarray(accum, np.float32)
    return (a + (e - a) / np.float32(count)).astype(np.float32)


def exact_di_f32(V, c32) -> np.ndarray:
    """exact_di evaluated as a float32 sum over the lights in order, each
    unblocked light's float32 contribution added with one rounding."""
    V = np.asarray(V)
    c = np.asarray(c32, np.float32)
    s = np.zeros(c.shape[0], np.float32)
    for i in range(c.shape[1]):
        take = (V[:, i] > 0) & (c[:, i] > 0)
        s = np.where(take, (s + c[:, i]).astype(np.float32), s)
    return s


# ----------------------------------------------------------------------------
# Clustered NVC (Section 3.6)
# ----------------------------------------------------------------------------

RIS_CANDIDATES = 4   # candidates drawn in the chosen cluster (streaming RIS)


def kmeans_lights(lights, init_idx, iters: int):
    """Lloyd's k-means (Section 3.6) of the light positions, float64.

    Centroids start at the lights ``init_idx`` (k distinct indices, drawn by
    the caller); each iteration assigns every light to its nearest centroid
    (squared distance (dx^2 + dy^2) + dz^2, ties to the lower index) and
    moves each centroid to the mean of its members, summed in light order (a
    cluster left empty keeps its centroid).  Returns (assign int32 [n],
    centroids float64 [k, 3]) after ``iters`` iterations, the assignment
    being the one the final centroids induce."""
    P = np.asarray(lights, np.float64)[:, :3]
    C = P[np.asarray(init_idx, np.int64)].copy()
    k = C.shape[0]

    def assign_to(C):
        d = P[:, None, :] - C[None, :, :]
        d2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
        return np.argmin(d2, axis=1)          # first minimum: ties to the lower index

    for _ in range(iters):
        a = assign_to(C)
        for y in range(k):
            members = np.nonzero(a == y)[0]
            if len(members) == 0:
                continue
            s = np.zeros(3)
            for i in members:                   # light order
                s = s + P[i]
            C[y] = s / len(members)
    return assign_to(C).astype(np.int32), C


def cluster_table(assign, k: int):
    """CSR cluster table: offsets [k + 1] and members [n], each cluster's
    lights in increasing index order."""
    assign = np.asarray(assign, np.int64)
    order = np.argsort(assign, kind="stable")
    counts = np.bincount(assign, minlength=k)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    return offsets, order.astype(np.int32)


def _member(offsets, members, y, r):
    """The member of cluster y chosen by the 32-bit word r: floor(r m_y / 2^32)."""
    m = (offsets[y + 1] - offsets[y]).astype(np.uint64)
    j = (np.asarray(r, np.uint64) * m) >> np.uint64(32)
    return members[offsets[y] + j.astype(np.int64)]


def cluster_targets(pos, lights, spheres, boxes, offsets, members, sample_ids, seed: int,
                    frame: int) -> np.ndarray:
    """Training targets of the clustered cache (Section 3.6): for each
    position and cluster y, the binary visibility of one member light drawn
    uniformly (word y of the stream (sample, frame, 0, TAG_CLUSTER)), so the
    network learns the cluster's average visibility.  [n, k] float64 0/1;
    empty clusters give 0."""
    offsets = np.asarray(offsets, np.int64)
    members = np.asarray(members, np.int64)
    k = len(offsets) - 1
    n = len(pos)
    r = _ph.stream_words(sample_ids, frame, 0, _ph.TAG_CLUSTER, k, seed)
    V = visibility(pos, lights, spheres, boxes, np.float32)       # [n, L]
    out = np.zeros((n, k))
    for y in range(k):
        if offsets[y + 1] == offsets[y]:
            continue
        x = _member(offsets, members, y, r[:, y])
        out[:, y] = V[np.arange(n), x]
    return out


def cluster_contributions(c32, offsets, members) -> np.ndarray:
    """c_hat_y = sum of the member lights' float32 contributions, in member
    order (float32): positive exactly when some member contributes, so every
    contributing light stays reachable through its cluster."""
    c32 = np.asarray(c32, np.float32)
    k = len(offsets) - 1
    out = np.zeros((c32.shape[0], k), np.float32)
    for y in range(k):
        s = np.zeros(c32.shape[0], np.float32)
        for i in members[offsets[y]:offsets[y + 1]]:
            s = (s + c32[:, i]).astype(np.float32)
        out[:, y] = s
    return out


CLUSTER_WEIGHT_MODES = ("sum", "visibility")


def cluster_weights(vis, c32, offsets, members, mode: str = "sum") -> np.ndarray:
    """float32 [n, k] weights of the first sampling step (Section 3.6).

    "sum":        w_y = max(v_y, 0.001) * c_hat_y, the cluster's inferred
                  average visibility times its members' summed contribution;
    "visibility": w_y = max(v_y, 0.001), the inferred average visibility
                  alone (the step's weight as the paper words it; the
                  contributions enter only through the RIS step).
    Empty clusters weigh 0 in both modes.  Every non-empty cluster whose
    members contribute keeps w_y > 0, so every contributing light stays
    reachable."""
    offsets = np.asarray(offsets, np.int64)
    m = (offsets[1:] - offsets[:-1]) > 0
    if mode == "sum":
        return light_weights_f32(vis, cluster_contributions(c32, offsets, members))
    if mode == "visibility":
        v = np.maximum(np.asarray(vis, np.float32), np.float32(0.001))
        return np.where(m[None, :], v, np.float32(0.0)).astype(np.float32)
    raise ValueError(mode)


def ris_weight(c_cand, j, w_y, w_sum, m_y):
    """Unbiased contribution weight of candidate j after streaming RIS with
    source pdf p(x) = (w(y) / w_sum) / m_y (the cluster's selection
    probability times a uniform member) and target pdf c(x):
        W = (sum_j c_j / M) / (p(x) c(x_j)),
    every operation rounded to float32 in this order."""
    c = np.asarray(c_cand, np.float32)
    M = np.float32(c.shape[-1])
    s = np.zeros(c.shape[:-1], np.float32)
    for t in range(c.shape[-1]):
        s = (s + c[..., t]).astype(np.float32)
    mean = (s / M).astype(np.float32)
    p = ((np.float32(w_y) / np.float32(w_sum)).astype(np.float32) / np.float32(m_y)).astype(np.float32)
    den = (p * np.take_along_axis(c, np.asarray(j)[..., None], -1)[..., 0]).astype(np.float32)
    return (mean / den).astype(np.float32)


def sample_clustered(vis, pos, nrm, lights, offsets, members, pixel_ids, seed: int,
                     frame: int, view: int, mode: str = "sum"):
    """Two-step light sampling of the clustered cache (Section 3.6).

    1. WRS over the k clusters with the weights of ``cluster_weights``
       (by default w_y = max(v_y, 0.001) c_hat_y; the integer reservoir of
       ``wrs_select``, stream TAG_WRS).
    2. Streaming RIS in the chosen cluster y: RIS_CANDIDATES members drawn
       uniformly (words 0..M-1 of stream (pixel, frame, view, TAG_RIS)), one
       kept by the integer reservoir on their float32 contributions (words
       M..2M-1), and its contribution weight from ``ris_weight``.

    vis: the cache's float32 cluster visibilities [n, k].  Returns (light
    int32 [n], -1 when nothing contributes; W float32 [n])."""
    offsets = np.asarray(offsets, np.int64)
    members = np.asarray(members, np.int64)
    c32 = contributions(pos, nrm, lights, np.float32)
    w = cluster_weights(vis, c32, offsets, members, mode)
    y, _, _ = wrs_select(w, pixel_ids, seed, frame, view)
    n = len(pos)
    M = RIS_CANDIDATES
    r = _ph.stream_words(pixel_ids, frame, view, _ph.TAG_RIS, 2 * M, seed)
    light = np.full(n, -1, np.int32)
    W = np.zeros(n, np.float32)
    wsum = np.zeros(n, np.float32)
    for t in range(w.shape[1]):
        wsum = (wsum + w[:, t]).astype(np.float32)
    for p in np.nonzero(y >= 0)[0]:
        yy = int(y[p])
        m_y = int(offsets[yy + 1] - offsets[yy])
        cand = np.array([_member(offsets, members, yy, r[p, t]) for t in range(M)], np.int64)
        cc = c32[p, cand].astype(np.float32)
        if not (cc > 0).any():
            continue
        q = quantize_weights(cc[None, :])[0]
        Q = np.uint64(0)
        j = -1
        for t in range(M):
            Q = Q + q[t]
            if q[t] > 0 and np.uint64(r[p, M + t]) * Q < q[t] * np.uint64(1 << 32):
                j = t
        light[p] = cand[j]
        W[p] = ris_weight(cc, np.int64(j), w[p, yy], wsum[p], m_y)
    return light, W


# ----------------------------------------------------------------------------
# The cache as ReSTIR's initial-candidate generator (Sections 3.1 and 4.2)
# ----------------------------------------------------------------------------

TEMPORAL_M_CAP = 20   # the previous reservoir counts at most 20x the new one


def integer_pick(w32: np.ndarray, r: np.ndarray) -> np.ndarray:
    """The integer streaming reservoir of ``wrs_select`` over the columns of
    w32 [n, m] with the words r [n, m]: index of the kept candidate, -1 when
    every weight is 0."""
    q = quantize_weights(np.asarray(w32, np.float32))
    r = np.asarray(r).astype(np.uint64)
    sel = np.full(q.shape[0], -1, np.int64)
    Q = np.zeros(q.shape[0], np.uint64)
    for i in range(q.shape[1]):
        Q = Q + q[:, i]
        take = (q[:, i] > 0) & (r[:, i] * Q < q[:, i] * np.uint64(1 << 32))
        sel = np.where(take, i, sel)
    return sel


def target_at(c32: np.ndarray, light: np.ndarray) -> np.ndarray:
    """The resampling target p_hat(y) = c_y, the float32 unshadowed
    contribution of light y at each pixel (0 for y = -1)."""
    light = np.asarray(light, np.int64)
    t = np.take_along_axis(np.asarray(c32, np.float32), np.maximum(light, 0)[:, None], 1)[:, 0]
    return np.where(light >= 0, t, np.float32(0)).astype(np.float32)


def temporal_merge(c32, cur_light, cur_W, prev_light, prev_W, prev_M, pixel_ids, seed: int,
                   frame: int, view: int):
    """Temporal resampling of a pixel's reservoirs (the ReSTIR combination
    the paper feeds with the cache's samples: Section 3.1, last paragraph,
    and Section 4.2).

    The frame's initial-candidate reservoir (y_c, W_c), made by the cache's
    sampler, counts M_c = 1 candidate; the previous frame's reservoir at the
    same pixel (y_p, W_p, M_p) counts M_p' = min(M_p, 20 M_c) (M_p = 0 where
    the pixel is disoccluded: the cache's candidate alone).  With the target
    p_hat(y) = c_y (float32 contributions c32 [n, L]):
        w_c = (M_c p_hat(y_c)) W_c,   w_p = (M_p' p_hat(y_p)) W_p,
    the integer reservoir picks y between [y_c, y_p] with words 0, 1 of
    stream (pixel, frame, view, TAG_TEMPORAL), and
        M = M_c + M_p',   W = (w_c + w_p) / (M p_hat(y)),
    every product, sum and quotient a float32 rounding in that order;
    y = -1 and W = 0 when both weights are 0.  Returns (light int32, W
    float32, M int32), each [n]."""
    n = len(cur_light)
    Mc = np.ones(n, np.int64)
    Mp = np.minimum(np.asarray(prev_M, np.int64), TEMPORAL_M_CAP * Mc)
    pc = target_at(c32, cur_light)
    pp = target_at(c32, prev_light)
    f32 = np.float32
    wc = ((Mc.astype(f32) * pc).astype(f32) * np.asarray(cur_W, f32)).astype(f32)
    wp = ((Mp.astype(f32) * pp).astype(f32) * np.asarray(prev_W, f32)).astype(f32)
    wc = np.where(np.asarray(cur_light) >= 0, wc, f32(0))
    wp = np.where((np.asarray(prev_light) >= 0) & (Mp > 0), wp, f32(0))
    r = _ph.stream_words(pixel_ids, frame, view, _ph.TAG_TEMPORAL, 2, seed)
    pick = integer_pick(np.stack([wc, wp], 1), r)
    light = np.where(pick == 0, cur_light, np.where(pick == 1, prev_light, -1)).astype(np.int32)
    M = (Mc + Mp).astype(np.int32)
    py = target_at(c32, light)
    s = (wc + wp).astype(f32)
    den = (M.astype(f32) * py).astype(f32)
    with np.errstate(divide="ignore", invalid="ignore"):
        W = np.where(light >= 0, (s / np.where(light >= 0, den, f32(1))).astype(f32), f32(0))
    return light, W.astype(np.float32), M


# ----------------------------------------------------------------------------
# Loss, backpropagation and Adam (Sections 3.3 and 3.4)
# ----------------------------------------------------------------------------

def loss_and_grad(loss: str, logits: np.ndarray, y: np.ndarray):
    """Mean loss over all (position, light) pairs and d loss / d logits.

    L2 (the paper's loss): mean (s - y)^2, gradient 2 (s - y) s (1 - s) / n.
    BCE: mean of -y log s - (1 - y) log(1 - s), gradient (s - y) / n.
    """
    z = np.asarray(logits, np.float64)
    y = np.asarray(y, np.float64)
    s = sigmoid(z)
    n = z.size
    if loss == "l2":
        return float(np.mean((s - y) ** 2)), 2.0 * (s - y) * s * (1.0 - s) / n
    if loss == "bce":
        # -y log s - (1-y) log(1-s) = softplus(z) - y z, in a stable form
        sp = np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))
        return float(np.mean(sp - y * z)), (s - y) / n
    raise ValueError(loss)


def mlp_backward(Ws, acts, zs, dlogits, slope: float):
    """Gradients of the weights ([dW_1, ..., dW_out]) and of the encoded
    input (dfeat), by the chain rule through h' = leaky_relu(h W^T)."""
    dWs = [None] * len(Ws)
    delta = np.asarray(dlogits, np.float64)
    dWs[-1] = delta.T @ acts[-1]
    g = delta @ Ws[-1]
    for k in range(len(Ws) - 2, -1, -1):
        delta = g * np.where(zs[k] > 0, 1.0, slope)
        dWs[k] = delta.T @ acts[k]
        g = delta @ Ws[k]
    return dWs, g


def learning_rate(cfg, step: int) -> float:
    """Learning rate of the ``step``-th update (1-based).

    Constant, or the paper's ramp: start at lr and lower it linearly to
    lr_end over the first lr_ramp_steps updates (Section 3.4).
    """
    if cfg.lr_schedule == "constant":
        return float(cfg.lr)
    if cfg.lr_schedule == "paper_ramp":
        s = min(step - 1, cfg.lr_ramp_steps)
        return float(cfg.lr + (cfg.lr_end - cfg.lr) * s / cfg.lr_ramp_steps)
    raise ValueError(cfg.lr_schedule)


def adam_update(theta, grad, m, v, step: int, lr: float, beta1: float,
                beta2: float, eps: float):
    """One Adam update (Kingma & Ba), bias-corrected, of every parameter:
    m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
    theta -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


@dataclass
class TrainState:
    params: np.ndarray                     # float64 flat vector
    m: np.ndarray
    v: np.ndarray
    step: int = 0
    skipped: int = 0

    @staticmethod
    def fresh(params) -> "TrainState":
        p = np.asarray(params, np.float64).copy()
        return TrainState(p, np.zeros_like(p), np.zeros_like(p))


def gradients(cfg, params, pos, targets):
    """Loss and d loss / d params (flat, float64) on a batch."""
    table, Ws = split_params(cfg, params)
    feat, aux = encode(cfg, table, pos, with_aux=True)
    logits, acts, zs = mlp_forward(Ws, feat, cfg.leaky_slope)
    loss, dlog = loss_and_grad(cfg.loss, logits, targets)
    dWs, dfeat = mlp_backward(Ws, acts, zs, dlog, cfg.leaky_slope)
    dtable = encode_backward(cfg, aux, dfeat)
    return loss, join_params(dtable, dWs)


def train_step(cfg, state: TrainState, scene, screen_pos, seed: int,
               frame: int, n_world: Optional[int] = None):
    """One online training step (Section 3.4): positions -> shadow-ray
    targets -> loss -> gradients -> Adam.  A non-finite gradient skips the
    update and counts it.  Returns the loss."""
    pos = training_positions(cfg.batch_positions, scene.world_min,
                             scene.world_max, screen_pos, seed, frame, n_world)
    y = visibility(pos, scene.lights, scene.spheres, scene.boxes, np.float32)
    loss, g = gradients(cfg, state.params, pos, y)
    if not np.all(np.isfinite(g)):
        state.skipped += 1
        return loss
    state.step += 1
    state.params, state.m, state.v = adam_update(
        state.params, g, state.m, state.v, state.step,
        learning_rate(cfg, state.step), cfg.beta1, cfg.beta2, cfg.eps)
    return loss


# ----------------------------------------------------------------------------
# One frame of the hot path
# ----------------------------------------------------------------------------

def shade(cfg, params, pos, nrm, lights, seed: int, frame: int, view: int = 0,
          pixel_offset: int = 0, vis: Optional[np.ndarray] = None):
    """Inference + WRS + Neural DI for a batch of pixels.

    ``vis`` (float32) overrides the oracle's own prediction, so the sampler
    can be checked bit-exactly on identical visibility.  Returns a dict with
    vis, idx, pdf, wsum and radiance (Neural DI).
    """
    if vis is None:
        vis64 = infer(cfg, params, pos)
        vis32 = vis64.astype(np.float32)
    else:
        vis32 = np.asarray(vis, np.float32)
        vis64 = vis32.astype(np.float64)
    c32 = contributions(pos, nrm, lights, np.float32)
    w = light_weights_f32(vis32, c32)
    ids = pixel_offset + np.arange(len(pos), dtype=np.int64)
    idx, pdf, wsum = wrs_select(w, ids, seed, frame, view)
    c64 = contributions(pos, nrm, lights, np.float64)
    return dict(vis=vis64, idx=idx, pdf=pdf, wsum=wsum,
                radiance=neural_di(vis64, c64))
