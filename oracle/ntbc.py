"""Oracle: NTBC network, inference to BC blocks, training losses/gradients, QAT, Adam.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this module.

Plain numpy, FP64 unless stated. Where floating point decides an integer (the
endpoint quantisation to RGB565 / u8, the palette argmax, the exported grid
codes) the decision is taken in FP32 like the kernels do, and the docstring says so.

Sections of the paper followed:
  * Sec. 3, Eq. palette / Eq. weightBC4: palettes (linear index n, weight w_n).
  * Sec. 3.2, Eq. dist: d_n = -||x - p_n||, n = argmax d_n.
  * Sec. 3.2, Eq. lossNTBC_e / lossNTBC_c: L_endpoint = L_e + L_cd, L_color = L_c + L_cd.
  * Sec. 3.2, Eq. softmax and App. A: straight-through argmax, backward of the
    softmax expectation with temperature T.
  * Sec. 2.3, Eq. quantize / dequantize / quantizer / scaling_factor, Sec. 3.3: per-level QAT.
  * Sec. 3.4: 3 x 64 SELU hidden layers, sigmoid outputs, multi-resolution 2D
    grids with 2 features per level from resolution 16, Adam (0.9, 0.999, 1e-15),
    learning rates 0.01 (grids) / 0.005 (MLPs), 10 warm-up steps then cosine to 0.
  * Sec. 4.1: conservative / aggressive packaging (outputs per texture).

Readings where the paper is silent or garbled (each one is listed in the design notes):
  * grid level resolution res_l = floor(N_min (N_max/N_min)^(l/(L-1)) + 0.5);
    each level is a dense res x res x F array (this reproduces the 13.37 MB and
    26.74 MB model sizes of Sec. 4.3 exactly);
  * corner-aligned bilinear lookup: p = u (res-1), i0 = min(floor p, res-2);
    texel centres u = (x+0.5)/W, block centres s = (bx+0.5)/(W/4);
  * the endpoint grid keeps the colour-grid levels whose resolution does not
    exceed the number of blocks per side (7 of 8 levels in Sec. 3.4);
  * Linear layers carry biases;
  * endpoints quantise as floor(e*31+0.5) (G: *63) or floor(e*255+0.5) in FP32;
    indices are chosen against the palette of the quantised endpoints, by
    least squared distance, ties to the lowest hardware code; BC1 blocks
    are ordered colour0 > colour1 by swapping, equal colours give all codes 0;
  * losses are means over their elements; L_e targets are the decoded stored
    endpoints of the reference blocks; L_cd decodes with the reference
    endpoints for both networks; the endpoint network's palette uses the
    unquantised prediction; training argmax ties go to the lowest linear n;
  * STE backward: d dec / d d_j = (1/T) sigma_j (P_j - sum_i sigma_i P_i), the
    corrected form of App. A's last equation (the derivation's own lines give
    w_n - w_hat, not n - w_hat); d||a - b||/da guarded by max(norm, 1e-6);
  * QAT zero point: the paper's z = round(alpha * s) is garbled; the range is
    [min(0, min level), max(0, max level)] and z = round(-alpha / s), so zero is
    exactly representable (the property the paper asks of z); round half away
    from zero; all-zero level: s = 1, z = 0; STE gradient 1 where unclamped;
  * one LR schedule spans the main and the QAT phase;
  * FP8 weights (an extension for the precision study; the paper stores FP16): E4M3
    round to nearest even, saturating; one power-of-two scale per layer shared by its
    weights and bias;
  * FP8 arithmetic (the same study): each layer's input rounded to E4M3 at a per-layer
    power-of-two scale calibrated on a fixed sample of the material (one binade of
    headroom above the sampled maximum), exact products and sums, the bias added
    exactly.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import bc as _bc

BC1, BC4 = _bc.BC1, _bc.BC4
SELU_LAMBDA = 1.0507009873554804934193349852946
SELU_ALPHA = 1.6732632423543772848170429916717
NORM_GUARD = 1e-6


# ----------------------------------------------------------------------------
# configuration
# ----------------------------------------------------------------------------

def level_resolutions(levels: int, n_min: int, n_max: int):
    """Per-level grid resolutions, geometric from n_min to n_max (Sec. 3.4)."""
    if levels == 1:
        return [int(n_min)]
    out = []
    for l in range(levels):
        out.append(int(math.floor(n_min * (n_max / n_min) ** (l / (levels - 1)) + 0.5)))
    return out


def endpoint_resolutions(color_res, blocks_per_side):
    return [r for r in color_res if r <= blocks_per_side]


@dataclass
class ModelDesc:
    width: int
    height: int
    formats: list                      # per texture: 1 (BC1) or 4 (BC4), in material order
    color_res: list
    endpoint_res: list
    features: int = 2
    hidden_layers: int = 3
    hidden_width: int = 64
    activation: str = "selu"           # 'selu' or 'relu'

    @property
    def blocks_x(self):
        return self.width // 4

    @property
    def blocks_y(self):
        return self.height // 4

    @property
    def n_blocks(self):
        return self.blocks_x * self.blocks_y

    @property
    def channels(self):
        return [_bc.channels(f) for f in self.formats]

    @property
    def out_color(self):
        """3 N_RGB + N_SC colour outputs (Sec. 4.1, aggressive packaging)."""
        return sum(self.channels)

    @property
    def out_endpoint(self):
        """6 N_RGB + 2 N_SC endpoint outputs."""
        return 2 * sum(self.channels)

    @property
    def in_color(self):
        return self.features * len(self.color_res)

    @property
    def in_endpoint(self):
        return self.features * len(self.endpoint_res)

    def color_offsets(self):
        off, out = 0, []
        for c in self.channels:
            out.append(off)
            off += c
        return out

    def endpoint_offsets(self):
        return [2 * o for o in self.color_offsets()]

    def mlp_dims(self, which):
        hidden = [self.hidden_width] * self.hidden_layers
        if which == "color":
            return [self.in_color] + hidden + [self.out_color]
        return [self.in_endpoint] + hidden + [self.out_endpoint]


def storage_bytes(desc: ModelDesc, grid_bits=8, weight_bytes=2):
    """Bytes of a stored model: all grid levels at grid_bits per feature plus both MLPs
    (weights and biases) at weight_bytes per value (Sec. 4.3 model sizes)."""
    grid = sum(r * r for r in desc.color_res) + sum(r * r for r in desc.endpoint_res)
    grid_b = grid * desc.features * grid_bits // 8
    mlp = 0
    for which in ("color", "endpoint"):
        d = desc.mlp_dims(which)
        mlp += sum(d[i] * d[i + 1] + d[i + 1] for i in range(len(d) - 1))
    return grid_b + mlp * weight_bytes


# ----------------------------------------------------------------------------
# coordinates and multi-resolution grid lookup
# ----------------------------------------------------------------------------

def texel_coords(w, h, xs, ys):
    return (np.asarray(xs, np.float64) + 0.5) / w, (np.asarray(ys, np.float64) + 0.5) / h


def block_coords(bw, bh, bxs, bys):
    return (np.asarray(bxs, np.float64) + 0.5) / bw, (np.asarray(bys, np.float64) + 0.5) / bh


def grid_lookup(levels, u, v):
    """Bilinear lookup of every level at normalised (u, v), features concatenated level-major.
    levels: list of [res, res, F] arrays (row = y). Returns (features [N, L*F], cache)."""
    feats, cache = [], []
    for g in levels:
        res = g.shape[0]
        px = u * (res - 1)
        py = v * (res - 1)
        ix = np.minimum(np.floor(px), res - 2).astype(np.int64)
        iy = np.minimum(np.floor(py), res - 2).astype(np.int64)
        fx = px - ix
        fy = py - iy
        w00 = (1 - fx) * (1 - fy)
        w01 = fx * (1 - fy)
        w10 = (1 - fx) * fy
        w11 = fx * fy
        val = (w00[:, None] * g[iy, ix] + w01[:, None] * g[iy, ix + 1]
               + w10[:, None] * g[iy + 1, ix] + w11[:, None] * g[iy + 1, ix + 1])
        feats.append(val)
        cache.append((res, ix, iy, (w00, w01, w10, w11)))
    return np.concatenate(feats, axis=1), cache


def grid_lookup_backward(levels, cache, g_feats, masks=None):
    """Scatter-add d loss / d features back to the grid corners; masks (optional, per
    level, same shape as the level) gate the gradient (QAT straight-through)."""
    grads = []
    F = levels[0].shape[2]
    for l, (res, ix, iy, ws) in enumerate(cache):
        g = g_feats[:, l * F:(l + 1) * F]
        acc = np.zeros(res * res * F)
        corners = ((iy, ix), (iy, ix + 1), (iy + 1, ix), (iy + 1, ix + 1))
        for (cy, cx), wgt in zip(corners, ws):
            for f in range(F):
                idx = (cy * res + cx) * F + f
                acc += np.bincount(idx, weights=wgt * g[:, f], minlength=res * res * F)
        acc = acc.reshape(res, res, F)
        if masks is not None:
            acc = acc * masks[l]
        grads.append(acc)
    return grads


# ----------------------------------------------------------------------------
# MLP (Sec. 3.4)
# ----------------------------------------------------------------------------

def selu(z):
    return np.where(z > 0, SELU_LAMBDA * z, SELU_LAMBDA * SELU_ALPHA * np.expm1(np.minimum(z, 0.0)))


def selu_grad(z):
    return np.where(z > 0, SELU_LAMBDA, SELU_LAMBDA * SELU_ALPHA * np.exp(np.minimum(z, 0.0)))


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def _act(z, kind):
    return selu(z) if kind == "selu" else np.maximum(z, 0.0)


def _act_grad(z, kind):
    return selu_grad(z) if kind == "selu" else (z > 0).astype(np.float64)


def bf16_round(x):
    """Nearest BFloat16 value (1 sign, 8 exponent, 7 mantissa bits: the FP32 exponent range
    with a 2^-7 relative spacing, subnormal spacing 2^-133), ties to even mantissa."""
    x = np.asarray(x, np.float64)
    a = np.abs(x)
    _, ex = np.frexp(np.maximum(a, 2.0 ** -126))          # a = m 2^ex, m in [0.5, 1)
    step = np.ldexp(1.0, ex - 1 - 7)
    q = np.round(a / step) * step
    return np.copysign(q, x)


def _act_grad_from_out(a, kind):
    """The activation's derivative written through its output a: SELU' = lambda (a > 0),
    a + lambda alpha (a <= 0, since SELU(z) = lambda alpha (e^z - 1) there); ReLU' = [a > 0]."""
    if kind == "selu":
        return np.where(a > 0, SELU_LAMBDA, a + SELU_LAMBDA * SELU_ALPHA)
    return (a > 0).astype(np.float64)


def mlp_forward(layers, x, kind, rnd=None):
    """layers: [(W [out, in], b [out]), ...]; hidden layers use `kind`, the last sigmoid.
    rnd (optional): rounding applied to every matrix-product operand (inputs, hidden
    activations, weights and biases), the products themselves exact: the reduced-precision
    training arithmetic (BF16 operands, wide accumulation)."""
    r = rnd or (lambda v: v)
    h = r(x)
    cache = []
    for i, (W, b) in enumerate(layers):
        z = h @ r(np.asarray(W, np.float64)).T + r(np.asarray(b, np.float64))
        cache.append((h, z))
        h = r(_act(z, kind)) if i + 1 < len(layers) else sigmoid(z)
    return h, cache


def mlp_backward(layers, cache, y, g_y, kind, rnd=None):
    """Returns (g_x, [(gW, gb), ...]). With rnd, every matrix-product operand of the backward
    (the deltas, the weights and the cached layer inputs) is rounded, and the activation
    derivative is taken from the rounded activation; the forward may have run on exact
    operands (a cached input the forward rounded already is unchanged by rounding again)."""
    grads = [None] * len(layers)
    r = rnd or (lambda v: v)
    g = r(g_y * y * (1.0 - y))                                # through the sigmoid
    for i in range(len(layers) - 1, -1, -1):
        W = r(np.asarray(layers[i][0], np.float64))
        h = r(cache[i][0])
        grads[i] = (g.T @ h, g.sum(axis=0))
        g_h = g @ W
        if i > 0:
            if rnd is None:
                g = g_h * _act_grad(cache[i - 1][1], kind)
            else:
                g = r(g_h * _act_grad_from_out(h, kind))
        else:
            g = g_h
    return g, grads


# ----------------------------------------------------------------------------
# QAT (Sec. 2.3, Sec. 3.3)
# ----------------------------------------------------------------------------

def _round_half_away(x):
    """C round(): nearest integer, halves away from zero (exact in the input's precision)."""
    x = np.asarray(x)
    t = np.trunc(x)
    frac = x - t                                   # exact for |x| < 2^23 (FP32) / 2^52 (FP64)
    return t + np.where(np.abs(frac) >= 0.5, np.sign(x), 0).astype(x.dtype)


def qat_scale_zero(level, bits, dtype=np.float64):
    """Per-level scale s and zero point z. dtype float32 reproduces the kernels' decision."""
    lv = np.asarray(level, dtype)
    a = min(dtype(0), lv.min())
    b = max(dtype(0), lv.max())
    if b - a == 0:
        return dtype(1), dtype(0)
    s = dtype(b - a) / dtype(2 ** bits - 1)
    z = _round_half_away(dtype(-a) / s).astype(dtype)
    return dtype(s), dtype(z)


def qat_quantize(level, s, z, bits, dtype=np.float64):
    """Eq. quantize: q = clamp(round(r / s) + z, 0, 2^b - 1)."""
    lv = np.asarray(level, dtype)
    q = _round_half_away(lv / dtype(s)) + dtype(z)
    return np.clip(q, 0, 2 ** bits - 1)


def qat_fake_quant(level, bits):
    """Eq. quantizer Q(w) = s (q - z) and the straight-through mask (1 where unclamped)."""
    s, z = qat_scale_zero(level, bits)
    raw = _round_half_away(np.asarray(level, np.float64) / s) + z
    q = np.clip(raw, 0, 2 ** bits - 1)
    mask = ((raw >= 0) & (raw <= 2 ** bits - 1)).astype(np.float64)
    return s * (q - z), mask


def export_grid(levels, bits):
    """Stored form of the grids: integer codes per level plus (s, z), decided in FP32."""
    codes, scales, zeros = [], [], []
    for g in levels:
        s, z = qat_scale_zero(g, bits, np.float32)
        codes.append(qat_quantize(g, s, z, bits, np.float32).astype(np.uint8))
        scales.append(float(s))
        zeros.append(float(z))
    return codes, np.array(scales, np.float32), np.array(zeros, np.float32)


def dequantize_grid(codes, scales, zeros):
    """Eq. dequantize r = s (q - z), per level (FP64)."""
    return [float(s) * (c.astype(np.float64) - float(z)) for c, s, z in zip(codes, scales, zeros)]


# ----------------------------------------------------------------------------
# FP8 E4M3 weights with per-layer power-of-two scales (weight-precision study;
# the paper stores FP16 MLP weights, Sec. 3.4)
# ----------------------------------------------------------------------------

E4M3_MAX = 448.0          # 1.75 * 2^8: largest finite E4M3 value (exponent bias 7, 3 mantissa bits)
E4M3_MIN_NORMAL = 2.0 ** -6


def e4m3_round(x):
    """Nearest FP8 E4M3 value, ties to even mantissa, saturating at +-448.

    E4M3 has 1 sign bit, 4 exponent bits (bias 7) and 3 mantissa bits, subnormals
    below 2^-6 with spacing 2^-9, and no infinities. In the binade [2^k, 2^(k+1))
    the spacing is 2^(k-3); np.round is half-to-even, so a tie lands on the
    neighbour with the even mantissa."""
    x = np.asarray(x, np.float64)
    a = np.minimum(np.abs(x), E4M3_MAX)
    _, ex = np.frexp(np.maximum(a, E4M3_MIN_NORMAL))      # a = m 2^ex, m in [0.5, 1)
    step = np.ldexp(1.0, ex - 1 - 3)                      # 2^(floor(log2 a) - 3)
    q = np.minimum(np.round(a / step) * step, E4M3_MAX)
    return np.where(x < 0, -q, q)


def e4m3_code(v):
    """Bit pattern (uint8) of an exactly representable E4M3 value v."""
    v = np.asarray(v, np.float64)
    a = np.abs(v)
    sign = np.signbit(v).astype(np.int64) << 7          # a negative value that rounds to zero keeps its sign
    _, ex = np.frexp(np.maximum(a, E4M3_MIN_NORMAL))
    normal = a >= E4M3_MIN_NORMAL
    efield = np.where(normal, ex - 1 + 7, 0)
    mant = np.where(normal, a / np.ldexp(1.0, ex - 1) - 1.0, a / 2.0 ** -6) * 8.0
    assert np.all(mant == np.round(mant)), "value not representable in E4M3"
    return (sign | (efield << 3) | mant.astype(np.int64)).astype(np.uint8)


def fp8_layer_exponent(values):
    """Per-layer scale 2^e: the smallest integer e with max|w| <= 448 * 2^e (e = 0 for an
    all-zero layer). Compared exactly (powers of two scale exactly)."""
    m = float(np.max(np.abs(np.asarray(values, np.float64)))) if np.size(values) else 0.0
    if m == 0.0:
        return 0
    e = math.frexp(m)[1] - 1 - 8
    while m > math.ldexp(E4M3_MAX, e):
        e += 1
    while m <= math.ldexp(E4M3_MAX, e - 1):
        e -= 1
    return e


def fp8_params(params):
    """MLP weights as the FP8 export holds them: per layer (W, b share one scale 2^e),
    w -> e4m3_round(w / 2^e) 2^e. Returns (params with the quantised MLPs, exponents in
    the order colour layers then endpoint layers, codes per layer as (W codes, b codes))."""
    out = dict(color_grid=params["color_grid"], endpoint_grid=params["endpoint_grid"])
    exps, codes = [], []
    for k in ("color_mlp", "endpoint_mlp"):
        layers = []
        for W, b in params[k]:
            W = np.asarray(W, np.float64)
            b = np.asarray(b, np.float64)
            e = fp8_layer_exponent(np.concatenate([W.ravel(), b.ravel()]))
            qW, qb = e4m3_round(np.ldexp(W, -e)), e4m3_round(np.ldexp(b, -e))
            layers.append((np.ldexp(qW, e), np.ldexp(qb, e)))
            exps.append(e)
            codes.append((e4m3_code(qW), e4m3_code(qb)))
        out[k] = layers
    return out, exps, codes


# FP8 arithmetic (an extension for the precision study, like the FP8 weights): activations
# in E4M3 too. Layer l's input x (the grid features for l = 0, the previous layer's
# activation otherwise) is rounded to E4M3 at the layer's scale 2^e_l,
# x -> e4m3_round(x 2^-e_l) 2^e_l; the weights are the FP8 ones (fp8_params); products and
# sums are exact and the bias is added exactly. The exponents come from a calibration
# sample of the material: FP8_CALIB_BLOCKS blocks at ids i * FP8_CALIB_STRIDE mod n_blocks
# (distinct for i < n_blocks, the stride being a prime above any block count), the endpoint
# network on their centres and the colour network on their 16 texel centres, in the
# network with the FP8 weights and exact activations; e_l is the smallest integer with
# 2 max|x_l| <= 448 2^e_l over the sample (one binade of headroom above the sampled maximum,
# for inputs outside the sample).

FP8_CALIB_BLOCKS = 2048
FP8_CALIB_STRIDE = 2654435761          # prime


def mlp_forward_fp8(layers, x, kind, act_exps):
    """Outputs of an MLP in the FP8 arithmetic: act_exps[l] is layer l's input exponent."""
    h = np.asarray(x, np.float64)
    for i, (W, b) in enumerate(layers):
        e = int(act_exps[i])
        hq = np.ldexp(e4m3_round(np.ldexp(h, -e)), e)
        z = hq @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        h = _act(z, kind) if i + 1 < len(layers) else sigmoid(z)
    return h


def fp8_calibration_ids(n_blocks, count=FP8_CALIB_BLOCKS):
    """Block ids of the calibration sample (int64)."""
    k = min(int(n_blocks), int(count))
    return (np.arange(k, dtype=np.int64) * FP8_CALIB_STRIDE) % int(n_blocks)


def fp8_activation_exponents(desc, params, color_grid=None, endpoint_grid=None):
    """Activation exponents of the FP8 arithmetic, colour layers then endpoint layers.
    params: the parameters with the FP8 weights (fp8_params); grids: the ones inference
    reads (dequantised exported grids), defaulting to the parameter grids."""
    ids = fp8_calibration_ids(desc.n_blocks)
    s, t = block_coords(desc.blocks_x, desc.blocks_y, ids % desc.blocks_x, ids // desc.blocks_x)
    xs, ys = block_texel_xy(desc, ids)
    u, v = texel_coords(desc.width, desc.height, xs.ravel(), ys.ravel())
    cg = color_grid if color_grid is not None else params["color_grid"]
    eg = endpoint_grid if endpoint_grid is not None else params["endpoint_grid"]
    exps = []
    for key, grid, (a, b) in (("color_mlp", cg, (u, v)), ("endpoint_mlp", eg, (s, t))):
        x, _ = grid_lookup(_as64(grid), a, b)
        _, cache = mlp_forward(params[key], x, desc.activation)
        exps += [fp8_layer_exponent(2.0 * h) for h, _ in cache]
    return exps


# ----------------------------------------------------------------------------
# forward over a material
# ----------------------------------------------------------------------------

def _as64(levels):
    return [np.asarray(g, np.float64) for g in levels]


def _net_forward(desc, layers, x, act_exps):
    if act_exps is None:
        return mlp_forward(layers, x, desc.activation)[0]
    return mlp_forward_fp8(layers, x, desc.activation, act_exps)


def endpoint_forward(desc, params, bxs, bys, grid=None, act_exps=None):
    s, t = block_coords(desc.blocks_x, desc.blocks_y, bxs, bys)
    levels = _as64(grid if grid is not None else params["endpoint_grid"])
    x, _ = grid_lookup(levels, s, t)
    return _net_forward(desc, params["endpoint_mlp"], x, act_exps)


def color_forward(desc, params, xs, ys, grid=None, act_exps=None):
    u, v = texel_coords(desc.width, desc.height, xs, ys)
    levels = _as64(grid if grid is not None else params["color_grid"])
    x, _ = grid_lookup(levels, u, v)
    return _net_forward(desc, params["color_mlp"], x, act_exps)


def block_texel_xy(desc, block_ids):
    """Texel coordinates of the 16 texels of each block: ([nb, 16], [nb, 16])."""
    block_ids = np.asarray(block_ids, np.int64)
    bx = block_ids % desc.blocks_x
    by = block_ids // desc.blocks_x
    i = np.arange(16)
    return 4 * bx[:, None] + (i % 4)[None, :], 4 * by[:, None] + (i // 4)[None, :]


def forward_blocks(desc, params, block_ids, color_grid=None, endpoint_grid=None, fp8_act=None):
    """Network outputs for the given blocks: e_hat [nb, out_e], c_hat [nb, 16, out_c] (FP64).
    fp8_act: activation exponents (colour layers, then endpoint layers) of the FP8
    arithmetic, or None for exact activations."""
    block_ids = np.asarray(block_ids, np.int64)
    nc = len(params["color_mlp"])
    ce, ee = (None, None) if fp8_act is None else (list(fp8_act[:nc]), list(fp8_act[nc:]))
    e_hat = endpoint_forward(desc, params, block_ids % desc.blocks_x, block_ids // desc.blocks_x, endpoint_grid, ee)
    xs, ys = block_texel_xy(desc, block_ids)
    c_hat = color_forward(desc, params, xs.ravel(), ys.ravel(), color_grid, ce)
    return e_hat, c_hat.reshape(len(block_ids), 16, desc.out_color)


# ----------------------------------------------------------------------------
# inference to blocks (Sec. 3.2, Fig. NTBC (a)); decisions in FP32
# ----------------------------------------------------------------------------

def _f32(x):
    return np.asarray(x, np.float32)


def quantize_endpoints_bc1(e):
    """e [n, 3] float32 in [0, 1] -> RGB565 integer fields, floor(e*31+0.5) (G: 63), FP32."""
    e = _f32(e)
    r = np.clip(np.floor(e[:, 0] * np.float32(31) + np.float32(0.5)), 0, 31).astype(np.int64)
    g = np.clip(np.floor(e[:, 1] * np.float32(63) + np.float32(0.5)), 0, 63).astype(np.int64)
    b = np.clip(np.floor(e[:, 2] * np.float32(31) + np.float32(0.5)), 0, 31).astype(np.int64)
    return _bc.pack565(r, g, b)


def quantize_endpoints_u8(e):
    e = _f32(e)
    return np.clip(np.floor(e * np.float32(255) + np.float32(0.5)), 0, 255).astype(np.int64)


def _sqdist_f32(c, pal):
    """Squared distances in FP32, channels summed in order: c [n,16,C], pal [n,K,C] -> [n,16,K]."""
    c = _f32(c)
    pal = _f32(pal)
    acc = None
    for ch in range(c.shape[-1]):
        d = c[:, :, None, ch] - pal[:, None, :, ch]
        sq = d * d
        acc = sq if acc is None else acc + sq
    return acc


def outputs_to_blocks(fmt, e_hat, c_hat):
    """Steps a6-a8: quantise predicted endpoints, order / mode, integer palette, argmax of
    -||c_hat - p_n|| over hardware codes (first = lowest code), pack.
    e_hat [n, 2C], c_hat [n, 16, C]; both cast to FP32 first. Returns [n, 8] uint8."""
    e = _f32(e_hat)
    c = _f32(c_hat)
    f255 = np.float32(255)
    if fmt == BC1:
        c0 = quantize_endpoints_bc1(e[:, 0:3])
        c1 = quantize_endpoints_bc1(e[:, 3:6])
        swap = c0 < c1
        c0, c1 = np.where(swap, c1, c0), np.where(swap, c0, c1)
        pal = _bc.bc1_palette(c0, c1).astype(np.float32) / f255          # n x 4 x 3
        codes = np.argmin(_sqdist_f32(c, pal), axis=-1)
        codes = np.where((c0 == c1)[:, None], 0, codes)
        return _bc.bc1_pack(c0, c1, codes)
    r0 = quantize_endpoints_u8(e[:, 0])
    r1 = quantize_endpoints_u8(e[:, 1])
    pal = _bc.bc4_palette(r0, r1).astype(np.float32) / f255              # n x 8
    codes = np.argmin(_sqdist_f32(c, pal[..., None]), axis=-1)
    return _bc.bc4_pack(r0, r1, codes)


def infer_blocks(desc, params, block_ids=None, color_grid=None, endpoint_grid=None, fp8_act=None):
    """NTBC inference to BC blocks for every texture: list of [nb, 8] uint8 (row-major blocks)."""
    if block_ids is None:
        block_ids = np.arange(desc.n_blocks)
    e_hat, c_hat = forward_blocks(desc, params, block_ids, color_grid, endpoint_grid, fp8_act)
    out = []
    for t, fmt in enumerate(desc.formats):
        ch = desc.channels[t]
        eo, co = desc.endpoint_offsets()[t], desc.color_offsets()[t]
        out.append(outputs_to_blocks(fmt, e_hat[:, eo:eo + 2 * ch], c_hat[:, :, co:co + ch]))
    return out


# ----------------------------------------------------------------------------
# training losses with the straight-through argmax (Sec. 3.2, App. A)
# ----------------------------------------------------------------------------

def palette_linear(fmt, e0, e1):
    """Float palette in the paper's linear order n. e0, e1 [..., C].
    Returns (P [..., K, C], a [..., K], b [..., K]) with P_n = a_n e0 + b_n e1 + const_n
    (a_n, b_n are the derivatives of P_n by e0 and e1)."""
    e0 = np.asarray(e0, np.float64)
    e1 = np.asarray(e1, np.float64)
    if fmt == BC1:
        w = np.arange(4) / 3.0
        a = np.broadcast_to(1.0 - w, e0.shape[:-1] + (4,)).copy()
        b = np.broadcast_to(w, e0.shape[:-1] + (4,)).copy()
        const = np.zeros_like(a)
    else:
        eight = (e0[..., 0] > e1[..., 0])[..., None]
        w8 = np.arange(8) / 7.0
        w6 = np.array([0.0, 0.0, 0.2, 0.4, 0.6, 0.8, 1.0, 0.0])
        interp6 = np.array([0.0, 1, 1, 1, 1, 1, 1, 0.0])
        a = np.where(eight, 1.0 - w8, (1.0 - w6) * interp6)
        b = np.where(eight, w8, w6 * interp6)
        const = np.where(eight, 0.0, np.array([0.0, 0, 0, 0, 0, 0, 0, 1.0]))
    P = a[..., None] * e0[..., None, :] + b[..., None] * e1[..., None, :] + const[..., None]
    return P, a, b


def softmax(x, axis=-1):
    m = x.max(axis=axis, keepdims=True)
    e = np.exp(x - m)
    return e / e.sum(axis=axis, keepdims=True)


def _ste_dec(d, P, T, soft):
    """Forward decode: hard one-hot of argmax d (or the softmax expectation when soft)."""
    P = np.broadcast_to(P, d.shape + (P.shape[-1],))
    sig = softmax(d / T)
    if soft:
        dec = np.einsum("...k,...kc->...c", sig, P)
    else:
        n = np.argmax(d, axis=-1)
        dec = np.take_along_axis(P, n[..., None, None].repeat(P.shape[-1], -1), axis=-2)[..., 0, :]
    return dec, sig


def _ste_grad_d(g_dec, sig, P, T):
    """d loss / d d_j = (1/T) sigma_j sum_c g_dec_c (P_jc - sum_i sigma_i P_ic)."""
    pbar = np.einsum("...k,...kc->...c", sig, P)
    return (1.0 / T) * sig * np.einsum("...c,...kc->...k", g_dec, P - pbar[..., None, :])


def _dist(a, P):
    diff = a[..., None, :] - P
    nrm = np.sqrt((diff * diff).sum(axis=-1))
    return -nrm, diff, np.maximum(nrm, NORM_GUARD)


def losses_and_grads(desc, params, textures, ref_blocks, block_ids, T=0.01, qat_bits=0, soft=False, bf16=False):
    """One training step's losses and gradients (FP64) for a batch of whole blocks.

    textures: list of uint8 arrays (H x W x 3 or H x W); ref_blocks: list of [nblocks, 8].
    soft=True evaluates the surrogate in which the forward decode is the softmax
    expectation itself (the backward is then that surrogate's exact gradient).
    bf16=True takes the tensor-core training arithmetic: the colour MLP's matrix-product operands
    rounded to BF16 in the forward and the backward; the endpoint MLP's forward on exact operands
    (its outputs steer the straight-through softmax, which amplifies an output error 1/T; the
    kernel splits each forward operand into BF16 hi + lo parts, ~2^-16 relative) and its backward
    on BF16 operands.
    Returns (losses dict, grads dict shaped like params).
    """
    block_ids = np.asarray(block_ids, np.int64)
    nb = len(block_ids)
    C_out, E_out = desc.out_color, desc.out_endpoint
    eoffs, coffs = desc.endpoint_offsets(), desc.color_offsets()

    def grids(key):
        lv = _as64(params[key])
        if qat_bits:
            fq = [qat_fake_quant(g, qat_bits) for g in lv]
            return [f[0] for f in fq], [f[1] for f in fq]
        return lv, None

    # ---- reference data for the batch
    xs, ys = block_texel_xy(desc, block_ids)
    c_ref = np.zeros((nb, 16, C_out))
    e_ref = np.zeros((nb, E_out))
    for t, fmt in enumerate(desc.formats):
        tex = np.asarray(textures[t])
        ch = desc.channels[t]
        if ch == 1:
            c_ref[:, :, coffs[t]] = tex[ys, xs] / 255.0
        else:
            c_ref[:, :, coffs[t]:coffs[t] + 3] = tex[ys, xs, :] / 255.0
        e_ref[:, eoffs[t]:eoffs[t] + 2 * ch] = _bc.reference_endpoints(fmt, np.asarray(ref_blocks[t])[block_ids])

    # ---- endpoint network
    eg, emask = grids("endpoint_grid")
    s, tt = block_coords(desc.blocks_x, desc.blocks_y, block_ids % desc.blocks_x, block_ids // desc.blocks_x)
    xe, ecache_g = grid_lookup(eg, s, tt)
    rnd = bf16_round if bf16 else None
    e_hat, ecache = mlp_forward(params["endpoint_mlp"], xe, desc.activation)
    L_e = np.mean((e_hat - e_ref) ** 2)
    g_e = 2.0 * (e_hat - e_ref) / e_hat.size
    n_cd = nb * 16 * C_out
    L_cd_e = 0.0
    for t, fmt in enumerate(desc.formats):
        ch = desc.channels[t]
        eo, co = eoffs[t], coffs[t]
        ehat0, ehat1 = e_hat[:, eo:eo + ch], e_hat[:, eo + ch:eo + 2 * ch]
        pe, a_n, b_n = palette_linear(fmt, ehat0, ehat1)                 # nb x K x C
        pr, _, _ = palette_linear(fmt, e_ref[:, eo:eo + ch], e_ref[:, eo + ch:eo + 2 * ch])
        c = c_ref[:, :, co:co + ch]                                      # nb x 16 x C
        d, diff, nrm = _dist(c, pe[:, None])                             # diff = c - p_n
        dec, sig = _ste_dec(d, pr[:, None], T, soft)
        L_cd_e += ((c - dec) ** 2).sum() / n_cd
        g_dec = -2.0 * (c - dec) / n_cd
        g_d = _ste_grad_d(g_dec, sig, pr[:, None], T)                     # nb x 16 x K
        g_p = g_d[..., None] * diff / nrm[..., None]                     # d d_n / d p_n = (c - p_n)/||.||
        g_e[:, eo:eo + ch] += np.einsum("bikc,bk->bc", g_p, a_n)
        g_e[:, eo + ch:eo + 2 * ch] += np.einsum("bikc,bk->bc", g_p, b_n)
    g_xe, g_emlp = mlp_backward(params["endpoint_mlp"], ecache, e_hat, g_e, desc.activation, rnd)
    g_egrid = grid_lookup_backward(eg, ecache_g, g_xe, emask)

    # ---- colour network
    cg, cmask = grids("color_grid")
    u, v = texel_coords(desc.width, desc.height, xs.ravel(), ys.ravel())
    xc, ccache_g = grid_lookup(cg, u, v)
    c_flat, ccache = mlp_forward(params["color_mlp"], xc, desc.activation, rnd)
    c_hat = c_flat.reshape(nb, 16, C_out)
    L_c = np.mean((c_hat - c_ref) ** 2)
    g_c = 2.0 * (c_hat - c_ref) / c_hat.size
    L_cd_c = 0.0
    for t, fmt in enumerate(desc.formats):
        ch = desc.channels[t]
        eo, co = eoffs[t], coffs[t]
        pr, _, _ = palette_linear(fmt, e_ref[:, eo:eo + ch], e_ref[:, eo + ch:eo + 2 * ch])
        chat = c_hat[:, :, co:co + ch]
        c = c_ref[:, :, co:co + ch]
        d, diff, nrm = _dist(chat, pr[:, None])                          # diff = c_hat - P_n
        dec, sig = _ste_dec(d, pr[:, None], T, soft)
        L_cd_c += ((c - dec) ** 2).sum() / n_cd
        g_dec = -2.0 * (c - dec) / n_cd
        g_d = _ste_grad_d(g_dec, sig, pr[:, None], T)
        g_c[:, :, co:co + ch] += np.einsum("bik,bikc->bic", g_d, -diff / nrm[..., None])
    g_xc, g_cmlp = mlp_backward(params["color_mlp"], ccache, c_flat, g_c.reshape(nb * 16, C_out), desc.activation,
                                rnd)
    g_cgrid = grid_lookup_backward(cg, ccache_g, g_xc, cmask)

    losses = dict(L_e=L_e, L_cd_endpoint=L_cd_e, L_c=L_c, L_cd_color=L_cd_c,
                  L_endpoint=L_e + L_cd_e, L_color=L_c + L_cd_c)
    grads = dict(color_grid=g_cgrid, endpoint_grid=g_egrid, color_mlp=g_cmlp, endpoint_mlp=g_emlp)
    return losses, grads


def outputs_vjp(desc, params, block_ids, g_e, g_c, qat_bits=0):
    """Vector-Jacobian product of the raw outputs: with f = sum g_e . e_hat + sum g_c . c_hat
    (e_hat [nb, out_e], c_hat [nb, 16, out_c] as forward_blocks returns them), the gradient
    of f w.r.t. every parameter, through the same backward the losses use (sigmoid, MLP,
    bilinear scatter, and with qat_bits the fake-quantised grids and straight-through mask).
    Returns (e_hat, c_hat, grads shaped like params)."""
    block_ids = np.asarray(block_ids, np.int64)
    nb = len(block_ids)

    def grids(key):
        lv = _as64(params[key])
        if qat_bits:
            fq = [qat_fake_quant(g, qat_bits) for g in lv]
            return [f[0] for f in fq], [f[1] for f in fq]
        return lv, None

    eg, emask = grids("endpoint_grid")
    s, t = block_coords(desc.blocks_x, desc.blocks_y, block_ids % desc.blocks_x, block_ids // desc.blocks_x)
    xe, ecache_g = grid_lookup(eg, s, t)
    e_hat, ecache = mlp_forward(params["endpoint_mlp"], xe, desc.activation)
    g_xe, g_emlp = mlp_backward(params["endpoint_mlp"], ecache, e_hat, np.asarray(g_e, np.float64), desc.activation)
    g_egrid = grid_lookup_backward(eg, ecache_g, g_xe, emask)

    cg, cmask = grids("color_grid")
    xs, ys = block_texel_xy(desc, block_ids)
    u, v = texel_coords(desc.width, desc.height, xs.ravel(), ys.ravel())
    xc, ccache_g = grid_lookup(cg, u, v)
    c_flat, ccache = mlp_forward(params["color_mlp"], xc, desc.activation)
    g_xc, g_cmlp = mlp_backward(params["color_mlp"], ccache, c_flat,
                                np.asarray(g_c, np.float64).reshape(nb * 16, desc.out_color), desc.activation)
    g_cgrid = grid_lookup_backward(cg, ccache_g, g_xc, cmask)
    grads = dict(color_grid=g_cgrid, endpoint_grid=g_egrid, color_mlp=g_cmlp, endpoint_mlp=g_emlp)
    return e_hat, c_flat.reshape(nb, 16, desc.out_color), grads


def loss_value(desc, params, textures, ref_blocks, block_ids, T=0.01, qat_bits=0, soft=False):
    """L_endpoint + L_color (the two networks share no parameters, so their sum's gradient
    is each network's own gradient)."""
    losses, _ = losses_and_grads(desc, params, textures, ref_blocks, block_ids, T, qat_bits, soft)
    return losses["L_endpoint"] + losses["L_color"]


# ----------------------------------------------------------------------------
# Adam and the learning-rate schedule (Sec. 3.4)
# ----------------------------------------------------------------------------

ADAM_BETA1, ADAM_BETA2, ADAM_EPS = 0.9, 0.999, 1e-15


def learning_rate(step, total_steps, lr_max, warmup=10):
    """Linear warm-up over `warmup` steps, then cosine annealing to 0 at the last step."""
    if step < warmup:
        return lr_max * (step + 1) / warmup
    span = max(total_steps - warmup, 1)
    return lr_max * 0.5 * (1.0 + math.cos(math.pi * (step - warmup) / span))


def adam_update(p, g, m, v, step, lr):
    """One Adam step with bias correction (step counts from 0). Returns (p, m, v)."""
    m = ADAM_BETA1 * m + (1 - ADAM_BETA1) * g
    v = ADAM_BETA2 * v + (1 - ADAM_BETA2) * g * g
    mh = m / (1 - ADAM_BETA1 ** (step + 1))
    vh = v / (1 - ADAM_BETA2 ** (step + 1))
    return p - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v


def flatten_params(params):
    """Canonical order of every parameter tensor: colour grid levels, endpoint grid levels,
    colour MLP (W, b per layer), endpoint MLP."""
    out = list(params["color_grid"]) + list(params["endpoint_grid"])
    for key in ("color_mlp", "endpoint_mlp"):
        for W, b in params[key]:
            out += [W, b]
    return out


def unflatten_like(params, flat):
    it = iter(flat)
    out = dict(color_grid=[next(it) for _ in params["color_grid"]],
               endpoint_grid=[next(it) for _ in params["endpoint_grid"]])
    for key in ("color_mlp", "endpoint_mlp"):
        out[key] = [(next(it), next(it)) for _ in params[key]]
    return out


def params_from_flat(desc, flat):
    """Parameters from one flat vector in the order of the C ABI's parameter layout: colour-
    grid levels ([res][res][F] each, row = y), endpoint-grid levels, colour MLP (W [out][in]
    then b [out] per layer), endpoint MLP. Sizes come from `desc`; the vector must be consumed
    exactly. Arrays are float64 views of the values."""
    flat = np.asarray(flat)
    off = 0

    def take(shape):
        nonlocal off
        n = int(np.prod(shape))
        if off + n > flat.size:
            raise ValueError("flat parameter vector too short for this model")
        a = flat[off:off + n].astype(np.float64).reshape(shape)
        off += n
        return a

    out = dict(color_grid=[take((r, r, desc.features)) for r in desc.color_res],
               endpoint_grid=[take((r, r, desc.features)) for r in desc.endpoint_res])
    for which in ("color", "endpoint"):
        dims = desc.mlp_dims(which)
        out[which + "_mlp"] = [(take((dims[l + 1], dims[l])), take((dims[l + 1],))) for l in range(len(dims) - 1)]
    if off != flat.size:
        raise ValueError(f"flat parameter vector has {flat.size} values, the model {off}")
    return out


def is_grid_index(params, i):
    return i < len(params["color_grid"]) + len(params["endpoint_grid"])


@dataclass
class TrainConfig:
    steps: int = 500
    batch_texels: int = 4096
    qat_fraction: float = 0.0          # > 0: extra ceil(fraction * steps) QAT steps
    grid_bits: int = 8
    lr_grid: float = 0.01
    lr_mlp: float = 0.005
    temperature: float = 0.01
    warmup: int = 10
    seed: int = 0

    @property
    def qat_steps(self):
        return int(math.ceil(self.qat_fraction * self.steps)) if self.qat_fraction > 0 else 0

    @property
    def total_steps(self):
        return self.steps + self.qat_steps


def train(desc, params, textures, ref_blocks, cfg: TrainConfig, sampler):
    """Full training loop (small materials only). sampler(step) -> block ids of that step."""
    flat = [np.asarray(x, np.float64).copy() for x in flatten_params(params)]
    m = [np.zeros_like(x) for x in flat]
    v = [np.zeros_like(x) for x in flat]
    history = []
    for step in range(cfg.total_steps):
        cur = unflatten_like(params, flat)
        qbits = cfg.grid_bits if step >= cfg.steps and cfg.qat_steps else 0
        losses, grads = losses_and_grads(desc, cur, textures, ref_blocks, sampler(step),
                                         cfg.temperature, qbits)
        gflat = flatten_params(grads)
        for i in range(len(flat)):
            lr = learning_rate(step, cfg.total_steps, cfg.lr_grid if is_grid_index(params, i) else cfg.lr_mlp, cfg.warmup)
            flat[i], m[i], v[i] = adam_update(flat[i], gflat[i], m[i], v[i], step, lr)
        history.append(losses)
    return unflatten_like(params, flat), history
