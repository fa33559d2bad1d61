"""Oracle: BC1 / BC4 block codec and reference encoder (plain numpy, integer + FP64).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this module.

Format facts (Sec. 2.1): a 4x4 texel block is 8 bytes in both formats.
  * BC1: two RGB565 endpoints and sixteen 2-bit indices; four-colour palette
    with two colours interpolated at 1/3 and 2/3 (Eq. palette, w_n = n/3).
  * BC4: two 8-bit endpoints and sixteen 3-bit indices; if e0 > e1 six values
    are interpolated (w_n = n/7), otherwise four, plus the constants 0 and 1
    (Eq. palette and Eq. weightBC4).
The paper gives only the field widths; the bit layout below is the standard
Direct3D one, and the interpolants round to nearest:
  * blocks are stored in row-major block order; texel i of a block is 4*y + x;
  * BC1: bytes 0-1 colour0 (little-endian u16: R5 bits 15..11, G6 10..5,
    B5 4..0), bytes 2-3 colour1, bytes 4-7 a little-endian u32 whose bits
    2i..2i+1 hold texel i's code;
  * BC4: byte 0 r0, byte 1 r1, bytes 2-7 a little-endian 48-bit field whose
    bits 3i..3i+2 hold texel i's code;
  * 5->8 bit expansion (x << 3) | (x >> 2), 6->8 bit (x << 2) | (x >> 4);
  * BC1 colour0 > colour1: code2 = (2c0 + c1 + 1) // 3, code3 = (c0 + 2c1 + 1) // 3;
    otherwise (3-colour mode, decode only) code2 = (c0 + c1 + 1) // 2, code3 = 0;
  * BC4 r0 > r1: code k+1 = ((7-k) r0 + k r1 + 3) // 7, k = 1..6;
    otherwise code k+1 = ((5-k) r0 + k r1 + 2) // 5, k = 1..4, code6 = 0, code7 = 255.

The paper's palette index n runs in linear order of the weight w_n; the
hardware code differs. LINEAR_TO_CODE_* give the map.

Reference encoder (stands in for the Compressonator encoder of Sec. 4.1; this
is our own range fit with exhaustive index assignment, no refinement):
  BC1: integer mean/covariance -> principal axis by 8 power iterations in FP64
       (explicit operation order, no fused multiply-add) -> the texels with the
       extreme projections become the endpoints -> RGB565 by (x*31+127)//255,
       (x*63+127)//255 -> each texel takes the code of least integer squared
       RGB distance (ties: lowest code) -> colour0 > colour1 by swapping
       (codes 0<->1, 2<->3); colour0 == colour1 gives all codes 0.
  BC4: candidate A is the 8-value mode with r0 = max, r1 = min; candidate B is
       the 6-value mode spanning the texels other than 0 and 255 (0..255 if
       there are none); each takes per-texel least |difference| codes (ties:
       lowest code), the smaller total squared error wins (ties: A); a solid
       block gives r0 = r1 = value and all codes 0.
"""
from __future__ import annotations

import numpy as np

BC1 = 1
BC4 = 4
# Compositions (Sec. 2.1: BC2, BC3 and BC5 combine BC1 and BC4), 16-byte blocks:
#   BC3 (RGBA8 texels): bytes 0-7 the alpha channel as a BC4 block, bytes 8-15 the colour as
#       a BC1 block that always decodes with the four-colour palette;
#   BC5 (two-channel texels): bytes 0-7 channel 0 as a BC4 block, bytes 8-15 channel 1.
BC3 = 3
BC5 = 5

# paper's linear index n (increasing weight w_n) -> hardware code
LINEAR_TO_CODE_BC1 = np.array([0, 2, 3, 1])
LINEAR_TO_CODE_BC4_8 = np.array([0, 2, 3, 4, 5, 6, 7, 1])          # e0 > e1
LINEAR_TO_CODE_BC4_6 = np.array([6, 0, 2, 3, 4, 5, 1, 7])          # e0 <= e1: n=0 -> 0.0, n=7 -> 1.0


def channels(fmt):
    if fmt == BC1:
        return 3
    if fmt == BC4:
        return 1
    if fmt == BC3:
        return 4
    if fmt == BC5:
        return 2
    raise ValueError(f"unsupported format {fmt}")


def block_bytes(w, h):
    """Size of one compressed texture: (w/4)*(h/4) blocks of 8 bytes (Sec. 1)."""
    if w % 4 or h % 4 or w <= 0 or h <= 0:
        raise ValueError("width and height must be positive multiples of 4")
    return (w // 4) * (h // 4) * 8


# ----------------------------------------------------------------------------
# texel <-> block layout
# ----------------------------------------------------------------------------

def to_blocks(tex, w, h):
    """H x W (x C) texels -> [nblocks, 16, C] int64, blocks row-major, texel i = 4y + x."""
    t = np.asarray(tex)
    if t.ndim == 2:
        t = t[..., None]
    c = t.shape[2]
    b = t.reshape(h // 4, 4, w // 4, 4, c).transpose(0, 2, 1, 3, 4)
    return b.reshape((h // 4) * (w // 4), 16, c).astype(np.int64)


def from_blocks(blk, w, h):
    c = blk.shape[2]
    t = blk.reshape(h // 4, w // 4, 4, 4, c).transpose(0, 2, 1, 3, 4).reshape(h, w, c)
    return t


# ----------------------------------------------------------------------------
# RGB565 and palettes
# ----------------------------------------------------------------------------

def expand565(c):
    c = np.asarray(c, dtype=np.int64)
    r5, g6, b5 = (c >> 11) & 31, (c >> 5) & 63, c & 31
    return np.stack([(r5 << 3) | (r5 >> 2), (g6 << 2) | (g6 >> 4), (b5 << 3) | (b5 >> 2)], axis=-1)


def pack565(r5, g6, b5):
    return (np.asarray(r5, np.int64) << 11) | (np.asarray(g6, np.int64) << 5) | np.asarray(b5, np.int64)


def bc1_palette(c0, c1):
    """Integer palette in hardware-code order: [..., 4, 3]."""
    c0 = np.asarray(c0, np.int64)
    c1 = np.asarray(c1, np.int64)
    e0, e1 = expand565(c0), expand565(c1)
    four = (c0 > c1)[..., None]
    p2 = np.where(four, (2 * e0 + e1 + 1) // 3, (e0 + e1 + 1) // 2)
    p3 = np.where(four, (e0 + 2 * e1 + 1) // 3, 0)
    return np.stack([e0, e1, p2, p3], axis=-2)


def bc1_palette4(c0, c1):
    """Four-colour palette whatever the endpoint order (the colour block of BC3)."""
    c0 = np.asarray(c0, np.int64)
    c1 = np.asarray(c1, np.int64)
    e0, e1 = expand565(c0), expand565(c1)
    return np.stack([e0, e1, (2 * e0 + e1 + 1) // 3, (e0 + 2 * e1 + 1) // 3], axis=-2)


def bc4_palette(r0, r1):
    """Integer palette in hardware-code order: [..., 8]."""
    r0 = np.asarray(r0, np.int64)
    r1 = np.asarray(r1, np.int64)
    eight = r0 > r1
    out = [r0, r1]
    for k in range(1, 7):
        v8 = ((7 - k) * r0 + k * r1 + 3) // 7
        if k <= 4:
            v6 = ((5 - k) * r0 + k * r1 + 2) // 5
        elif k == 5:
            v6 = np.zeros_like(r0)
        else:
            v6 = np.full_like(r0, 255)
        out.append(np.where(eight, v8, v6))
    return np.stack(out, axis=-1)


# ----------------------------------------------------------------------------
# pack / unpack
# ----------------------------------------------------------------------------

def bc1_pack(c0, c1, codes):
    """codes [n, 16] in 0..3 -> [n, 8] uint8."""
    c0 = np.asarray(c0, np.int64)
    c1 = np.asarray(c1, np.int64)
    codes = np.asarray(codes, np.int64)
    idx = np.zeros(codes.shape[0], np.int64)
    for i in range(16):
        idx |= codes[:, i] << (2 * i)
    out = np.zeros((codes.shape[0], 8), np.uint8)
    out[:, 0] = c0 & 255
    out[:, 1] = c0 >> 8
    out[:, 2] = c1 & 255
    out[:, 3] = c1 >> 8
    for k in range(4):
        out[:, 4 + k] = (idx >> (8 * k)) & 255
    return out


def bc1_unpack(blocks):
    b = np.asarray(blocks, np.int64).reshape(-1, 8)
    c0 = b[:, 0] | (b[:, 1] << 8)
    c1 = b[:, 2] | (b[:, 3] << 8)
    idx = b[:, 4] | (b[:, 5] << 8) | (b[:, 6] << 16) | (b[:, 7] << 24)
    codes = np.stack([(idx >> (2 * i)) & 3 for i in range(16)], axis=1)
    return c0, c1, codes


def bc4_pack(r0, r1, codes):
    r0 = np.asarray(r0, np.int64)
    r1 = np.asarray(r1, np.int64)
    codes = np.asarray(codes, np.int64)
    idx = np.zeros(codes.shape[0], np.int64)
    for i in range(16):
        idx |= codes[:, i] << (3 * i)
    out = np.zeros((codes.shape[0], 8), np.uint8)
    out[:, 0] = r0
    out[:, 1] = r1
    for k in range(6):
        out[:, 2 + k] = (idx >> (8 * k)) & 255
    return out


def bc4_unpack(blocks):
    b = np.asarray(blocks, np.int64).reshape(-1, 8)
    idx = np.zeros(b.shape[0], np.int64)
    for k in range(6):
        idx |= b[:, 2 + k] << (8 * k)
    codes = np.stack([(idx >> (3 * i)) & 7 for i in range(16)], axis=1)
    return b[:, 0], b[:, 1], codes


# ----------------------------------------------------------------------------
# decode (ground truth for every PSNR)
# ----------------------------------------------------------------------------

def decode(fmt, blocks, w, h):
    """Compressed blocks -> H x W x 3 (BC1), H x W (BC4), H x W x 4 (BC3), H x W x 2 (BC5) uint8."""
    if fmt in (BC3, BC5):
        b16 = np.asarray(blocks, np.uint8).reshape(-1, 16)
        first = decode(BC4, b16[:, :8], w, h)
        if fmt == BC5:
            return np.stack([first, decode(BC4, b16[:, 8:], w, h)], axis=-1)
        c0, c1, codes = bc1_unpack(b16[:, 8:])
        pal = bc1_palette4(c0, c1)
        rgb = from_blocks(np.take_along_axis(pal, codes[..., None].repeat(3, -1), axis=1), w, h).astype(np.uint8)
        return np.concatenate([rgb, first[..., None]], axis=-1)
    blocks = np.asarray(blocks, np.uint8).reshape(-1, 8)
    if blocks.shape[0] != (w // 4) * (h // 4):
        raise ValueError("block count does not match the texture size")
    if fmt == BC1:
        c0, c1, codes = bc1_unpack(blocks)
        pal = bc1_palette(c0, c1)                                    # n x 4 x 3
        tex = np.take_along_axis(pal, codes[..., None].repeat(3, -1), axis=1)
        return from_blocks(tex, w, h).astype(np.uint8)
    if fmt == BC4:
        r0, r1, codes = bc4_unpack(blocks)
        pal = bc4_palette(r0, r1)                                    # n x 8
        tex = np.take_along_axis(pal, codes, axis=1)[..., None]
        return from_blocks(tex, w, h)[..., 0].astype(np.uint8)
    raise ValueError(f"unsupported format {fmt}")


# ----------------------------------------------------------------------------
# reference encoder
# ----------------------------------------------------------------------------

POWER_ITERATIONS = 8


def _bc1_endpoints(x):
    """x: [n, 16, 3] int64 -> indices (imax, imin) of the extreme texels along the principal axis."""
    n = x.shape[0]
    s = x.sum(axis=1)                                                # n x 3
    d = 16 * x - s[:, None, :]                                       # n x 16 x 3 (16 * deviation)
    cov = np.empty((n, 3, 3), dtype=np.int64)
    for j in range(3):
        for k in range(3):
            cov[:, j, k] = (d[:, :, j] * d[:, :, k]).sum(axis=1)
    C = cov.astype(np.float64)
    rng_ = (x.max(axis=1) - x.min(axis=1)).astype(np.float64)       # n x 3
    widest = np.argmax(rng_, axis=1)                                  # first max
    v0 = rng_.copy()
    for c in range(3):
        flip = (widest != c) & (cov[np.arange(n), widest, c] < 0)
        v0[:, c] = np.where(flip, -v0[:, c], v0[:, c])
    v = v0.copy()
    live = np.ones(n, dtype=bool)
    for _ in range(POWER_ITERATIONS):
        w_ = np.empty_like(v)
        for j in range(3):
            w_[:, j] = (C[:, j, 0] * v[:, 0] + C[:, j, 1] * v[:, 1]) + C[:, j, 2] * v[:, 2]
        m = np.maximum(np.maximum(np.abs(w_[:, 0]), np.abs(w_[:, 1])), np.abs(w_[:, 2]))
        live = live & (m > 0.0)
        safe = np.where(live, m, 1.0)
        for j in range(3):
            v[:, j] = np.where(live, w_[:, j] / safe, v[:, j])
    xf = x.astype(np.float64)
    proj = (xf[:, :, 0] * v[:, None, 0] + xf[:, :, 1] * v[:, None, 1]) + xf[:, :, 2] * v[:, None, 2]
    return np.argmax(proj, axis=1), np.argmin(proj, axis=1)


def bc1_encode_blocks(x):
    """x: [n, 16, 3] int RGB8 -> [n, 8] uint8 BC1 blocks."""
    x = np.asarray(x, np.int64)
    n = x.shape[0]
    imax, imin = _bc1_endpoints(x)
    hi = x[np.arange(n), imax]
    lo = x[np.arange(n), imin]

    def q565(p):
        return pack565((p[:, 0] * 31 + 127) // 255, (p[:, 1] * 63 + 127) // 255, (p[:, 2] * 31 + 127) // 255)

    c0, c1 = q565(hi), q565(lo)
    swap = c0 < c1
    c0, c1 = np.where(swap, c1, c0), np.where(swap, c0, c1)
    pal = bc1_palette(c0, c1)                                        # n x 4 x 3
    diff = x[:, :, None, :] - pal[:, None, :, :]                     # n x 16 x 4 x 3
    err = (diff * diff).sum(axis=-1)                                 # n x 16 x 4
    codes = np.argmin(err, axis=-1)                                  # first min = lowest code
    codes = np.where((c0 == c1)[:, None], 0, codes)
    return bc1_pack(c0, c1, codes)


def _bc4_codes(x, r0, r1):
    pal = bc4_palette(r0, r1)                                        # n x 8
    err = np.abs(x[:, :, None] - pal[:, None, :])                    # n x 16 x 8
    codes = np.argmin(err, axis=-1)
    sel = np.take_along_axis(pal, codes, axis=1)
    sse = ((x - sel) ** 2).sum(axis=1)
    return codes, sse


def bc4_encode_blocks(x):
    """x: [n, 16] int R8 -> [n, 8] uint8 BC4 blocks."""
    x = np.asarray(x, np.int64).reshape(-1, 16)
    mx, mn = x.max(axis=1), x.min(axis=1)
    codes_a, sse_a = _bc4_codes(x, mx, mn)
    inner = (x != 0) & (x != 255)
    has = inner.any(axis=1)
    lo = np.where(has, np.where(inner, x, 256).min(axis=1), 0)
    hi = np.where(has, np.where(inner, x, -1).max(axis=1), 255)
    codes_b, sse_b = _bc4_codes(x, lo, hi)
    use_a = sse_a <= sse_b
    r0 = np.where(use_a, mx, lo)
    r1 = np.where(use_a, mn, hi)
    codes = np.where(use_a[:, None], codes_a, codes_b)
    solid = mx == mn
    r0 = np.where(solid, mx, r0)
    r1 = np.where(solid, mx, r1)
    codes = np.where(solid[:, None], 0, codes)
    return bc4_pack(r0, r1, codes)


# ----------------------------------------------------------------------------
# optional refinement of the reference encoder (the "refine steps" Sec. 4.1 mentions for
# Compressonator, whose definition the paper does not give; reading: least-squares
# endpoints for the current codes, re-quantised, codes re-chosen, kept while the block's
# squared error strictly falls, at most `iterations` times). All integer arithmetic.
# ----------------------------------------------------------------------------

BC1_CODE_W3 = np.array([0, 3, 1, 2])                    # code -> weight of e1, in thirds
BC4_8_CODE_W7 = np.array([0, 7, 1, 2, 3, 4, 5, 6])       # r0 > r1: code -> weight of r1, in sevenths
BC4_6_CODE_W5 = np.array([0, 5, 1, 2, 3, 4, -1, -1])     # r0 <= r1: in fifths; codes 6, 7 are 0 and 255


def ls_endpoints(x, wts, D, use):
    """Least-squares endpoints for fixed codes: minimise sum_i |x_i - ((D - w_i) a + w_i b) / D|^2
    over the texels with use_i. x [n, 16, C] int, wts [n, 16] weights in units of 1/D.
    With A11 = sum (D-w)^2, A12 = sum (D-w) w, A22 = sum w^2, R1 = sum (D-w) x, R2 = sum w x
    (normal equations times D^2): a = D (A22 R1 - A12 R2) / det, b = D (A11 R2 - A12 R1) / det,
    det = A11 A22 - A12^2. Returns the integer numerators [n, C] of a and b (without the
    factor D) and det [n]."""
    x = np.asarray(x, np.int64)
    w = np.where(use, np.asarray(wts, np.int64), 0)
    u = np.where(use, D - w, 0)
    A11, A12, A22 = (u * u).sum(1), (u * w).sum(1), (w * w).sum(1)
    R1 = (u[..., None] * x).sum(1)
    R2 = (w[..., None] * x).sum(1)
    det = A11 * A22 - A12 * A12
    return A22[:, None] * R1 - A12[:, None] * R2, A11[:, None] * R2 - A12[:, None] * R1, det


def quantise_ls(num, det, D, L):
    """round-half-up(D num / det * L / 255) clamped to [0, L] (exact integer arithmetic,
    det > 0; a non-positive numerator gives 0)."""
    num = np.asarray(num, np.int64)
    d = np.maximum(det, 1)[..., None] if num.ndim > np.ndim(det) else np.maximum(det, 1)
    q = (2 * D * num * L + 255 * d) // (510 * d)
    return np.where(num <= 0, 0, np.minimum(q, L))


def bc1_sse(x, c0, c1, codes):
    pal = bc1_palette(c0, c1)
    sel = np.take_along_axis(pal, np.asarray(codes, np.int64)[..., None].repeat(3, -1), axis=1)
    return ((np.asarray(x, np.int64) - sel) ** 2).sum(axis=(1, 2))


def bc1_refine(x, blocks, iterations):
    """x [n, 16, 3] RGB8, blocks [n, 8] -> refined [n, 8]."""
    x = np.asarray(x, np.int64)
    c0, c1, codes = bc1_unpack(blocks)
    sse = bc1_sse(x, c0, c1, codes)
    for _ in range(iterations):
        wts = BC1_CODE_W3[codes]
        na, nb, det = ls_endpoints(x, wts, 3, np.ones_like(codes, bool))
        ok = det > 0
        lv = np.array([31, 63, 31])
        qa = np.stack([quantise_ls(na[:, c], det, 3, lv[c]) for c in range(3)], 1)
        qb = np.stack([quantise_ls(nb[:, c], det, 3, lv[c]) for c in range(3)], 1)
        a0, a1 = pack565(qa[:, 0], qa[:, 1], qa[:, 2]), pack565(qb[:, 0], qb[:, 1], qb[:, 2])
        n0, n1 = np.maximum(a0, a1), np.minimum(a0, a1)
        pal = bc1_palette(n0, n1)
        err = ((x[:, :, None, :] - pal[:, None, :, :]) ** 2).sum(-1)
        ncodes = np.where((n0 == n1)[:, None], 0, np.argmin(err, -1))
        nsse = bc1_sse(x, n0, n1, ncodes)
        better = ok & (nsse < sse)
        c0, c1 = np.where(better, n0, c0), np.where(better, n1, c1)
        codes = np.where(better[:, None], ncodes, codes)
        sse = np.where(better, nsse, sse)
    return bc1_pack(c0, c1, codes)


def bc4_refine(x, blocks, iterations):
    """x [n, 16] R8, blocks [n, 8] -> refined [n, 8] (the block's mode is kept)."""
    x = np.asarray(x, np.int64)
    r0, r1, codes = bc4_unpack(blocks)
    sse = ((x - np.take_along_axis(bc4_palette(r0, r1), codes, axis=1)) ** 2).sum(1)
    for _ in range(iterations):
        eight = r0 > r1
        D = np.where(eight, 7, 5)
        wts = np.where(eight[:, None], BC4_8_CODE_W7[codes], BC4_6_CODE_W5[codes])
        use = wts >= 0
        na8, nb8, det8 = ls_endpoints(x[..., None], wts, 7, use)
        na6, nb6, det6 = ls_endpoints(x[..., None], wts, 5, use)
        na, nb, det = np.where(eight[:, None], na8, na6)[:, 0], np.where(eight[:, None], nb8, nb6)[:, 0], \
            np.where(eight, det8, det6)
        qa = np.where(eight, quantise_ls(na, det, 7, 255), quantise_ls(na, det, 5, 255))
        qb = np.where(eight, quantise_ls(nb, det, 7, 255), quantise_ls(nb, det, 5, 255))
        # keep the mode: r0 > r1 for eight values, r0 <= r1 for six
        n0 = np.where(eight, np.maximum(qa, qb), np.minimum(qa, qb))
        n1 = np.where(eight, np.minimum(qa, qb), np.maximum(qa, qb))
        ok = (det > 0) & np.where(eight, n0 > n1, True)
        pal = bc4_palette(n0, n1)
        ncodes = np.argmin(np.abs(x[:, :, None] - pal[:, None, :]), -1)
        nsse = ((x - np.take_along_axis(pal, ncodes, axis=1)) ** 2).sum(1)
        better = ok & (nsse < sse)
        r0, r1 = np.where(better, n0, r0), np.where(better, n1, r1)
        codes = np.where(better[:, None], ncodes, codes)
        sse = np.where(better, nsse, sse)
    return bc4_pack(r0, r1, codes)


def encode_refined(fmt, tex, w, h, iterations=2):
    """The reference encoder followed by `iterations` least-squares refinement steps."""
    blk = to_blocks(tex, w, h)
    if fmt == BC1:
        return bc1_refine(blk, bc1_encode_blocks(blk), iterations)
    if fmt == BC4:
        return bc4_refine(blk[..., 0], bc4_encode_blocks(blk[..., 0]), iterations)
    raise ValueError(f"unsupported format {fmt}")


def encode(fmt, tex, w, h):
    """Reference BC encode of a whole texture -> [(w/4)*(h/4), 8] uint8 (BC1, BC4) or
    [(w/4)*(h/4), 16] (BC3: alpha by the BC4 encoder, colour by the BC1 encoder, whose
    blocks already have colour0 >= colour1; BC5: one BC4 block per channel)."""
    if fmt == BC3:
        t = np.asarray(tex)
        return np.concatenate([encode(BC4, t[..., 3], w, h), encode(BC1, t[..., :3], w, h)], axis=1)
    if fmt == BC5:
        t = np.asarray(tex)
        return np.concatenate([encode(BC4, t[..., 0], w, h), encode(BC4, t[..., 1], w, h)], axis=1)
    blk = to_blocks(tex, w, h)
    if fmt == BC1:
        return bc1_encode_blocks(blk)
    if fmt == BC4:
        return bc4_encode_blocks(blk[..., 0])
    raise ValueError(f"unsupported format {fmt}")


def reference_endpoints(fmt, blocks):
    """Decoded endpoints of stored blocks in [0, 1], in stored order: BC1 [n, 6], BC4 [n, 2].
    These are the endpoint targets e0, e1 of Eq. lossNTBC_e."""
    if fmt == BC1:
        c0, c1, _ = bc1_unpack(blocks)
        return np.concatenate([expand565(c0), expand565(c1)], axis=1).astype(np.float64) / 255.0
    r0, r1, _ = bc4_unpack(blocks)
    return np.stack([r0, r1], axis=1).astype(np.float64) / 255.0


# ----------------------------------------------------------------------------
# metric (Sec. 4.3)
# ----------------------------------------------------------------------------

def psnr(a, b):
    """PSNR over all channels of one texture, values in [0, 1]: 10 log10(1 / MSE)."""
    a = np.asarray(a, np.float64) / 255.0
    b = np.asarray(b, np.float64) / 255.0
    mse = np.mean((a - b) ** 2)
    return float("inf") if mse == 0 else float(10.0 * np.log10(1.0 / mse))
