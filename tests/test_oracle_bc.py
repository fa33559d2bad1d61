"""Pins of the oracle's BC1 / BC4 codec and reference encoder (CPU only).

Each test checks the oracle against something other than itself: the paper's
block size, hand-derived blocks, exact rational arithmetic for the palette
rounding, exhaustive round trips and brute force over codes / endpoint pairs.
"""
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import bc
from conftest import golden

RNG = np.random.default_rng(1234)


def test_block_size_matches_paper():
    # Sec. 1: BC1 and BC4 compress each 4x4 block to 8 bytes; a 4k texture needs 8 MB.
    g = golden("paper_numbers.txt")
    assert bc.block_bytes(4096, 4096) == int(g["bc_texture_4k_bytes"][0])
    tex = np.zeros((8, 12, 3), np.uint8)
    assert bc.encode(bc.BC1, tex, 12, 8).shape == (6, 8)
    with pytest.raises(ValueError):
        bc.block_bytes(10, 8)


def test_expansion_tracks_exact_rescale():
    # bit replication: within 1 of x * 255 / (2^k - 1), strictly increasing, 0 -> 0, max -> 255
    for bits, shift, ch in ((5, 11, 0), (6, 5, 1), (5, 0, 2)):
        vals = [int(bc.expand565(x << shift)[ch]) for x in range(2 ** bits)]
        for x, got in enumerate(vals):
            assert abs(Fraction(got) - Fraction(x * 255, 2 ** bits - 1)) < 1
        assert vals[0] == 0 and vals[-1] == 255 and all(b > a for a, b in zip(vals, vals[1:]))


def test_bc4_palette_exhaustive_rounding():
    # every interpolant of every endpoint pair is the nearest integer to the exact
    # weighted mean (Eq. palette with w_n = n/7 or n/5), endpoints sit at codes 0/1,
    # and the 6-value mode carries the constants 0 and 255 (Eq. weightBC4).
    r0, r1 = np.meshgrid(np.arange(256), np.arange(256), indexing="ij")
    r0, r1 = r0.ravel(), r1.ravel()
    pal = bc.bc4_palette(r0, r1)
    assert (pal[:, 0] == r0).all() and (pal[:, 1] == r1).all()
    eight = r0 > r1
    for k in range(1, 7):
        num8 = (7 - k) * r0 + k * r1
        assert (np.abs(7 * pal[eight, k + 1] - num8[eight]) <= 3).all()
    for k in range(1, 5):
        num6 = (5 - k) * r0 + k * r1
        assert (np.abs(5 * pal[~eight, k + 1] - num6[~eight]) <= 2).all()
    assert (pal[~eight, 6] == 0).all() and (pal[~eight, 7] == 255).all()


def test_bc4_exhaustive_roundtrip():
    # decode(pack(r0, r1, codes)) reproduces the palette entry of each code, for all
    # 65536 endpoint pairs and all 8 codes; unpack(pack(x)) == x.
    r0, r1 = np.meshgrid(np.arange(256), np.arange(256), indexing="ij")
    r0, r1 = r0.ravel(), r1.ravel()
    pal = bc.bc4_palette(r0, r1)
    for shift in range(8):
        codes = (np.arange(16)[None, :] + shift + r0[:, None]) % 8
        blocks = bc.bc4_pack(r0, r1, codes)
        u0, u1, uc = bc.bc4_unpack(blocks)
        assert (u0 == r0).all() and (u1 == r1).all() and (uc == codes).all()
        w = 4 * len(r0)
        tex = bc.decode(bc.BC4, blocks, w, 4)
        dec_blocks = bc.to_blocks(tex, w, 4)[..., 0]
        assert (dec_blocks == np.take_along_axis(pal, codes, axis=1)).all()


def test_bc1_palette_rounding_and_roundtrip():
    n = 1_000_000
    c0 = RNG.integers(0, 65536, n)
    c1 = RNG.integers(0, 65536, n)
    pal = bc.bc1_palette(c0, c1)
    e0, e1 = bc.expand565(c0), bc.expand565(c1)
    four = c0 > c1
    assert (pal[:, 0] == e0).all() and (pal[:, 1] == e1).all()
    assert (np.abs(3 * pal[four, 2] - (2 * e0[four] + e1[four])) <= 1).all()
    assert (np.abs(3 * pal[four, 3] - (e0[four] + 2 * e1[four])) <= 1).all()
    half = 2 * pal[~four, 2] - (e0[~four] + e1[~four])
    assert ((half == 0) | (half == 1)).all()
    assert (pal[~four, 3] == 0).all()
    codes = RNG.integers(0, 4, (n, 16))
    blocks = bc.bc1_pack(c0, c1, codes)
    u0, u1, uc = bc.bc1_unpack(blocks)
    assert (u0 == c0).all() and (u1 == c1).all() and (uc == codes).all()
    sub = slice(0, 20000)
    w = 4 * 20000
    tex = bc.decode(bc.BC1, blocks[sub], w, 4)
    dec = bc.to_blocks(tex, w, 4)
    want = np.take_along_axis(pal[sub], codes[sub][..., None].repeat(3, -1), axis=1)
    assert (dec == want).all()


def _parse_texels(s, ch):
    vals = [int(t, 16) for t in s.split(",")]
    if ch == 3:
        return np.array([[(v >> 16) & 255, (v >> 8) & 255, v & 255] for v in vals], np.uint8)
    return np.array(vals, np.uint8)


@pytest.mark.parametrize("name", ["bc1_checker", "bc1_solid_red", "bc4_checker", "bc4_solid"])
def test_hand_derived_blocks(name):
    texels, want = golden("bc_blocks.txt")[name]
    fmt = bc.BC1 if name.startswith("bc1") else bc.BC4
    ch = bc.channels(fmt)
    px = _parse_texels(texels, ch)
    tex = px.reshape(4, 4, 3) if ch == 3 else px.reshape(4, 4)
    got = bc.encode(fmt, tex, 4, 4)[0]
    assert bytes(got).hex() == want.replace(",", "")
    assert (bc.decode(fmt, got[None], 4, 4) == tex).all()


def _brute_codes_sse(px, pal):
    """Pure-Python exhaustive per-texel choice: minimal squared error over all codes."""
    total = 0
    for p in px:
        best = None
        for entry in pal:
            e = sum((int(a) - int(b)) ** 2 for a, b in zip(np.atleast_1d(p), np.atleast_1d(entry)))
            best = e if best is None else min(best, e)
        total += best
    return total


@pytest.mark.parametrize("fmt", [bc.BC1, bc.BC4])
def test_reference_indices_are_optimal_for_chosen_endpoints(fmt):
    n = 300
    tex = synth.random_blocks_texels(n, fmt, seed=7)
    blocks = bc.encode(fmt, tex, 4 * n, 4)
    dec = bc.to_blocks(bc.decode(fmt, blocks, 4 * n, 4), 4 * n, 4)
    src = bc.to_blocks(tex, 4 * n, 4)
    for b in range(n):
        if fmt == bc.BC1:
            c0, c1, _ = bc.bc1_unpack(blocks[b:b + 1])
            pal = bc.bc1_palette(c0, c1)[0]
            if c0[0] == c1[0]:
                pal = pal[:1]
        else:
            r0, r1, _ = bc.bc4_unpack(blocks[b:b + 1])
            pal = bc.bc4_palette(r0, r1)[0]
        sse = int(((src[b] - dec[b]) ** 2).sum())
        assert sse == _brute_codes_sse(src[b], pal)


def test_bc4_reference_vs_all_endpoint_pairs():
    # brute force over all 65536 (r0, r1) pairs with exhaustive codes: the reference is
    # never better than the optimum (sanity of the brute force) and equals it on blocks
    # with at most two distinct values
    n = 60
    tex = synth.random_blocks_texels(n, bc.BC4, seed=11)
    src = bc.to_blocks(tex, 4 * n, 4)[..., 0]
    blocks = bc.encode(bc.BC4, tex, 4 * n, 4)
    dec = bc.to_blocks(bc.decode(bc.BC4, blocks, 4 * n, 4), 4 * n, 4)[..., 0]
    r0, r1 = np.meshgrid(np.arange(256), np.arange(256), indexing="ij")
    pal = bc.bc4_palette(r0.ravel(), r1.ravel())                       # 65536 x 8
    for b in range(n):
        err = (src[b][None, :, None] - pal[:, None, :]) ** 2            # 65536 x 16 x 8
        best = err.min(axis=2).sum(axis=1).min()
        ref = int(((src[b] - dec[b]) ** 2).sum())
        assert ref >= best
        if len(np.unique(src[b])) <= 2:
            assert ref == best == 0


def test_bc1_exact_on_two_representable_colours_and_solids():
    rng = np.random.default_rng(5)
    for _ in range(200):
        cols = bc.expand565(rng.integers(0, 65536, 2))                 # representable RGB8
        pick = rng.integers(0, 2, 16)
        px = cols[pick].astype(np.uint8).reshape(4, 4, 3)
        blk = bc.encode(bc.BC1, px, 4, 4)
        assert (bc.decode(bc.BC1, blk, 4, 4) == px).all()
    for _ in range(50):
        v = rng.integers(0, 256, 1)
        px = np.full((4, 4), v[0], np.uint8)
        assert (bc.decode(bc.BC4, bc.encode(bc.BC4, px, 4, 4), 4, 4) == px).all()


def test_reference_encoder_quality_on_material():
    mat = synth.tiny_material()
    for fmt, tex in zip(mat.formats, mat.textures):
        dec = bc.decode(fmt, bc.encode(fmt, tex, mat.width, mat.height), mat.width, mat.height)
        assert bc.psnr(dec, tex) > 30.0


def test_psnr_closed_form():
    a = np.full((8, 8), 100, np.uint8)
    b = a + 1
    assert bc.psnr(a, b) == pytest.approx(20 * np.log10(255.0), abs=1e-12)
    assert bc.psnr(a, a) == float("inf")


def test_linear_to_code_maps_follow_weights():
    # the paper's linear index n orders the palette by weight w_n (Eq. palette / weightBC4)
    r0, r1 = 200, 20
    pal = bc.bc4_palette(np.array([r0]), np.array([r1]))[0]
    lin = pal[bc.LINEAR_TO_CODE_BC4_8]
    assert (np.diff(lin) < 0).all() and lin[0] == r0 and lin[-1] == r1
    pal6 = bc.bc4_palette(np.array([r1]), np.array([r0]))[0]
    lin6 = pal6[bc.LINEAR_TO_CODE_BC4_6]
    assert lin6[0] == 0 and lin6[-1] == 255 and lin6[1] == r1 and lin6[6] == r0
    assert (np.diff(lin6[1:7]) > 0).all()
    c0, c1 = 0xF800, 0x001F
    p = bc.bc1_palette(np.array([c0]), np.array([c1]))[0]
    lin1 = p[bc.LINEAR_TO_CODE_BC1]
    assert (np.diff(lin1[:, 0]) < 0).all() and (np.diff(lin1[:, 2]) > 0).all()


# ----------------------------------------------------------------------------
# BC3 / BC5 (compositions of BC1 and BC4, Sec. 2.1)
# ----------------------------------------------------------------------------

def test_bc5_is_two_bc4_blocks():
    rng = np.random.default_rng(11)
    tex = rng.integers(0, 256, (16, 24, 2), dtype=np.uint8)
    blocks = bc.encode(bc.BC5, tex, 24, 16)
    assert blocks.shape == (24, 16)
    for k in range(2):
        np.testing.assert_array_equal(blocks[:, 8 * k:8 * k + 8], bc.encode(bc.BC4, tex[..., k], 24, 16))
    dec = bc.decode(bc.BC5, blocks, 24, 16)
    for k in range(2):
        np.testing.assert_array_equal(dec[..., k], bc.decode(bc.BC4, blocks[:, 8 * k:8 * k + 8], 24, 16))


def test_bc3_colour_block_decodes_in_four_colour_mode():
    # the four-colour palette is symmetric: swapping the endpoints and the codes 0<->1, 2<->3
    # gives the same texels -- which the three-colour mode (c0 <= c1 in BC1) would break
    rng = np.random.default_rng(12)
    n = 64
    c0 = rng.integers(0, 1 << 16, n)
    c1 = rng.integers(0, 1 << 16, n)
    codes = rng.integers(0, 4, (n, 16))
    alpha = bc.bc4_pack(rng.integers(0, 256, n), rng.integers(0, 256, n), rng.integers(0, 8, (n, 16)))
    swap = np.array([1, 0, 3, 2])
    a = np.concatenate([alpha, bc.bc1_pack(c0, c1, codes)], axis=1)
    b = np.concatenate([alpha, bc.bc1_pack(c1, c0, swap[codes])], axis=1)
    da, db = bc.decode(bc.BC3, a, 32, 32), bc.decode(bc.BC3, b, 32, 32)
    np.testing.assert_array_equal(da, db)
    three = (c0 <= c1) & (c0 != c1)
    assert three.any()
    # the same colour blocks read as BC1 differ wherever BC1 would use its three-colour mode
    d1 = bc.decode(bc.BC1, bc.bc1_pack(c0, c1, codes), 32, 32)
    assert not np.array_equal(d1, da[..., :3])


def test_bc3_round_trip_alpha_and_colour():
    rng = np.random.default_rng(13)
    tex = rng.integers(0, 256, (8, 8, 4), dtype=np.uint8)
    tex[..., 3] = 200                                            # solid alpha is exact
    blocks = bc.encode(bc.BC3, tex, 8, 8)
    dec = bc.decode(bc.BC3, blocks, 8, 8)
    assert np.all(dec[..., 3] == 200)
    np.testing.assert_array_equal(dec[..., :3], bc.decode(bc.BC1, blocks[:, 8:], 8, 8))


# ----------------------------------------------------------------------------
# least-squares refinement of the reference encoder
# ----------------------------------------------------------------------------

def test_least_squares_endpoints_solve_the_normal_equations():
    # exact rationals: the residual of the fitted line is orthogonal to both basis weights
    from fractions import Fraction
    rng = np.random.default_rng(21)
    x = rng.integers(0, 256, (5, 16, 3))
    w = rng.integers(0, 4, (5, 16))
    na, nb, det = bc.ls_endpoints(x, w, 3, np.ones((5, 16), bool))
    for n in range(5):
        if det[n] == 0:
            continue
        for c in range(3):
            a = Fraction(3 * int(na[n, c]), int(det[n]))
            b_ = Fraction(3 * int(nb[n, c]), int(det[n]))
            r = [Fraction(int(x[n, i, c])) - (Fraction(3 - int(w[n, i])) * a + Fraction(int(w[n, i])) * b_) / 3
                 for i in range(16)]
            assert sum(ri * (3 - int(w[n, i])) for i, ri in enumerate(r)) == 0
            assert sum(ri * int(w[n, i]) for i, ri in enumerate(r)) == 0
            # and agrees with a library least-squares solve
            A = np.stack([(3 - w[n]) / 3.0, w[n] / 3.0], 1)
            sol = np.linalg.lstsq(A, x[n, :, c].astype(float), rcond=None)[0]
            assert abs(sol[0] - float(a)) < 1e-8 and abs(sol[1] - float(b_)) < 1e-8


def test_quantise_ls_is_round_half_up_clamped():
    from fractions import Fraction
    rng = np.random.default_rng(22)
    num = rng.integers(-2000, 200000, 3000)
    det = rng.integers(1, 5000, 3000)
    for D, L in ((3, 31), (3, 63), (7, 255), (5, 255)):
        q = bc.quantise_ls(num, det, D, L)
        for k in range(0, 3000, 37):
            v = Fraction(D * int(num[k]), int(det[k])) * L / 255
            want = 0 if num[k] <= 0 else min(L, int((v + Fraction(1, 2)) // 1))
            assert q[k] == want


@pytest.mark.parametrize("fmt", [1, 4])
def test_refinement_never_increases_error(fmt):
    mat = synth.tiny_material()
    tex = mat.textures[0 if fmt == 1 else 1][:64, :64]
    base = bc.encode(fmt, tex, 64, 64)
    np.testing.assert_array_equal(bc.encode_refined(fmt, tex, 64, 64, 0), base)
    err = lambda b: ((bc.decode(fmt, b, 64, 64).astype(np.int64) - tex.astype(np.int64)) ** 2)  # noqa: E731
    e0 = err(base).reshape(16, 4, 16, 4, -1).sum(axis=(1, 3, 4))
    for k in (1, 2, 4):
        ek = err(bc.encode_refined(fmt, tex, 64, 64, k)).reshape(16, 4, 16, 4, -1).sum(axis=(1, 3, 4))
        assert np.all(ek <= e0)
        assert ek.sum() < e0.sum()
