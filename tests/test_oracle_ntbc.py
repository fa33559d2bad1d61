"""Pins of the oracle's NTBC network, losses, straight-through backward, QAT and Adam (CPU).

Pins come from outside the oracle: numbers the paper prints (model sizes, grid
shapes, hyper-parameters), closed forms (affine fields under bilinear lookup,
one Adam step, the LR schedule ends), adjoint identities, finite differences of
the surrogate loss, invariants of the quantiser, brute force over palette
entries, and the published Philox known answers.
"""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import bc, ntbc, philox
from conftest import golden

G = golden("paper_numbers.txt")


def paper_desc(n_bc1, n_bc4, side=4096):
    cres = ntbc.level_resolutions(int(G["color_levels"][0]), int(G["color_min_res"][0]), int(G["color_max_res"][0]))
    eres = ntbc.endpoint_resolutions(cres, side // 4)
    return ntbc.ModelDesc(side, side, [1] * n_bc1 + [4] * n_bc4, cres, eres)


# ----------------------------------------------------------------------------
# configuration and storage (Sec. 3.4, Sec. 4.3)
# ----------------------------------------------------------------------------

def test_level_resolutions_paper_grids():
    cres = ntbc.level_resolutions(8, 16, 2048)
    assert cres == [16 * 2 ** i for i in range(8)]
    eres = ntbc.endpoint_resolutions(cres, 1024)
    assert len(eres) == int(G["endpoint_levels"][0]) and eres[-1] == int(G["endpoint_max_res"][0])
    d = paper_desc(2, 4)
    assert d.in_color == int(G["color_input_dims"][0])
    assert d.in_endpoint == int(G["endpoint_input_dims"][0])
    # the ends of a geometric ladder are exact for other level counts too
    for L, lo, hi in ((4, 16, 128), (12, 16, 2048), (5, 7, 333)):
        r = ntbc.level_resolutions(L, lo, hi)
        assert r[0] == lo and r[-1] == hi and all(b > a for a, b in zip(r, r[1:]))


def test_storage_matches_paper_model_sizes():
    # Sec. 4.3: one aggressive model is 13.37 MB and the conservative pair 26.74 MB
    # (u8 grids, half-precision MLPs, MetalPlates013 with 2 BC1 + 4 BC4 textures).
    mib = 2 ** 20
    agg = ntbc.storage_bytes(paper_desc(2, 4), grid_bits=8, weight_bytes=2)
    cons = ntbc.storage_bytes(paper_desc(2, 0), 8, 2) + ntbc.storage_bytes(paper_desc(0, 4), 8, 2)
    assert round(agg / mib, 2) == float(G["storage_aggressive_mb"][0])
    assert round(cons / mib, 2) == float(G["storage_conservative_mb"][0])
    # the size barely depends on the texture count (Sec. 5)
    assert abs(ntbc.storage_bytes(paper_desc(1, 1), 8, 2) - agg) < 0.01 * agg


# ----------------------------------------------------------------------------
# grid lookup
# ----------------------------------------------------------------------------

def test_bilinear_reproduces_affine_fields():
    rng = np.random.default_rng(0)
    levels = []
    coef = []
    for res in (2, 5, 16, 33):
        a, b, c = rng.normal(size=3)
        iy, ix = np.meshgrid(np.arange(res), np.arange(res), indexing="ij")
        g = np.stack([a + b * ix + c * iy, -a + 2 * c * ix - b * iy], axis=-1)
        levels.append(g)
        coef.append((a, b, c, res))
    u = rng.random(1000)
    v = rng.random(1000)
    u[:3] = [0.0, 1.0, 0.5]
    v[:3] = [0.0, 1.0, 0.5]
    feats, _ = ntbc.grid_lookup(levels, u, v)
    for l, (a, b, c, res) in enumerate(coef):
        x, y = u * (res - 1), v * (res - 1)
        np.testing.assert_allclose(feats[:, 2 * l], a + b * x + c * y, atol=1e-12)
        np.testing.assert_allclose(feats[:, 2 * l + 1], -a + 2 * c * x - b * y, atol=1e-12)


def test_grid_corners_and_single_cell():
    g = np.arange(8, dtype=np.float64).reshape(2, 2, 2)
    f, _ = ntbc.grid_lookup([g], np.array([0.0, 1.0, 0.0, 1.0]), np.array([0.0, 0.0, 1.0, 1.0]))
    np.testing.assert_array_equal(f, g.reshape(4, 2))


def test_grid_backward_is_adjoint_of_lookup():
    rng = np.random.default_rng(1)
    levels = [rng.normal(size=(r, r, 2)) for r in (3, 7, 10)]
    u, v = rng.random(500), rng.random(500)
    feats, cache = ntbc.grid_lookup(levels, u, v)
    y = rng.normal(size=feats.shape)
    back = ntbc.grid_lookup_backward(levels, cache, y)
    lhs = (feats * y).sum()
    rhs = sum((g * b).sum() for g, b in zip(levels, back))
    assert lhs == pytest.approx(rhs, rel=1e-12)


# ----------------------------------------------------------------------------
# MLP pieces
# ----------------------------------------------------------------------------

def test_activations_match_library_and_closed_forms():
    z = np.linspace(-8, 8, 1001)
    np.testing.assert_allclose(ntbc.selu(z), torch.nn.functional.selu(torch.tensor(z)).numpy(), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(ntbc.sigmoid(z), torch.sigmoid(torch.tensor(z)).numpy(), rtol=1e-12)
    assert ntbc.selu(np.array([1.0]))[0] == pytest.approx(1.0507009873554805)
    assert ntbc.selu(np.array([-1e3]))[0] == pytest.approx(-1.0507009873554805 * 1.6732632423543772)
    h = 1e-6
    for z0 in (-2.0, -0.3, 0.4, 3.0):
        fd = (ntbc.selu(np.array([z0 + h])) - ntbc.selu(np.array([z0 - h])))[0] / (2 * h)
        assert ntbc.selu_grad(np.array([z0]))[0] == pytest.approx(fd, rel=1e-7)


def test_mlp_forward_matches_textbook_matmul():
    rng = np.random.default_rng(2)
    layers = [(rng.normal(size=(5, 3)), rng.normal(size=5)), (rng.normal(size=(2, 5)), rng.normal(size=2))]
    x = rng.normal(size=(7, 3))
    y, _ = ntbc.mlp_forward(layers, x, "relu")
    t = torch.tensor
    ref = torch.sigmoid(torch.relu(t(x) @ t(layers[0][0]).T + t(layers[0][1])) @ t(layers[1][0]).T + t(layers[1][1]))
    np.testing.assert_allclose(y, ref.numpy(), rtol=1e-12)


# ----------------------------------------------------------------------------
# losses and the straight-through backward (Sec. 3.2, App. A)
# ----------------------------------------------------------------------------

def _fd_setup(act, seed=3):
    mat = synth.make_material("fd", 32, ["sine_rgb", "sine_r", "sine_r", "sine_rgb"], seed)
    cres, eres = [4, 6, 9], [4, 6]
    desc = ntbc.ModelDesc(32, 32, mat.formats, cres, eres, hidden_layers=2, hidden_width=8, activation=act)
    p0 = synth.init_params(cres, eres, 2, desc.mlp_dims("color"), desc.mlp_dims("endpoint"), seed=seed)
    p = synth.random_params_like(p0, seed=seed + 1, grid_scale=0.5)
    refs = [bc.encode(f, t, 32, 32) for f, t in zip(mat.formats, mat.textures)]
    return desc, p, mat, refs


@pytest.mark.parametrize("act,T", [("selu", 1.0), ("selu", 0.05), ("relu", 1.0), ("selu", 0.01)])
def test_backward_equals_fd_of_soft_surrogate(act, T):
    desc, p, mat, refs = _fd_setup(act)
    ids = np.array([0, 5, 17, 33, 63, 40])
    _, g = ntbc.losses_and_grads(desc, p, mat.textures, refs, ids, T=T, soft=True)
    flat = [np.asarray(x, np.float64).copy() for x in ntbc.flatten_params(p)]
    gflat = ntbc.flatten_params(g)
    rng = np.random.default_rng(0)
    h = 1e-7 if T < 0.02 else 1e-6
    checked = 0
    for _ in range(40):
        i = rng.integers(len(flat))
        j = rng.integers(flat[i].size)
        fp = [x.copy() for x in flat]
        fm = [x.copy() for x in flat]
        fp[i].flat[j] += h
        fm[i].flat[j] -= h
        lp = ntbc.loss_value(desc, ntbc.unflatten_like(p, fp), mat.textures, refs, ids, T=T, soft=True)
        lm = ntbc.loss_value(desc, ntbc.unflatten_like(p, fm), mat.textures, refs, ids, T=T, soft=True)
        fd = (lp - lm) / (2 * h)
        an = np.asarray(gflat[i]).flat[j]
        if abs(fd) + abs(an) > 1e-7:
            assert an == pytest.approx(fd, rel=2e-4, abs=1e-9)
            checked += 1
    assert checked >= 10


def test_hard_forward_loss_is_direct_evaluation():
    # the hard forward decodes with the argmax entry of the reference palette
    desc, p, mat, refs = _fd_setup("selu")
    ids = np.arange(64)
    losses, _ = ntbc.losses_and_grads(desc, p, mat.textures, refs, ids)
    e_hat, c_hat = ntbc.forward_blocks(desc, p, ids)
    xs, ys = ntbc.block_texel_xy(desc, ids)
    total = 0.0
    for t, fmt in enumerate(desc.formats):
        tex = mat.textures[t].astype(np.float64) / 255.0
        c = tex[ys, xs] if tex.ndim == 2 else tex[ys, xs, :]
        c = c.reshape(64, 16, -1)
        eref = bc.reference_endpoints(fmt, refs[t][ids])
        ch = c.shape[-1]
        for b in range(64):
            pal, _, _ = ntbc.palette_linear(fmt, eref[b:b + 1, :ch], eref[b:b + 1, ch:])
            for i in range(16):
                d = [-np.linalg.norm(c_hat[b, i, desc.color_offsets()[t]:desc.color_offsets()[t] + ch] - pal[0, n])
                     for n in range(pal.shape[1])]
                n = int(np.argmax(d))
                total += ((c[b, i] - pal[0, n]) ** 2).sum()
    assert losses["L_cd_color"] == pytest.approx(total / (64 * 16 * desc.out_color), rel=1e-12)


def test_expected_weight_derivative_appendix_a():
    # App. A: w_hat = sum_i w_i sigma(d_i) with w_i = i/3; its derivative is
    # (1/T) sigma_n (w_n - w_hat). The appendix's final line prints (n - w_hat),
    # which is 3x too large in the index units its own derivation lines use.
    rng = np.random.default_rng(4)
    T = 0.3
    w = np.arange(4) / 3.0
    for _ in range(20):
        d = rng.normal(size=4)
        sig = ntbc.softmax(d / T)
        w_hat = (w * sig).sum()
        for n in range(4):
            e = np.zeros(4)
            e[n] = 1e-7
            fd = ((w * ntbc.softmax((d + e) / T)).sum() - (w * ntbc.softmax((d - e) / T)).sum()) / 2e-7
            assert fd == pytest.approx(sig[n] * (w[n] - w_hat) / T, rel=1e-6, abs=1e-9)


def test_ste_single_texel_hand_case():
    # one BC1 texel, uniform softmax (T -> large): d loss/d d_j = (1/T) (1/4) g . (P_j - mean P)
    P = np.array([[0.0, 0.0, 0.0], [1 / 3, 1 / 3, 1 / 3], [2 / 3, 2 / 3, 2 / 3], [1.0, 1.0, 1.0]])
    g = np.array([1.0, 2.0, 3.0])
    T = 1e6
    sig = np.full(4, 0.25)
    got = ntbc._ste_grad_d(g, sig, P, T)
    want = np.array([(g * (P[j] - P.mean(axis=0))).sum() * 0.25 / T for j in range(4)])
    np.testing.assert_allclose(got, want, rtol=1e-12)


# ----------------------------------------------------------------------------
# QAT (Sec. 2.3, Sec. 3.3)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("bits", [8, 4])
def test_quantizer_invariants(bits):
    rng = np.random.default_rng(6)
    lv = rng.uniform(-0.3, 0.7, (17, 17, 2))
    q, mask = ntbc.qat_fake_quant(lv, bits)
    s, z = ntbc.qat_scale_zero(lv, bits)
    assert np.all(mask == 1)
    assert np.max(np.abs(q - lv)) <= s / 2 + 1e-15                     # error at most s/2 in range
    q2, _ = ntbc.qat_fake_quant(q, bits)
    np.testing.assert_allclose(q2, q, atol=1e-12)                       # idempotent
    assert len(np.unique(np.round(q / s))) <= 2 ** bits
    assert 0 <= z <= 2 ** bits - 1
    assert ntbc.qat_quantize(np.zeros(1), s, z, bits)[0] == z          # real zero is representable
    codes, scales, zeros = ntbc.export_grid([lv], bits)
    deq = ntbc.dequantize_grid(codes, scales, zeros)[0]
    assert np.max(np.abs(deq - lv)) <= scales[0] * 0.5001


def test_quantizer_step_ratio_u8_u4():
    lv = np.random.default_rng(7).normal(size=(9, 9, 2))
    s8, _ = ntbc.qat_scale_zero(lv, 8)
    s4, _ = ntbc.qat_scale_zero(lv, 4)
    assert s4 / s8 == pytest.approx(255 / 15)


def test_quantizer_rounding_is_half_away_from_zero():
    x = np.array([0.5, 1.5, 2.5, -0.5, -1.5, 0.49999997], np.float32)
    np.testing.assert_array_equal(ntbc._round_half_away(x), np.array([1, 2, 3, -1, -2, 0], np.float32))
    np.testing.assert_array_equal(ntbc._round_half_away(x.astype(np.float64)), [1, 2, 3, -1, -2, 0])


# ----------------------------------------------------------------------------
# Adam and LR schedule (Sec. 3.4)
# ----------------------------------------------------------------------------

def test_adam_closed_form_steps():
    assert (ntbc.ADAM_BETA1, ntbc.ADAM_BETA2, ntbc.ADAM_EPS) == (
        float(G["adam_beta1"][0]), float(G["adam_beta2"][0]), float(G["adam_eps"][0]))
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 0.0])
    p1, m, v = ntbc.adam_update(p, g, np.zeros(3), np.zeros(3), 0, 0.01)
    # step 1: bias-corrected m = g, v = g^2, update = lr * sign(g)
    np.testing.assert_allclose(p1, p - 0.01 * np.sign(g), rtol=1e-12)
    # a second step with the same gradient moves by lr again
    p2, _, _ = ntbc.adam_update(p1, g, m, v, 1, 0.01)
    np.testing.assert_allclose(p2, p - 0.02 * np.sign(g), rtol=1e-12)
    # minimising (p - 3)^2 from 0 converges near 3
    x, m, v = np.array([0.0]), np.zeros(1), np.zeros(1)
    for t in range(2000):
        x, m, v = ntbc.adam_update(x, 2 * (x - 3.0), m, v, t, 0.05)
    assert abs(x[0] - 3.0) < 1e-2


def test_learning_rate_schedule():
    lr, S = 0.01, 1000
    assert ntbc.learning_rate(0, S, lr) == pytest.approx(lr / 10)
    assert ntbc.learning_rate(9, S, lr) == pytest.approx(lr)
    assert ntbc.learning_rate(10, S, lr) == pytest.approx(lr)
    assert ntbc.learning_rate(10 + (S - 10) // 2, S, lr) == pytest.approx(lr / 2)
    assert ntbc.learning_rate(S, S, lr) == pytest.approx(0.0, abs=1e-18)
    last = ntbc.learning_rate(S - 1, S, lr)
    assert 0 < last < lr * 1e-4
    vals = [ntbc.learning_rate(t, S, lr) for t in range(10, S)]
    assert all(b <= a for a, b in zip(vals, vals[1:]))


# ----------------------------------------------------------------------------
# inference decisions (Sec. 3.2): exact palette hits, brute-force argmax, ordering
# ----------------------------------------------------------------------------

def test_exact_palette_colour_is_chosen():
    rng = np.random.default_rng(8)
    n = 500
    e = rng.random((n, 6)).astype(np.float32)
    blocks = ntbc.outputs_to_blocks(1, e, np.zeros((n, 16, 3), np.float32))
    c0, c1, _ = bc.bc1_unpack(blocks)
    assert (c0 >= c1).all()
    pal = bc.bc1_palette(c0, c1)
    pick = rng.integers(0, 4, (n, 16))
    c = np.take_along_axis(pal, pick[..., None].repeat(3, -1), axis=1).astype(np.float32) / np.float32(255)
    out = ntbc.outputs_to_blocks(1, e, c)
    dec = bc.to_blocks(bc.decode(1, out, 4 * n, 4), 4 * n, 4)
    want = np.take_along_axis(pal, pick[..., None].repeat(3, -1), axis=1)
    four = c0 > c1
    assert (dec[four] == want[four]).all()
    _, _, codes = bc.bc1_unpack(out)
    assert (codes[~four] == 0).all()


def test_argmax_brute_force_bc4():
    rng = np.random.default_rng(9)
    n = 200
    e = rng.random((n, 2)).astype(np.float32)
    c = rng.random((n, 16, 1)).astype(np.float32)
    out = ntbc.outputs_to_blocks(4, e, c)
    r0, r1, codes = bc.bc4_unpack(out)
    for b in range(n):
        assert r0[b] == min(255, max(0, math.floor(float(np.float32(e[b, 0]) * np.float32(255)) + 0.5)))
        pal = bc.bc4_palette(np.array([r0[b]]), np.array([r1[b]]))[0]
        for i in range(16):
            d = [float((np.float32(c[b, i, 0]) - np.float32(p) / np.float32(255)) ** 2) for p in pal]
            assert codes[b, i] == d.index(min(d))


# ----------------------------------------------------------------------------
# Philox batch sampler
# ----------------------------------------------------------------------------

def test_philox_known_answers():
    for name, vals in golden("philox_kat.txt").items():
        words = [int(x, 16) for x in vals]
        out = philox.philox4x32(np.array(words[:4], np.uint64)[None], np.array(words[4:6], np.uint64)[None])[0]
        assert [int(x) for x in out] == words[6:10], name


def test_sampler_range_and_uniformity():
    ids = philox.sample_blocks(seed=5, step=3, n_samples=200_000, n_blocks=1000)
    assert ids.min() >= 0 and ids.max() < 1000
    counts = np.bincount(ids, minlength=1000)
    chi2 = ((counts - 200.0) ** 2 / 200.0).sum()
    assert chi2 < 1000 + 5 * math.sqrt(2000)
    assert not np.array_equal(ids[:100], philox.sample_blocks(5, 4, 100, 1000))
    np.testing.assert_array_equal(ids[:100], philox.sample_blocks(5, 3, 100, 1000))


# ----------------------------------------------------------------------------
# the learned part: training improves on the untrained network (Sec. 4.3 ordering)
# ----------------------------------------------------------------------------

def test_training_beats_untrained_and_stays_below_reference():
    mat = synth.make_material("train", 64, ["sine_rgb", "sine_r"], 0)
    cres = ntbc.level_resolutions(3, 8, 32)
    eres = ntbc.endpoint_resolutions(cres, 16)
    desc = ntbc.ModelDesc(64, 64, mat.formats, cres, eres, hidden_layers=2, hidden_width=32, activation="relu")
    p0 = synth.init_params(cres, eres, 2, desc.mlp_dims("color"), desc.mlp_dims("endpoint"), seed=0)
    refs = [bc.encode(f, t, 64, 64) for f, t in zip(mat.formats, mat.textures)]
    cfg = ntbc.TrainConfig(steps=150, batch_texels=1024)
    nb = cfg.batch_texels // 16
    p1, hist = ntbc.train(desc, p0, mat.textures, refs, cfg,
                          lambda s: philox.sample_blocks(cfg.seed, s, nb, desc.n_blocks))
    assert hist[-1]["L_color"] < 0.5 * hist[0]["L_color"]
    for t, fmt in enumerate(desc.formats):
        ref_psnr = bc.psnr(bc.decode(fmt, refs[t], 64, 64), mat.textures[t])
        before = bc.psnr(bc.decode(fmt, ntbc.infer_blocks(desc, p0)[t], 64, 64), mat.textures[t])
        after = bc.psnr(bc.decode(fmt, ntbc.infer_blocks(desc, p1)[t], 64, 64), mat.textures[t])
        assert after > before + 3.0
        assert after < ref_psnr


# ----------------------------------------------------------------------------
# FP8 E4M3 weights (precision study)
# ----------------------------------------------------------------------------

def _e4m3_table():
    """All finite non-negative E4M3 values from the format definition: exponent field
    e (bias 7), mantissa m; e = 0 is subnormal m 2^-9; code 0x7F is NaN."""
    vals = []
    for code in range(0x7F):
        e, m = code >> 3, code & 7
        vals.append(m * 2.0 ** -9 if e == 0 else (1 + m / 8) * 2.0 ** (e - 7))
    return np.array(vals)


def test_e4m3_round_brute_force_nearest_ties_even():
    table = _e4m3_table()
    assert table.max() == 448.0 and len(np.unique(table)) == 127
    rng = np.random.default_rng(0)
    mags = np.concatenate([np.exp(rng.uniform(np.log(1e-4), np.log(600.0), 4000)),
                           (table[:-1] + table[1:]) / 2,             # every tie
                           table, [0.0, 448.0, 449.0, 464.0, 1e6]])
    x = mags * np.where(rng.random(mags.size) < 0.5, -1.0, 1.0)
    got = ntbc.e4m3_round(x)
    a = np.minimum(np.abs(x), 448.0)
    d = np.abs(a[:, None] - table[None, :])
    best = d.min(axis=1, keepdims=True)
    cand = np.where(d == best, np.arange(127)[None, :], 10 ** 6)
    # among equidistant neighbours take the even mantissa (code & 1 == 0)
    even = np.where((cand % 2 == 0) & (cand < 10 ** 6), cand, 10 ** 6).min(axis=1)
    pick = np.where(even < 10 ** 6, even, cand.min(axis=1))
    want = np.sign(x) * table[pick]
    np.testing.assert_array_equal(np.abs(got), np.abs(want))
    assert np.all(np.sign(got[got != 0]) == np.sign(x[got != 0]))


def test_e4m3_round_matches_torch_cast_in_range():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(20000) * np.exp(rng.uniform(-8, 5, 20000))
    # FP32 inputs (the weights are FP32): torch converts through FP32, which would round
    # an FP64 input twice
    x = x[np.abs(x) <= 448.0].astype(np.float32).astype(np.float64)
    want = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(ntbc.e4m3_round(x), want)


def test_e4m3_codes_round_trip():
    table = _e4m3_table()
    codes = ntbc.e4m3_code(table)
    np.testing.assert_array_equal(codes, np.arange(127, dtype=np.uint8))
    np.testing.assert_array_equal(ntbc.e4m3_code(-table), np.arange(127, dtype=np.uint8) | 0x80)
    assert ntbc.e4m3_code(ntbc.e4m3_round(-1e-5)) == 0x80                       # rounds to -0


@pytest.mark.parametrize("m", [1.0, 448.0, 448.0 * 2 ** -5, 448.0 * 2 ** 3 + 1e-9, 0.0731, 3.5e-3, 1234.5, 2.0 ** -20])
def test_fp8_layer_exponent_is_smallest(m):
    e = ntbc.fp8_layer_exponent(np.array([0.5 * m, -m, 0.0]))
    assert m <= 448.0 * 2.0 ** e and m > 448.0 * 2.0 ** (e - 1)
    assert ntbc.fp8_layer_exponent(np.zeros(4)) == 0


def test_fp8_params_error_bound():
    """Relative error of a normal E4M3 rounding is at most 2^-4; every layer's maximum
    lands in the top binade (no saturation)."""
    rng = np.random.default_rng(2)
    params = dict(color_grid=[], endpoint_grid=[],
                  color_mlp=[(rng.standard_normal((64, 24)) * 0.3, rng.standard_normal(64) * 0.01)],
                  endpoint_mlp=[(rng.standard_normal((16, 64)) * 3.0, np.zeros(16))])
    q, exps, codes = ntbc.fp8_params(params)
    for (W, b), (qW, qb), e in zip(params["color_mlp"] + params["endpoint_mlp"], q["color_mlp"] + q["endpoint_mlp"], exps):
        for v, qv in ((W, qW), (b, qb)):
            big = np.abs(v) >= 2.0 ** (e - 6)
            assert np.all(np.abs(qv - v)[big] <= 2.0 ** -4 * np.abs(v)[big])
            assert np.all(np.abs(qv - v)[~big] <= 2.0 ** (e - 10))
        assert np.max(np.abs(np.concatenate([qW.ravel(), qb.ravel()]))) <= 448.0 * 2.0 ** e


# ----------------------------------------------------------------------------
# FP8 arithmetic (E4M3 activations, precision study)
# ----------------------------------------------------------------------------

def _one(w, b):
    return [(np.array([[float(w)]]), np.array([float(b)]))]


def test_fp8_forward_rounds_inputs_to_nearest_even():
    # 1 + 1/16 lies half-way between 1 (mantissa 000) and 1.125 (001): to 1; 1 + 3/16 half-way
    # between 1.125 (001) and 1.25 (010): to 1.25; one layer w = 1, b = 0 -> sigmoid(x_q)
    y = ntbc.mlp_forward_fp8(_one(1, 0), np.array([[1.0625], [1.1875], [1.0]]), "selu", [0])
    np.testing.assert_allclose(y[:, 0], 1 / (1 + np.exp(-np.array([1.0, 1.25, 1.0]))), rtol=0, atol=1e-15)


def test_fp8_forward_applies_the_scale_and_saturates():
    # 1000 2^-2 = 250 -> 256 (spacing 16 in [128, 256)) -> 1024; 1000 2^-3 = 125 -> 128
    # (spacing 8) -> 1024; unscaled, 1000 saturates to 448; b = -1024 centres the sigmoid
    x = np.array([[1000.0]])
    assert ntbc.mlp_forward_fp8(_one(1, -1024), x, "selu", [2])[0, 0] == 0.5
    assert ntbc.mlp_forward_fp8(_one(1, -1024), x, "selu", [3])[0, 0] == 0.5
    assert ntbc.mlp_forward_fp8(_one(1, -1024), x, "selu", [0])[0, 0] < 1e-200
    # below the normal range: 2^-9 spacing at scale 1, so 3e-3 -> 2^-9 * 2 (3e-3 / 2^-9 = 1.536)
    y = ntbc.mlp_forward_fp8(_one(1, 0), np.array([[3e-3]]), "selu", [0])[0, 0]
    assert y == 1 / (1 + math.exp(-2.0 ** -8))


def test_fp8_forward_uses_each_layers_own_exponent():
    # ReLU, x = 3 -> layer 0 (w 100): h = 300 (3 2^7 = 384 is exact, e0 = -7 keeps it;
    # e0 = -8 gives 768 -> 448 -> 1.75, h = 175 -> 176 at e1 = 0, spacing 16); layer 1 rounds
    # h: 300 -> 288 at e1 = 0 or 1 (spacing 32 / 16), -> 448 2^-1 = 224 at e1 = -1
    # (saturated); b1 = -288 centres the output
    layers = [(np.array([[100.0]]), np.array([0.0])), (np.array([[1.0]]), np.array([-288.0]))]
    f = lambda e: ntbc.mlp_forward_fp8(layers, np.array([[3.0]]), "relu", e)[0, 0]
    assert f([-7, 0]) == 0.5 and f([-7, 1]) == 0.5 and f([0, 0]) == 0.5
    assert f([-7, -1]) == pytest.approx(1 / (1 + math.exp(64.0)), rel=1e-12)
    assert f([-8, 0]) == pytest.approx(1 / (1 + math.exp(288.0 - 176.0)), rel=1e-12)


def test_fp8_forward_exact_on_representable_activations():
    """A ReLU network whose inputs and activations are small integers (every integer up to 16
    is an E4M3 value) computes exactly what the exact-activation network does."""
    rng = np.random.default_rng(3)
    W0 = rng.integers(-1, 2, (8, 4)).astype(np.float64)
    W1 = rng.integers(0, 2, (3, 8)).astype(np.float64) * 0.5
    layers = [(W0, np.zeros(8)), (W1, np.array([0.25, -0.5, 0.0]))]
    x = rng.integers(0, 3, (50, 4)).astype(np.float64)
    h = np.maximum(x @ W0.T, 0.0)
    assert h.max() <= 16
    want, _ = ntbc.mlp_forward(layers, x, "relu")
    np.testing.assert_array_equal(ntbc.mlp_forward_fp8(layers, x, "relu", [0, 0]), want)


def test_fp8_forward_error_bound_against_exact_activations():
    """Forward error bound of the E4M3 input roundings, propagated with absolute values: a
    rounding of y has error <= 2^-4 |y| + 2^(e - 10) (relative half-spacing 2^-4 for normal
    values, absolute 2^-10 2^e below the normal range at scale 2^e); a layer maps input
    errors d to pre-activation errors |W| d; SELU is Lipschitz with lambda alpha, the
    sigmoid with 1/4. The FP8 outputs lie within the bound, and differ from the exact ones
    (the rounding is applied)."""
    rng = np.random.default_rng(4)
    layers = [(rng.standard_normal((64, 16)) * 0.4, rng.standard_normal(64) * 0.1),
              (rng.standard_normal((64, 64)) * 0.15, rng.standard_normal(64) * 0.1),
              (rng.standard_normal((8, 64)) * 0.15, np.zeros(8))]
    x = rng.standard_normal((500, 16))
    want, cache = ntbc.mlp_forward(layers, x, "selu")
    exps = [ntbc.fp8_layer_exponent(2.0 * h) for h, _ in cache]
    got = ntbc.mlp_forward_fp8(layers, x, "selu", exps)
    err = np.zeros_like(x)
    for l, ((W, _), (h, _)) in enumerate(zip(layers, cache)):
        rounded = err + 2.0 ** -4 * (np.abs(h) + err) + 2.0 ** (exps[l] - 10)
        zerr = rounded @ np.abs(W).T
        err = zerr * (ntbc.SELU_LAMBDA * ntbc.SELU_ALPHA if l + 1 < len(layers) else 0.25)
    d = np.abs(got - want)
    assert np.all(d <= err)
    assert d.max() > 1e-4


def test_fp8_calibration_ids():
    # 2654435761 = 7 * 379205108 + 5, so the ids for 7 blocks are 5 i mod 7; = 1 mod 10
    np.testing.assert_array_equal(ntbc.fp8_calibration_ids(7), [0, 5, 3, 1, 6, 4, 2])
    np.testing.assert_array_equal(ntbc.fp8_calibration_ids(10), np.arange(10))
    ids = ntbc.fp8_calibration_ids(1024 * 1024)
    assert ids.size == ntbc.FP8_CALIB_BLOCKS == len(np.unique(ids)) and ids.min() >= 0 and ids.max() < 1024 * 1024


def test_fp8_activation_exponents_no_sample_input_saturates():
    """With the calibrated exponents every sampled layer input sits at or below half the E4M3
    maximum after scaling, and above a quarter of it (the exponent is the smallest such)."""
    cres = [4, 8]
    desc = ntbc.ModelDesc(32, 32, [1, 4], cres, ntbc.endpoint_resolutions(cres, 8), hidden_layers=2)
    p0 = synth.init_params(cres, desc.endpoint_res, 2, desc.mlp_dims("color"), desc.mlp_dims("endpoint"), 0)
    params = ntbc.fp8_params(synth.random_params_like(p0, seed=1))[0]
    exps = ntbc.fp8_activation_exponents(desc, params)
    assert len(exps) == 6
    ids = np.arange(desc.n_blocks)                  # 64 blocks: the sample is every block
    xs, ys = ntbc.block_texel_xy(desc, ids)
    u, v = ntbc.texel_coords(32, 32, xs.ravel(), ys.ravel())
    s, t = ntbc.block_coords(8, 8, ids % 8, ids // 8)
    for k, (key, grid, a, b) in enumerate((("color_mlp", "color_grid", u, v), ("endpoint_mlp", "endpoint_grid", s, t))):
        x, _ = ntbc.grid_lookup(params[grid], a, b)
        h = x
        for l, (W, bias) in enumerate(params[key]):
            m = np.abs(h).max() * 2.0 ** -exps[3 * k + l]
            assert 112.0 < m <= 224.0, (key, l, m)
            z = h @ W.T + bias
            h = ntbc.selu(z)


# ----------------------------------------------------------------------------
# vector-Jacobian product of the raw outputs (the differentiable-function form)
# ----------------------------------------------------------------------------

def _vjp_case(seed=0, act="selu"):
    cres = [4, 7]
    desc = ntbc.ModelDesc(16, 16, [1, 4], cres, ntbc.endpoint_resolutions(cres, 4), hidden_layers=2, activation=act)
    p0 = synth.init_params(cres, desc.endpoint_res, 2, desc.mlp_dims("color"), desc.mlp_dims("endpoint"), seed)
    params = synth.random_params_like(p0, seed=seed + 1)
    rng = np.random.default_rng(seed + 2)
    ids = np.array([0, 3, 5, 15, 3])
    g_e = rng.standard_normal((len(ids), desc.out_endpoint))
    g_c = rng.standard_normal((len(ids), 16, desc.out_color))
    return desc, params, ids, g_e, g_c


@pytest.mark.parametrize("act", ["selu", "relu"])
def test_outputs_vjp_directional_finite_difference(act):
    desc, params, ids, g_e, g_c = _vjp_case(act=act)
    e, c, grads = ntbc.outputs_vjp(desc, params, ids, g_e, g_c)
    e2, c2 = ntbc.forward_blocks(desc, params, ids)
    np.testing.assert_allclose(e, e2, rtol=1e-12)
    np.testing.assert_allclose(c, c2, rtol=1e-12)
    parts = [np.asarray(a, np.float64) for a in ntbc.flatten_params(params)]
    flat = np.concatenate([a.ravel() for a in parts])
    gflat = np.concatenate([np.asarray(a, np.float64).ravel() for a in ntbc.flatten_params(grads)])
    cuts = np.cumsum([a.size for a in parts])[:-1]

    def unflat(x):
        return ntbc.unflatten_like(params, [c.reshape(a.shape) for c, a in zip(np.split(x, cuts), parts)])

    rng = np.random.default_rng(7)
    h = 1e-6
    for _ in range(4):
        d = rng.standard_normal(flat.size)

        def f(x):
            p = unflat(x)
            ee, cc = ntbc.forward_blocks(desc, p, ids)
            return float(np.sum(g_e * ee) + np.sum(g_c * cc))
        fd = (f(flat + h * d) - f(flat - h * d)) / (2 * h)
        assert abs(fd - float(gflat @ d)) <= 1e-6 * max(1.0, abs(fd))


def test_outputs_vjp_qat_is_straight_through():
    # with QAT the gradient is the float-grid gradient taken at the fake-quantised grids,
    # times the unclamped mask (Sec. 2.3: the STE passes the gradient through round())
    desc, params, ids, g_e, g_c = _vjp_case(seed=3)
    _, _, gq = ntbc.outputs_vjp(desc, params, ids, g_e, g_c, qat_bits=4)
    fq = dict(params)
    masks = {}
    for key in ("color_grid", "endpoint_grid"):
        pairs = [ntbc.qat_fake_quant(g, 4) for g in params[key]]
        fq[key] = [p[0] for p in pairs]
        masks[key] = [p[1] for p in pairs]
    _, _, gf = ntbc.outputs_vjp(desc, fq, ids, g_e, g_c)
    for key in ("color_grid", "endpoint_grid"):
        for a, b, m in zip(gq[key], gf[key], masks[key]):
            np.testing.assert_allclose(a, b * m, rtol=1e-12, atol=1e-15)
    for key in ("color_mlp", "endpoint_mlp"):
        for (aW, ab), (bW, bb) in zip(gq[key], gf[key]):
            np.testing.assert_allclose(aW, bW, rtol=1e-12)
            np.testing.assert_allclose(ab, bb, rtol=1e-12)


# ----------------------------------------------------------------------------
# BF16 operand rounding (the reduced-precision training arithmetic)
# ----------------------------------------------------------------------------

def test_bf16_round_brute_force_and_torch():
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(50000) * np.exp(rng.uniform(-40, 40, 50000))).astype(np.float32).astype(np.float64)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(ntbc.bf16_round(x), want)
    # every BF16 value in [1, 2) and the midpoints between neighbours: ties go to the even mantissa
    vals = 1.0 + np.arange(129) / 128.0
    np.testing.assert_array_equal(ntbc.bf16_round(vals), vals)
    mids = (vals[:-1] + vals[1:]) / 2
    even = np.where(np.arange(128) % 2 == 0, vals[:-1], vals[1:])
    np.testing.assert_array_equal(ntbc.bf16_round(mids), even)
    np.testing.assert_array_equal(ntbc.bf16_round(-mids), -even)


@pytest.mark.parametrize("act", ["selu", "relu"])
def test_backward_through_activation_output_equals_through_preactivation(act):
    # the BF16 mode takes act' from the activation's output; with an identity rounding it
    # must give exactly the gradients of the default (pre-activation) form
    rng = np.random.default_rng(4)
    layers = [(rng.standard_normal((16, 6)), rng.standard_normal(16)), (rng.standard_normal((16, 16)), rng.standard_normal(16)),
              (rng.standard_normal((3, 16)), rng.standard_normal(3))]
    x = rng.standard_normal((40, 6))
    y, cache = ntbc.mlp_forward(layers, x, act)
    g_y = rng.standard_normal(y.shape)
    gx0, g0 = ntbc.mlp_backward(layers, cache, y, g_y, act)
    y1, cache1 = ntbc.mlp_forward(layers, x, act, rnd=lambda v: v)
    gx1, g1 = ntbc.mlp_backward(layers, cache1, y1, g_y, act, rnd=lambda v: v)
    np.testing.assert_allclose(gx1, gx0, rtol=1e-12, atol=1e-13)
    for (a, b), (c, d) in zip(g1, g0):
        np.testing.assert_allclose(a, c, rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(b, d, rtol=1e-12, atol=1e-13)


def test_bf16_mode_rounds_the_colour_forward_only():
    # the training arithmetic's mode: the endpoint forward on exact operands, so its losses are
    # the FP64 mode's to the last bit; the colour forward on BF16 operands, so its losses move
    desc, p, mat, refs = _fd_setup("selu")
    ids = np.array([0, 5, 17, 33, 63, 40])
    L64, _ = ntbc.losses_and_grads(desc, p, mat.textures, refs, ids, T=0.01)
    L16, _ = ntbc.losses_and_grads(desc, p, mat.textures, refs, ids, T=0.01, bf16=True)
    assert L16["L_e"] == L64["L_e"] and L16["L_cd_endpoint"] == L64["L_cd_endpoint"]
    assert L16["L_c"] != L64["L_c"]
    assert L16["L_c"] == pytest.approx(L64["L_c"], rel=2e-2)


def test_bf16_backward_rounds_an_exact_forward_input():
    # one sigmoid unit y = s(3 x), x = 1 + 2^-10 (not a BF16 value: it rounds to 1), forward
    # exact; by hand the rounded backward gives g = bf16(y (1 - y)), dL/dW = g * bf16(x) = g,
    # dL/db = g, dL/dx = g * 3 (3 is a BF16 value)
    x = np.array([[1.0 + 2.0 ** -10]])
    layers = [(np.array([[3.0]]), np.array([0.0]))]
    y, cache = ntbc.mlp_forward(layers, x, "selu")
    y_exact = 1.0 / (1.0 + math.exp(-3.0 * (1.0 + 2.0 ** -10)))
    assert y[0, 0] == pytest.approx(y_exact, rel=1e-15)
    gx, grads = ntbc.mlp_backward(layers, cache, y, np.ones_like(y), "selu", rnd=ntbc.bf16_round)
    g = float(ntbc.bf16_round(y_exact * (1.0 - y_exact)))
    assert grads[0][0][0, 0] == g and grads[0][1][0] == g and gx[0, 0] == 3.0 * g
    # without the rounding the weight gradient carries the input's 2^-10
    _, grads64 = ntbc.mlp_backward(layers, cache, y, np.ones_like(y), "selu")
    assert grads64[0][0][0, 0] == pytest.approx(y_exact * (1 - y_exact) * (1.0 + 2.0 ** -10), rel=1e-14)


def test_params_from_flat_inverts_the_canonical_order():
    # the flat reader takes exactly the values of flatten_params, in that order, and its size is
    # the paper-pinned parameter count (4096^2 material, 8 levels 16..2048: the storage figure of
    # Sec. 4.3 counts the same values)
    cres = ntbc.level_resolutions(4, 4, 16)
    desc = ntbc.ModelDesc(32, 32, [1, 4], cres, ntbc.endpoint_resolutions(cres, 8), hidden_layers=2)
    p = synth.random_params_like(synth.init_params(cres, desc.endpoint_res, 2, desc.mlp_dims("color"),
                                                   desc.mlp_dims("endpoint"), seed=4), seed=5)
    flat = np.concatenate([np.asarray(a, np.float64).ravel() for a in ntbc.flatten_params(p)])
    q = ntbc.params_from_flat(desc, flat)
    for a, b in zip(ntbc.flatten_params(p), ntbc.flatten_params(q)):
        assert a.shape == b.shape and np.array_equal(a, b)
    with pytest.raises(ValueError):
        ntbc.params_from_flat(desc, flat[:-1])
    with pytest.raises(ValueError):
        ntbc.params_from_flat(desc, np.concatenate([flat, [0.0]]))
    big = ntbc.ModelDesc(4096, 4096, [1, 1, 4, 4, 4, 4], ntbc.level_resolutions(8, 16, 2048),
                         ntbc.endpoint_resolutions(ntbc.level_resolutions(8, 16, 2048), 1024))
    n = sum(r * r * 2 for r in big.color_res + big.endpoint_res)
    for which in ("color", "endpoint"):
        d = big.mlp_dims(which)
        n += sum(d[i] * d[i + 1] + d[i + 1] for i in range(len(d) - 1))
    assert ntbc.storage_bytes(big, grid_bits=32, weight_bytes=4) == 4 * n
