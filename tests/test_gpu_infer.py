"""GPU parity of NTBC inference against the FP64 oracle network on the same weights.

Bars: pre-quantisation outputs within 1e-3 relative of the FP64 oracle; at most
0.1% of endpoint or index fields differ after quantisation (a field flips only
where FP32 and FP64 outputs straddle a rounding or argmax boundary); decoded
PSNR within 0.05 dB; exported grid codes bit-exact (FP32 decisions on both sides).
"""
import numpy as np
import pytest
import torch

import descs
import synth
from oracle import bc as obc, ntbc as ont

nt = pytest.importorskip("paper_2407_09543_gb300")
pytestmark = pytest.mark.gpu
DEV = "cuda"
RTOL = 1e-3
# pure FP16 activations (NTBC_PREC_FP16_FAST): four FP16 roundings of the activations
# (features + three hidden layers), unit roundoff u = 2^-11, each amplified at most ~2x by
# the rest of the network: 8u ~ 4e-3
RTOL_FAST = 4e-3


def make_case(side=64, kinds=("sine_rgb", "sine_r"), levels=3, lo=4, hi=16, hidden=2, act="selu", seed=0,
              height=None):
    mat = synth.make_material(f"inf{side}", side, list(kinds), seed)
    h = height or side
    desc, odesc = descs.case_descs(nt, mat.formats, side, levels, lo, hi, hidden, act, height=h)
    params = synth.random_params_like(descs.init_params(odesc, seed), seed=seed + 1)
    return mat, desc, odesc, params


def gpu_model(desc, params, grid_bits=0, weight_prec=0):
    m = nt.Model(desc)
    m.set_params(torch.from_numpy(nt.configs.flatten(desc, params)).to(DEV))
    m.export(grid_bits=grid_bits, weight_prec=weight_prec)
    return m


def gpu_forward(model, ids):
    lay = model.layout
    t = torch.from_numpy(np.asarray(ids, np.int32)).to(DEV)
    e = torch.empty(len(ids), lay.out_endpoint, device=DEV)
    c = torch.empty(len(ids), 16, lay.out_color, device=DEV)
    model.forward(t, e, c)
    torch.cuda.synchronize()
    return e.cpu().numpy().astype(np.float64), c.cpu().numpy().astype(np.float64)


def gpu_blocks(model, desc):
    n = (desc.width // 4) * (desc.height // 4)
    outs = [torch.empty(n * 8, dtype=torch.uint8, device=DEV) for _ in range(desc.n_textures)]
    model.infer_to_bc(outs)
    torch.cuda.synchronize()
    return [o.cpu().numpy().reshape(-1, 8) for o in outs]


def field_mismatch(fmt, a, b):
    """(mismatched endpoint + index fields, total fields)."""
    if fmt == 1:
        a0, a1, ac = obc.bc1_unpack(a)
        b0, b1, bc_ = obc.bc1_unpack(b)
    else:
        a0, a1, ac = obc.bc4_unpack(a)
        b0, b1, bc_ = obc.bc4_unpack(b)
    mism = int((a0 != b0).sum() + (a1 != b1).sum() + (ac != bc_).sum())
    return mism, a0.size * 18


def oracle_params_fp16(params):
    out = dict(color_grid=params["color_grid"], endpoint_grid=params["endpoint_grid"])
    for k in ("color_mlp", "endpoint_mlp"):
        out[k] = [(W.astype(np.float16).astype(np.float64), b.astype(np.float16).astype(np.float64)) for W, b in params[k]]
    return out


@pytest.mark.parametrize("act,hidden", [("selu", 2), ("relu", 2), ("selu", 3), ("selu", 1)])
def test_forward_fp32_matches_oracle(act, hidden):
    mat, desc, odesc, params = make_case(act=act, hidden=hidden)
    model = gpu_model(desc, params)
    ids = np.arange(odesc.n_blocks)
    e, c = gpu_forward(model, ids)
    er, cr = ont.forward_blocks(odesc, params, ids)
    np.testing.assert_allclose(e, er, rtol=RTOL, atol=1e-6)
    np.testing.assert_allclose(c, cr, rtol=RTOL, atol=1e-6)


# pure FP16: outputs off by up to ~RTOL_FAST flip the decisions of texels whose colour
# lies within that distance of a boundary between palette entries (spacing ~|e1 - e0| / 3
# for BC1, / 7 for BC4): measured 0.16%, bound 0.5%
MISMATCH_FAST = 0.005


def check_blocks(mat, desc, odesc, got, ref, max_mismatch=0.001):
    total_m, total_f = 0, 0
    for t, fmt in enumerate(mat.formats):
        m, f = field_mismatch(fmt, got[t], ref[t])
        total_m += m
        total_f += f
        dec_g = obc.decode(fmt, got[t], desc.width, desc.height)
        dec_r = obc.decode(fmt, ref[t], desc.width, desc.height)
        src = mat.textures[t][:desc.height]
        assert abs(obc.psnr(dec_g, src) - obc.psnr(dec_r, src)) <= 0.05
    assert total_m <= max_mismatch * total_f, (total_m, total_f)


@pytest.mark.parametrize("side,height", [(64, 64), (264, 132)])
def test_infer_to_bc_fp32(side, height):
    mat, desc, odesc, params = make_case(side=side, height=height, levels=4, lo=4, hi=32)
    model = gpu_model(desc, params)
    check_blocks(mat, desc, odesc, gpu_blocks(model, desc), ont.infer_blocks(odesc, params))


def test_export_u8_codes_bit_exact_and_inference():
    mat, desc, odesc, params = make_case(side=128, levels=4, lo=8, hi=64, hidden=3)
    model = gpu_model(desc, params, grid_bits=8, weight_prec=nt.PREC_FP16)
    lay = model.layout
    levels = desc.color_levels + desc.endpoint_levels
    codes = torch.empty(lay.grid_floats, dtype=torch.uint8, device=DEV)
    sc = torch.empty(levels, device=DEV)
    zr = torch.empty(levels, device=DEV)
    model.exported_grid(codes, sc, zr)
    torch.cuda.synchronize()
    oc, os_, oz = ont.export_grid(params["color_grid"] + params["endpoint_grid"], 8)
    np.testing.assert_array_equal(sc.cpu().numpy(), os_)
    np.testing.assert_array_equal(zr.cpu().numpy(), oz)
    np.testing.assert_array_equal(codes.cpu().numpy(), np.concatenate([c.ravel() for c in oc]))
    deq = ont.dequantize_grid(oc, os_, oz)
    nc = desc.color_levels
    p16 = oracle_params_fp16(params)
    ids = np.arange(odesc.n_blocks)
    e, c = gpu_forward(model, ids)
    er, cr = ont.forward_blocks(odesc, p16, ids, color_grid=deq[:nc], endpoint_grid=deq[nc:])
    np.testing.assert_allclose(e, er, rtol=RTOL, atol=1e-6)
    np.testing.assert_allclose(c, cr, rtol=RTOL, atol=1e-6)
    ref = ont.infer_blocks(odesc, p16, color_grid=deq[:nc], endpoint_grid=deq[nc:])
    check_blocks(mat, desc, odesc, gpu_blocks(model, desc), ref)


def test_blob_roundtrip_reproduces_blocks():
    mat, desc, odesc, params = make_case(side=64, levels=3, lo=4, hi=16)
    model = gpu_model(desc, params, grid_bits=8, weight_prec=nt.PREC_FP16)
    before = gpu_blocks(model, desc)
    blob = torch.empty(model.blob_size(), dtype=torch.uint8).pin_memory()
    model.save(blob)
    other = nt.Model(desc)
    other.load(blob)
    after = gpu_blocks(other, desc)
    for a, b in zip(before, after):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("side,height,chunks,prec", [(68, 60, 1, 1), (68, 60, 3, 1), (256, 256, 16, 1),
                                                     (256, 192, 5, 2), (132, 100, 4, 0)])
def test_infer_to_host_matches_device(side, height, chunks, prec):
    # blocks delivered to pinned host memory range by range equal the device-resident result;
    # 68 x 60 is 255 blocks (a ragged last work unit), 256^2 with 16 ranges of 256 blocks
    mat, desc, odesc, params = make_case(side=side, height=height, levels=3, lo=4, hi=16)
    model = gpu_model(desc, params, grid_bits=8, weight_prec=prec)
    want = gpu_blocks(model, desc)
    n = (desc.width // 4) * (desc.height // 4)
    host = [torch.zeros(n * 8, dtype=torch.uint8).pin_memory() for _ in range(desc.n_textures)]
    model.infer_to_host(host, chunks=chunks)
    torch.cuda.synchronize()
    for a, h in zip(want, host):
        np.testing.assert_array_equal(a, h.numpy().reshape(-1, 8))
    # a second call reuses the staging the model keeps
    for h in host:
        h.zero_()
    model.infer_to_host(host, chunks=chunks)
    torch.cuda.synchronize()
    for a, h in zip(want, host):
        np.testing.assert_array_equal(a, h.numpy().reshape(-1, 8))


def test_infer_to_host_rejects_bad_chunks():
    mat, desc, odesc, params = make_case(side=64, levels=3, lo=4, hi=16)
    model = gpu_model(desc, params, grid_bits=8, weight_prec=nt.PREC_FP16)
    host = [torch.zeros(16 * 16 * 8, dtype=torch.uint8) for _ in range(desc.n_textures)]
    for bad in (0, 17):
        with pytest.raises(nt.NTBCError):
            model.infer_to_host(host, chunks=bad)


def test_blob_u4_packed_two_codes_per_byte():
    # a 4-bit export stores two grid codes per byte (low nibble first): the blob is half a
    # byte per grid value smaller than the 8-bit one, its packed part matches the exported
    # codes, and a fresh model loaded from it reproduces the blocks
    import ctypes
    mat, desc, odesc, params = make_case(side=64, levels=3, lo=4, hi=16)
    model = gpu_model(desc, params, grid_bits=8, weight_prec=nt.PREC_FP16)
    size8 = model.blob_size()
    model.export(grid_bits=4, weight_prec=nt.PREC_FP16)
    lay = model.layout
    assert size8 - model.blob_size() == lay.grid_floats - (lay.grid_floats + 1) // 2
    before = gpu_blocks(model, desc)
    blob = torch.empty(model.blob_size(), dtype=torch.uint8).pin_memory()
    model.save(blob)
    levels = desc.color_levels + desc.endpoint_levels
    head = 8 + ctypes.sizeof(nt.ModelDesc) + 8 + 8 * levels
    packed = blob.numpy()[head:head + (lay.grid_floats + 1) // 2]
    oc, _, _ = ont.export_grid(params["color_grid"] + params["endpoint_grid"], 4)
    codes = np.concatenate([c.reshape(-1) for c in oc]).astype(np.uint8)
    assert codes.size == lay.grid_floats and codes.max() <= 15
    np.testing.assert_array_equal(packed & 15, codes[0::2])
    np.testing.assert_array_equal(packed[:codes[1::2].size] >> 4, codes[1::2])
    other = nt.Model(desc)
    other.load(blob)
    for a, b in zip(before, gpu_blocks(other, desc)):
        np.testing.assert_array_equal(a, b)


def _blob_fp8_part(model, desc, n_layers, mma=False, grid_bits=8):
    """(per-layer exponents, codes in parameter-layout order) from a saved FP8 blob: header
    (magic, version, desc, grid_bits, weight_prec), (s, z) per level, the grid (one code per
    byte, two per byte for 4-bit grids, FP32 for grid_bits 0), then the
    MLP part as 2 * NTBC_MAX_MLP_LAYERS int32 weight exponents (for NTBC_PREC_FP8_MMA as many
    activation exponents after them) followed by one code per parameter. With mma the
    exponents are returned as (weight exponents, activation exponents)."""
    import ctypes
    blob = torch.empty(model.blob_size(), dtype=torch.uint8).pin_memory()
    model.save(blob)
    b = blob.numpy()
    lay = model.layout
    levels = desc.color_levels + desc.endpoint_levels
    head = 8 + ctypes.sizeof(nt.ModelDesc) + 8
    grid_bytes = {8: lay.grid_floats, 4: (lay.grid_floats + 1) // 2, 0: 4 * lay.grid_floats}[grid_bits]
    wpart = b[head + 8 * levels + grid_bytes:]
    nw = lay.total - lay.grid_floats
    n_exp = 2 * nt.MAX_MLP_LAYERS * (2 if mma else 1)
    ints = wpart[:4 * n_exp].view(np.int32)
    exps = (ints[:n_layers], ints[2 * nt.MAX_MLP_LAYERS:2 * nt.MAX_MLP_LAYERS + n_layers]) if mma else ints[:n_layers]
    return exps, wpart[4 * n_exp:4 * n_exp + nw]


def test_fp8_weights_codes_and_parity():
    mat, desc, odesc, params = make_case(side=128, levels=4, lo=8, hi=64, hidden=3)
    model = gpu_model(desc, params, grid_bits=8, weight_prec=nt.PREC_FP8)
    p8, exps, codes = ont.fp8_params(params)
    # codes and exponents bit-exact with the oracle's E4M3 rounding
    gexps, gcodes = _blob_fp8_part(model, desc, len(exps))
    np.testing.assert_array_equal(gexps, np.array(exps))
    code_params = dict(color_grid=params["color_grid"], endpoint_grid=params["endpoint_grid"],
                       color_mlp=codes[:len(params["color_mlp"])], endpoint_mlp=codes[len(params["color_mlp"]):])
    want = nt.configs.flatten(desc, code_params)[model.layout.grid_floats:].astype(np.uint8)
    np.testing.assert_array_equal(gcodes, want)
    # outputs within 1e-3 of the FP64 network with the same FP8 weights
    oc, os_, oz = ont.export_grid(params["color_grid"] + params["endpoint_grid"], 8)
    deq = ont.dequantize_grid(oc, os_, oz)
    nc = desc.color_levels
    ids = np.arange(odesc.n_blocks)
    e, c = gpu_forward(model, ids)
    er, cr = ont.forward_blocks(odesc, p8, ids, color_grid=deq[:nc], endpoint_grid=deq[nc:])
    np.testing.assert_allclose(e, er, rtol=RTOL, atol=1e-6)
    np.testing.assert_allclose(c, cr, rtol=RTOL, atol=1e-6)
    ref = ont.infer_blocks(odesc, p8, color_grid=deq[:nc], endpoint_grid=deq[nc:])
    check_blocks(mat, desc, odesc, gpu_blocks(model, desc), ref)
    # the stored blob reproduces the blocks
    before = gpu_blocks(model, desc)
    blob = torch.empty(model.blob_size(), dtype=torch.uint8).pin_memory()
    model.save(blob)
    other = nt.Model(desc)
    other.load(blob)
    for a, b in zip(before, gpu_blocks(other, desc)):
        np.testing.assert_array_equal(a, b)


def _fp8_mma_case(mat, desc, odesc, params, bits=8):
    """The FP8-arithmetic model on the GPU and the oracle's side of it: FP8 weights, its own
    grid export and its own calibration of the activation exponents."""
    model = gpu_model(desc, params, grid_bits=bits, weight_prec=nt.PREC_FP8_MMA)
    p8, wexps, codes = ont.fp8_params(params)
    if bits:
        oc, os_, oz = ont.export_grid(params["color_grid"] + params["endpoint_grid"], bits)
        deq = ont.dequantize_grid(oc, os_, oz)
        nc = desc.color_levels
        grids = dict(color_grid=deq[:nc], endpoint_grid=deq[nc:])
    else:                                   # FP32 grids (the parameters as the library stores them)
        p32 = descs.as_float32(params)
        grids = dict(color_grid=p32["color_grid"], endpoint_grid=p32["endpoint_grid"])
    aexps = ont.fp8_activation_exponents(odesc, p8, **grids)
    return model, p8, wexps, codes, aexps, grids


# FP8 arithmetic: the GPU and the oracle round every layer input to E4M3 from values that
# differ only by FP32 arithmetic (~1e-6 relative), so they take the same rounding decisions
# except where a value sits within that distance of an E4M3 rounding boundary (a "flip": one
# input moves by one E4M3 spacing). Outputs without a flip agree like the split FP16 path
# (1e-3 relative); flips are rare (expected well under 0.5 % of the outputs: ~10^-5 per
# rounding, a few hundred roundings upstream of an output), and even a flipped output stays
# within twice the propagated E4M3 error bound (both evaluations lie within that bound of the
# exact-activation network). The decisions after quantisation then differ no more than the
# split path allows.
FP8_FLIP_FRACTION = 0.005


def _fp8_error_bound(odesc, p8, aexps, ids, grids):
    """Elementwise bound on |FP8 arithmetic - exact activations| for the outputs of the given
    blocks: every E4M3 rounding of a layer input y at scale 2^a errs by at most
    2^-4 |y| + 2^(a - 10), layer errors propagate through |W|, SELU (Lipschitz lambda alpha)
    and the sigmoid (Lipschitz 1/4)."""
    ids = np.asarray(ids, np.int64)
    s, t = ont.block_coords(odesc.blocks_x, odesc.blocks_y, ids % odesc.blocks_x, ids // odesc.blocks_x)
    xs, ys = ont.block_texel_xy(odesc, ids)
    u, v = ont.texel_coords(odesc.width, odesc.height, xs.ravel(), ys.ravel())
    nc = len(p8["color_mlp"])
    out = []
    for key, grid, (a, b), ex in (("endpoint_mlp", grids["endpoint_grid"], (s, t), aexps[nc:]),
                                  ("color_mlp", grids["color_grid"], (u, v), aexps[:nc])):
        x, _ = ont.grid_lookup([np.asarray(g, np.float64) for g in grid], a, b)
        _, cache = ont.mlp_forward(p8[key], x, odesc.activation)
        err = np.zeros_like(x)
        for l, ((W, _), (h, _)) in enumerate(zip(p8[key], cache)):
            zerr = (err + 2.0 ** -4 * (np.abs(h) + err) + 2.0 ** (ex[l] - 10)) @ np.abs(W).T
            err = zerr * (ont.SELU_LAMBDA * ont.SELU_ALPHA if l + 1 < len(p8[key]) else 0.25)
        out.append(err)
    return out[0], out[1].reshape(len(ids), 16, -1)


def check_fp8_mma_outputs(got, want, bound):
    d = np.abs(got - want)
    assert np.mean(d > RTOL * np.abs(want) + 1e-6) <= FP8_FLIP_FRACTION, float(np.mean(d > RTOL * np.abs(want) + 1e-6))
    assert np.all(d <= 2 * bound + 1e-5), float(np.max(d - 2 * bound))


def test_fp8_mma_exponents_codes_and_parity():
    mat, desc, odesc, params = make_case(side=128, levels=4, lo=8, hi=64, hidden=3)
    model, p8, wexps, codes, aexps, grids = _fp8_mma_case(mat, desc, odesc, params)
    (gw, ga), gcodes = _blob_fp8_part(model, desc, len(wexps), mma=True)
    np.testing.assert_array_equal(gw, np.array(wexps))
    np.testing.assert_array_equal(ga, np.array(aexps))
    code_params = dict(color_grid=params["color_grid"], endpoint_grid=params["endpoint_grid"],
                       color_mlp=codes[:len(params["color_mlp"])], endpoint_mlp=codes[len(params["color_mlp"]):])
    want = nt.configs.flatten(desc, code_params)[model.layout.grid_floats:].astype(np.uint8)
    np.testing.assert_array_equal(gcodes, want)
    ids = np.arange(odesc.n_blocks)
    e, c = gpu_forward(model, ids)
    er, cr = ont.forward_blocks(odesc, p8, ids, fp8_act=aexps, **grids)
    be, bc_ = _fp8_error_bound(odesc, p8, aexps, ids, grids)
    check_fp8_mma_outputs(e, er, be)
    check_fp8_mma_outputs(c, cr, bc_)
    # the FP8 arithmetic is not the exact-activation network: outputs move by up to a few
    # per cent (within the bound), which is what the mode costs in accuracy
    ex, cx = ont.forward_blocks(odesc, p8, ids, **grids)
    assert np.all(np.abs(c - cx) <= bc_ + 1e-5) and np.abs(c - cx).max() > 1e-3
    got = gpu_blocks(model, desc)
    check_blocks(mat, desc, odesc, got, ont.infer_blocks(odesc, p8, fp8_act=aexps, **grids))
    # the stored blob (FP8 codes and both exponent lists) reproduces the blocks
    blob = torch.empty(model.blob_size(), dtype=torch.uint8).pin_memory()
    model.save(blob)
    other = nt.Model(desc)
    other.load(blob)
    for a, b in zip(got, gpu_blocks(other, desc)):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("act,hidden,bits", [("relu", 2, 8), ("selu", 1, 4), ("selu", 3, 0)])
def test_fp8_mma_activations_depths_and_grids(act, hidden, bits):
    """ReLU and SELU, one to three hidden layers, 8-bit, 4-bit and FP32 grids; a non-square
    material whose block count is not a multiple of the work unit."""
    mat, desc, odesc, params = make_case(side=264, height=132, levels=4, lo=4, hi=32, hidden=hidden, act=act)
    model, p8, _, _, aexps, grids = _fp8_mma_case(mat, desc, odesc, params, bits=bits)
    (_, ga), _ = _blob_fp8_part(model, desc, len(aexps), mma=True, grid_bits=bits)
    np.testing.assert_array_equal(ga, np.array(aexps))
    ids = np.arange(odesc.n_blocks)
    e, c = gpu_forward(model, ids)
    er, cr = ont.forward_blocks(odesc, p8, ids, fp8_act=aexps, **grids)
    be, bc_ = _fp8_error_bound(odesc, p8, aexps, ids, grids)
    check_fp8_mma_outputs(e, er, be)
    check_fp8_mma_outputs(c, cr, bc_)
    check_blocks(mat, desc, odesc, gpu_blocks(model, desc), ont.infer_blocks(odesc, p8, fp8_act=aexps, **grids))


def test_full_size_4k_sampled():
    # the 4096^2 four-texture workload in the launch configuration the benchmark times;
    # the oracle evaluates a seeded sample of blocks one by one
    w = nt.configs.WORKLOADS["mat4k"]
    formats = [1, 1, 4, 4]
    desc, odesc = descs.case_descs(nt, formats, 4096, w.levels, w.min_res, w.max_res, 3, "selu")
    params = synth.random_params_like(descs.init_params(odesc, 3), seed=4)
    model = gpu_model(desc, params, grid_bits=8, weight_prec=nt.PREC_FP16)
    oc, os_, oz = ont.export_grid(params["color_grid"] + params["endpoint_grid"], 8)
    deq = ont.dequantize_grid(oc, os_, oz)
    nc = desc.color_levels
    p16 = oracle_params_fp16(params)
    ids = np.sort(np.random.default_rng(0).choice(odesc.n_blocks, 400, replace=False))
    e, c = gpu_forward(model, ids)
    er, cr = ont.forward_blocks(odesc, p16, ids, color_grid=deq[:nc], endpoint_grid=deq[nc:])
    np.testing.assert_allclose(e, er, rtol=RTOL, atol=1e-6)
    np.testing.assert_allclose(c, cr, rtol=RTOL, atol=1e-6)
    got = gpu_blocks(model, desc)
    ref = ont.infer_blocks(odesc, p16, block_ids=ids, color_grid=deq[:nc], endpoint_grid=deq[nc:])
    total_m = total_f = 0
    for t, fmt in enumerate(formats):
        m, f = field_mismatch(fmt, got[t][ids], ref[t])
        total_m += m
        total_f += f
    assert total_m <= 0.001 * total_f


def test_split_tail_launch_equals_unsplit_launch():
    """On a full grid the single-material launch sends its partial last round to a second,
    chained launch of half-size work units. The 4096^2 material's blocks must equal those of
    the work-queue batch launch (128-block units throughout, no split) and of the host
    delivery (ranges, only the last one split), bit for bit: the units differ only in how
    many rows their endpoint MMA holds."""
    w = nt.configs.WORKLOADS["mat4k"]
    formats = [1, 1, 4, 4]
    desc, odesc = descs.case_descs(nt, formats, 4096, w.levels, w.min_res, w.max_res, 3, "selu")
    params = synth.random_params_like(descs.init_params(odesc, 5), seed=6)
    model = gpu_model(desc, params, grid_bits=8, weight_prec=nt.PREC_FP16)
    torch.cuda.synchronize()
    single = gpu_blocks(model, desc)
    n = odesc.n_blocks
    outs = [torch.zeros(n * 8, dtype=torch.uint8, device=DEV) for _ in formats]
    batch = nt.Batch([model], [outs], mode=nt.BATCH_QUEUE)
    batch.infer()
    torch.cuda.synchronize()
    host = [torch.empty(n * 8, dtype=torch.uint8).pin_memory() for _ in formats]
    model.infer_to_host(host, chunks=3)
    torch.cuda.synchronize()
    for t in range(len(formats)):
        q = outs[t].cpu().numpy().reshape(-1, 8)
        np.testing.assert_array_equal(single[t], q)
        np.testing.assert_array_equal(single[t], host[t].numpy().reshape(-1, 8))
    batch.close()


def test_forward_split_tail_outputs_land_in_place():
    """ntbc_forward over every block of the 4096^2 material runs as full rounds plus a split
    tail whose raw outputs go to the tail's offset in e_hat / c_hat: they must equal a forward
    of just the last 2000 blocks (one partial round, no split), bit for bit, and a sample of
    the head must equal a forward of those blocks alone."""
    w = nt.configs.WORKLOADS["mat4k"]
    desc, odesc = descs.case_descs(nt, [1, 1, 4, 4], 4096, w.levels, w.min_res, w.max_res, 3, "selu")
    params = synth.random_params_like(descs.init_params(odesc, 7), seed=8)
    model = gpu_model(desc, params, grid_bits=8, weight_prec=nt.PREC_FP16)
    n = odesc.n_blocks
    assert model.infer_plan()[0] == 2
    lay = model.layout
    ids = torch.arange(n, dtype=torch.int32, device=DEV)
    e = torch.empty(n, lay.out_endpoint, device=DEV)
    c = torch.empty(n, 16, lay.out_color, device=DEV)
    model.forward(ids, e, c)
    for sel in (np.arange(n - 2000, n), np.sort(np.random.default_rng(2).choice(n - 2000, 500, replace=False))):
        es, cs = gpu_forward(model, sel)
        np.testing.assert_array_equal(e[torch.from_numpy(sel).to(DEV)].cpu().numpy().astype(np.float64), es)
        np.testing.assert_array_equal(c[torch.from_numpy(sel).to(DEV)].cpu().numpy().astype(np.float64), cs)


def test_infer_plan():
    """The launch plan: a small material fits one partial round (one launch); the 4096^2
    material runs full rounds plus a split tail (two launches); FP32 is the SIMT kernel."""
    mat, desc, odesc, params = make_case(side=64)
    model = gpu_model(desc, params, grid_bits=8, weight_prec=nt.PREC_FP16)
    launches, ub, flight = model.infer_plan()
    assert launches == 1 and ub == 128 and flight > 0
    model.export(grid_bits=8, weight_prec=nt.PREC_FP32)
    assert model.infer_plan() == (1, 0, 0)
    w = nt.configs.WORKLOADS["mat4k"]
    desc4, odesc4 = descs.case_descs(nt, [1, 1, 4, 4], 4096, w.levels, w.min_res, w.max_res, 3, "selu")
    big = nt.Model(desc4)
    big.export(grid_bits=8, weight_prec=nt.PREC_FP16)
    launches, ub, flight = big.infer_plan()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert ub == 128 and flight % sms == 0
    units = odesc4.n_blocks // 128
    assert launches == (2 if units % flight else 1)
    unexported = nt.Model(desc)
    with pytest.raises(nt.NTBCError):
        unexported.infer_plan()


def test_full_size_4k_sampled_fp8_arithmetic():
    """The 4096^2 four-texture workload in the FP8 arithmetic: the calibration exponents over
    the whole material's sample equal the oracle's, and sampled blocks meet the FP8 bars."""
    w = nt.configs.WORKLOADS["mat4k"]
    formats = [1, 1, 4, 4]
    desc, odesc = descs.case_descs(nt, formats, 4096, w.levels, w.min_res, w.max_res, 3, "selu")
    params = synth.random_params_like(descs.init_params(odesc, 3), seed=4)
    model, p8, wexps, _, aexps, grids = _fp8_mma_case(None, desc, odesc, params)
    (gw, ga), _ = _blob_fp8_part(model, desc, len(wexps), mma=True)
    np.testing.assert_array_equal(gw, np.array(wexps))
    np.testing.assert_array_equal(ga, np.array(aexps))
    ids = np.sort(np.random.default_rng(1).choice(odesc.n_blocks, 300, replace=False))
    e, c = gpu_forward(model, ids)
    er, cr = ont.forward_blocks(odesc, p8, ids, fp8_act=aexps, **grids)
    be, bc_ = _fp8_error_bound(odesc, p8, aexps, ids, grids)
    check_fp8_mma_outputs(e, er, be)
    check_fp8_mma_outputs(c, cr, bc_)
    got = gpu_blocks(model, desc)
    ref = ont.infer_blocks(odesc, p8, block_ids=ids, fp8_act=aexps, **grids)
    total_m = total_f = 0
    for t, fmt in enumerate(formats):
        m, f = field_mismatch(fmt, got[t][ids], ref[t])
        total_m += m
        total_f += f
    assert total_m <= 0.005 * total_f


def test_fp16_fast_mode_stated_tolerance():
    mat, desc, odesc, params = make_case(side=128, levels=4, lo=8, hi=64, hidden=3)
    model = gpu_model(desc, params, grid_bits=8, weight_prec=nt.PREC_FP16_FAST)
    oc, os_, oz = ont.export_grid(params["color_grid"] + params["endpoint_grid"], 8)
    deq = ont.dequantize_grid(oc, os_, oz)
    nc = desc.color_levels
    p16 = oracle_params_fp16(params)
    ids = np.arange(odesc.n_blocks)
    e, c = gpu_forward(model, ids)
    er, cr = ont.forward_blocks(odesc, p16, ids, color_grid=deq[:nc], endpoint_grid=deq[nc:])
    np.testing.assert_allclose(e, er, rtol=RTOL_FAST, atol=1e-5)
    np.testing.assert_allclose(c, cr, rtol=RTOL_FAST, atol=1e-5)
    ref = ont.infer_blocks(odesc, p16, color_grid=deq[:nc], endpoint_grid=deq[nc:])
    check_blocks(mat, desc, odesc, gpu_blocks(model, desc), ref, MISMATCH_FAST)


@pytest.mark.parametrize("prec", [1, 2])
def test_tensor_core_ragged_and_fp32_grids(prec):
    # block count not a multiple of the 128-block work unit, FP32 (unquantised) grids
    mat, desc, odesc, params = make_case(side=264, height=132, levels=4, lo=4, hi=32, hidden=2)
    model = gpu_model(desc, params, grid_bits=0, weight_prec=prec)
    p16 = oracle_params_fp16(params)
    ids = np.arange(odesc.n_blocks)
    e, c = gpu_forward(model, ids)
    er, cr = ont.forward_blocks(odesc, p16, ids)
    tol = RTOL if prec == 1 else RTOL_FAST
    np.testing.assert_allclose(e, er, rtol=tol, atol=1e-5)
    np.testing.assert_allclose(c, cr, rtol=tol, atol=1e-5)
    check_blocks(mat, desc, odesc, gpu_blocks(model, desc), ont.infer_blocks(odesc, p16),
                 0.001 if prec == 1 else MISMATCH_FAST)


def _oracle_trained(bits, seed=5):
    """Weights trained by the oracle (FP64 Adam, QAT at `bits`) on a 64^2 three-texture material:
    realistic, sharper weights than random ones, and none of it comes from the CUDA path."""
    from oracle import philox
    mat = synth.make_material("trained", 64, ["sine_rgb", "sine_r", "sine_rgb"], seed)
    desc, odesc = descs.case_descs(nt, mat.formats, 64, 4, 8, 32, 3, "selu")
    p0 = descs.init_params(odesc, seed)
    refs = [obc.encode(f, t, 64, 64) for f, t in zip(mat.formats, mat.textures)]
    cfg = ont.TrainConfig(steps=200, batch_texels=1024, qat_fraction=0.1, grid_bits=bits)
    p1, _ = ont.train(odesc, p0, mat.textures, refs, cfg, lambda s: philox.sample_blocks(1, s, 64, odesc.n_blocks))
    p32 = descs.as_float32(p1)          # the float32 weights both sides use
    return mat, desc, odesc, p32


@pytest.mark.parametrize("bits", [8, 4])
def test_trained_weights_parity_all_modes(bits):
    mat, desc, odesc, params = _oracle_trained(bits)
    oc, os_, oz = ont.export_grid(params["color_grid"] + params["endpoint_grid"], bits)
    deq = ont.dequantize_grid(oc, os_, oz)
    nc = desc.color_levels
    ids = np.arange(odesc.n_blocks)
    for prec, rtol, mism in ((nt.PREC_FP32, RTOL, 0.001), (nt.PREC_FP16, RTOL, 0.001),
                             (nt.PREC_FP16_FAST, RTOL_FAST, MISMATCH_FAST), (nt.PREC_FP8, RTOL, 0.001)):
        model = gpu_model(desc, params, grid_bits=bits, weight_prec=prec)
        if prec == nt.PREC_FP32:
            pw = params
        elif prec == nt.PREC_FP8:
            pw = ont.fp8_params(params)[0]
        else:
            pw = oracle_params_fp16(params)
        e, c = gpu_forward(model, ids)
        er, cr = ont.forward_blocks(odesc, pw, ids, color_grid=deq[:nc], endpoint_grid=deq[nc:])
        np.testing.assert_allclose(e, er, rtol=rtol, atol=1e-6)
        np.testing.assert_allclose(c, cr, rtol=rtol, atol=1e-6)
        ref = ont.infer_blocks(odesc, pw, color_grid=deq[:nc], endpoint_grid=deq[nc:])
        check_blocks(mat, desc, odesc, gpu_blocks(model, desc), ref, mism)


@pytest.mark.parametrize("prec", [0, 1])
def test_strided_outputs_make_bc3_and_bc5(prec):
    # textures [BC1 colour, BC4 alpha, BC4 r, BC4 g]: (alpha, colour) -> one BC3 texture,
    # (r, g) -> one BC5 texture, the same blocks as the unstrided outputs interleaved
    mat, desc, odesc, params = make_case(side=64, kinds=("sine_rgb", "sine_r", "sine_r", "sine_r"), levels=3)
    model = gpu_model(desc, params, grid_bits=8, weight_prec=prec)
    plain = gpu_blocks(model, desc)
    n = (desc.width // 4) * (desc.height // 4)
    bc3 = torch.zeros(n * 16, dtype=torch.uint8, device=DEV)
    bc5 = torch.zeros(n * 16, dtype=torch.uint8, device=DEV)
    model.infer_to_bc([bc3.data_ptr() + 8, bc3.data_ptr(), bc5.data_ptr(), bc5.data_ptr() + 8],
                      strides=[16, 16, 16, 16])
    torch.cuda.synchronize()
    b3 = bc3.cpu().numpy().reshape(-1, 16)
    b5 = bc5.cpu().numpy().reshape(-1, 16)
    np.testing.assert_array_equal(b3[:, :8], plain[1])
    np.testing.assert_array_equal(b3[:, 8:], plain[0])
    np.testing.assert_array_equal(b5[:, :8], plain[2])
    np.testing.assert_array_equal(b5[:, 8:], plain[3])
    # the BC3 decode of the composed blocks equals the parts' decodes
    dec = obc.decode(obc.BC3, b3, desc.width, desc.height)
    np.testing.assert_array_equal(dec[..., 3], obc.decode(obc.BC4, plain[1], desc.width, desc.height))
