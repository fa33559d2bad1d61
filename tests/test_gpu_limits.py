"""The largest models the kernels take (8 textures, 16 colour levels: 32 input features, 18
colour and 36 endpoint outputs; 8 BC1 textures with 16 endpoint levels: 32 endpoint inputs and
48 outputs) and the degenerate cases of the method: every block solid (equal endpoints: BC1
all codes 0, BC4 six-value mode with r0 = r1), an empty block list."""
import numpy as np
import pytest
import torch

import descs
import synth
from oracle import bc as obc, ntbc as ont

nt = pytest.importorskip("paper_2407_09543_gb300")
pytestmark = pytest.mark.gpu
DEV = "cuda"
KINDS = ["sine_rgb", "sine_r", "sine_rgb", "sine_rgb", "sine_r", "sine_rgb", "sine_r", "sine_rgb"]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).ravel()).to(DEV)


def max_case(seed=0):
    side = 64
    mat = synth.make_material("limits", side, KINDS, seed)
    assert len(mat.formats) == nt.MAX_TEXTURES
    desc, odesc = descs.case_descs(nt, mat.formats, side, nt.MAX_LEVELS, 4, 64, 3, "selu")
    assert desc.color_levels == nt.MAX_LEVELS
    params = synth.random_params_like(descs.init_params(odesc, seed), seed=seed + 1)
    return mat, desc, odesc, params


def fp16_params(params):
    out = dict(params)
    for k in ("color_mlp", "endpoint_mlp"):
        out[k] = [(W.astype(np.float16).astype(np.float64), b.astype(np.float16).astype(np.float64)) for W, b in params[k]]
    return out


def run_blocks(model, desc):
    n = (desc.width // 4) * (desc.height // 4)
    outs = [torch.empty(n * 8, dtype=torch.uint8, device=DEV) for _ in range(desc.n_textures)]
    model.infer_to_bc(outs)
    torch.cuda.synchronize()
    return [o.cpu().numpy().reshape(-1, 8) for o in outs]


def mismatch(formats, got, ref):
    m = f = 0
    for fmt, a, b in zip(formats, got, ref):
        unpack = obc.bc1_unpack if fmt == 1 else obc.bc4_unpack
        a0, a1, ac = unpack(a)
        b0, b1, bc_ = unpack(b)
        m += int((a0 != b0).sum() + (a1 != b1).sum() + (ac != bc_).sum())
        f += a0.size * 18
    return m, f


@pytest.mark.parametrize("prec", [0, 1])
def test_largest_model_inference(prec):
    mat, desc, odesc, params = max_case()
    assert odesc.out_color == 18 and odesc.out_endpoint == 36 and odesc.in_color == 32
    m = nt.Model(desc)
    m.set_params(_dev(nt.configs.flatten(desc, params)))
    m.export(grid_bits=8, weight_prec=prec)
    oc, os_, oz = ont.export_grid(params["color_grid"] + params["endpoint_grid"], 8)
    deq = ont.dequantize_grid(oc, os_, oz)
    nc = desc.color_levels
    pw = params if prec == 0 else fp16_params(params)
    ids = np.arange(odesc.n_blocks)
    lay = m.layout
    e = torch.empty(len(ids), lay.out_endpoint, device=DEV)
    c = torch.empty(len(ids), 16, lay.out_color, device=DEV)
    m.forward(_dev(ids.astype(np.int32)), e, c)
    torch.cuda.synchronize()
    er, cr = ont.forward_blocks(odesc, pw, ids, color_grid=deq[:nc], endpoint_grid=deq[nc:])
    np.testing.assert_allclose(e.cpu().numpy(), er, rtol=1e-3, atol=1e-6)
    np.testing.assert_allclose(c.cpu().numpy(), cr, rtol=1e-3, atol=1e-6)
    got = run_blocks(m, desc)
    mm, ff = mismatch(mat.formats, got, ont.infer_blocks(odesc, pw, color_grid=deq[:nc], endpoint_grid=deq[nc:]))
    assert mm <= 0.001 * ff


def check_gradients(mat, desc, odesc, params, side, ids, precision):
    refs = [obc.encode(f, t, side, side) for f, t in zip(mat.formats, mat.textures)]
    tex_d = [_dev(t) for t in mat.textures]
    ref_d = [_dev(r) for r in refs]
    material = nt.Material.make(side, side, mat.formats, tex_d, ref_d)
    m = nt.Model(desc)
    m.set_params(_dev(nt.configs.flatten(desc, params)))
    grads = torch.empty(m.n_params, device=DEV)
    losses = torch.empty(6, device=DEV)
    m.train_grads(material, _dev(ids.astype(np.int32)), grads, losses, qat_bits=8, precision=precision)
    torch.cuda.synchronize()
    L, g = ont.losses_and_grads(odesc, params, mat.textures, refs, ids, qat_bits=8, bf16=bool(precision))
    want_l = [L["L_e"], L["L_cd_endpoint"], L["L_c"], L["L_cd_color"], L["L_endpoint"], L["L_color"]]
    np.testing.assert_allclose(losses.cpu().numpy(), want_l, rtol=2e-3)
    gg = nt.configs.unflatten(desc, grads.cpu().numpy())
    tol = 5e-3 if precision else 2e-3
    for key in ("color_grid", "endpoint_grid"):
        for a, b in zip(gg[key], g[key]):
            assert np.linalg.norm(a - b) <= tol * max(np.linalg.norm(b), 1e-30), key
    for key in ("color_mlp", "endpoint_mlp"):
        for (aW, ab), (bW, bb) in zip(gg[key], g[key]):
            assert np.linalg.norm(aW - bW) <= tol * np.linalg.norm(bW), key
            assert np.linalg.norm(ab - bb) <= tol * np.linalg.norm(bb), key


@pytest.mark.parametrize("precision", [0, 1])
def test_largest_model_gradients(precision):
    # BF16: the colour pass needs 272 TMEM columns here, so it runs one warpgroup per CTA
    mat, desc, odesc, params = max_case(seed=2)
    ids = np.array([0, 3, 7, 15, 100, 255, 128, 64, 3, 200], np.int64)
    check_gradients(mat, desc, odesc, params, 64, ids, precision)


@pytest.mark.parametrize("precision", [0, 1])
def test_largest_endpoint_network_gradients(precision):
    # the widest endpoint network: 16 endpoint levels (every colour level no finer than the 64
    # blocks per side) and 8 BC1 textures, 32 inputs and 48 outputs; its BF16 pass, with the
    # split forward's lo weight image, is the largest shared-memory footprint of the training
    # kernels
    side = 256
    mat = synth.make_material("limits", side, ["sine_rgb"] * nt.MAX_TEXTURES, 4)
    desc, odesc = descs.case_descs(nt, mat.formats, side, nt.MAX_LEVELS, 4, 64, 3, "selu")
    assert len(odesc.endpoint_res) == nt.MAX_LEVELS and odesc.out_endpoint == 48
    params = synth.random_params_like(descs.init_params(odesc, 4), seed=5)
    ids = np.array([0, 3, 77, 1000, 4095, 2048, 513, 64, 3, 3000], np.int64)
    check_gradients(mat, desc, odesc, params, side, ids, precision)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_solid_blocks_everywhere(prec):
    # endpoint MLP output layer W = 0: every block gets the same endpoints, one constant
    # per channel; BC1 colour0 == colour1 -> all codes 0; BC4 r0 == r1 -> six-value mode
    mat, desc, odesc, params = max_case(seed=4)
    params = dict(params)
    W, b = params["endpoint_mlp"][-1]
    params["endpoint_mlp"] = params["endpoint_mlp"][:-1] + [(np.zeros_like(W), np.full_like(b, 0.3))]
    m = nt.Model(desc)
    m.set_params(_dev(nt.configs.flatten(desc, params)))
    m.export(grid_bits=8, weight_prec=prec)
    oc, os_, oz = ont.export_grid(params["color_grid"] + params["endpoint_grid"], 8)
    deq = ont.dequantize_grid(oc, os_, oz)
    nc = desc.color_levels
    pw = params if prec == 0 else fp16_params(params)
    got = run_blocks(m, desc)
    ref = ont.infer_blocks(odesc, pw, color_grid=deq[:nc], endpoint_grid=deq[nc:])
    mm, ff = mismatch(mat.formats, got, ref)
    assert mm <= (0.001 if prec < 2 else 0.005) * ff
    for fmt, a, r in zip(mat.formats, got, ref):
        np.testing.assert_array_equal(a[:, :2 if fmt == 4 else 4], r[:, :2 if fmt == 4 else 4])   # endpoints
        if fmt == 1:
            c0, c1, codes = obc.bc1_unpack(a)
            assert np.all(c0 == c1) and np.all(codes == 0)
        else:
            r0, r1, _ = obc.bc4_unpack(a)
            assert np.all(r0 == r1)


def test_empty_block_list():
    mat, desc, odesc, params = max_case()
    m = nt.Model(desc)
    m.set_params(_dev(nt.configs.flatten(desc, params)))
    m.export(grid_bits=8, weight_prec=1)
    lay = m.layout
    e = torch.zeros(1, lay.out_endpoint, device=DEV)
    c = torch.zeros(1, 16, lay.out_color, device=DEV)
    m.forward(torch.empty(0, dtype=torch.int32, device=DEV), e, c)
    torch.cuda.synchronize()
    assert float(e.abs().sum()) == 0.0 and float(c.abs().sum()) == 0.0


def test_bounded_wait_gives_up_and_context_survives():
    # the failure path of every MMA wait: an mbarrier that nothing completes, polled with the
    # kernels' bounded loop under a small limit, gives up with NTBC_ETIMEOUT, and the GPU
    # context stays usable (a normal inference right after matches one from before)
    desc, odesc = descs.case_descs(nt, [nt.BC1, nt.BC4], 64, 3, 4, 16, 2, "selu")
    p0 = descs.init_params(odesc, 0)
    model = nt.Model(desc)
    model.set_params(torch.from_numpy(nt.configs.flatten(desc, synth.random_params_like(p0, seed=1))).to("cuda"))
    model.export(grid_bits=8, weight_prec=nt.PREC_FP16)
    outs = [torch.empty(16 * 16 * 8, dtype=torch.uint8, device="cuda") for _ in range(2)]
    model.infer_to_bc(outs)
    before = [o.clone() for o in outs]
    for polls in (1, 1 << 12, 1 << 16):
        status, sec = nt.ntbc_wait_probe(polls)
        assert status == 4, nt.STATUS_NAMES.get(status, status)
        assert 0.0 <= sec < 10.0
    for o in outs:
        o.zero_()
    model.infer_to_bc(outs)
    torch.cuda.synchronize()
    for a, b in zip(before, outs):
        assert torch.equal(a, b)


def test_nonfinite_loss_is_reported_and_the_next_encode_works():
    # a diverged encode, injected on the host (NTBC_FAULT=nan poisons the finalised losses):
    # ntbc_train returns NTBC_ENONFINITE instead of a silent NaN model; without the injection
    # the same call on a fresh model succeeds with finite losses
    import os
    mat = synth.make_material("nan", 32, ["sine_rgb", "sine_r"], 0)
    desc, odesc = descs.case_descs(nt, mat.formats, 32, 3, 4, 8, 2, "selu")
    p0 = descs.init_params(odesc, 0)
    tex = [_dev(t) for t in mat.textures]
    refs = [_dev(obc.encode(f, t, 32, 32)) for f, t in zip(mat.formats, mat.textures)]
    material = nt.Material.make(32, 32, mat.formats, tex, refs)
    cfg = nt.TrainConfig.make(steps=3, batch_texels=256, seed=0, precision=nt.TRAIN_BF16)
    m = nt.Model(desc)
    m.set_params(_dev(nt.configs.flatten(desc, p0)))
    os.environ["NTBC_FAULT"] = "nan"
    try:
        with pytest.raises(nt.NTBCError) as e:
            m.train(material, cfg)
        assert e.value.status == 5 and "non-finite" in str(e.value)
    finally:
        del os.environ["NTBC_FAULT"]
    m2 = nt.Model(desc)
    m2.set_params(_dev(nt.configs.flatten(desc, p0)))
    assert all(np.isfinite(m2.train(material, cfg)))


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_smallest_material_matches_oracle(prec):
    # 8x8 texels = 2x2 blocks: one partial 8-block tile of one partial work unit
    mat = synth.make_material("tiny8", 8, ["sine_rgb", "sine_r"], 4)
    desc, odesc = descs.case_descs(nt, mat.formats, 8, 2, 2, 8, 2, "selu")
    params = synth.random_params_like(descs.init_params(odesc, 4), seed=5)
    m = nt.Model(desc)
    m.set_params(_dev(nt.configs.flatten(desc, params)))
    m.export(grid_bits=0, weight_prec=prec)
    outs = [torch.empty(4 * 8, dtype=torch.uint8, device=DEV) for _ in mat.formats]
    m.infer_to_bc(outs)
    torch.cuda.synchronize()
    pw = dict(params)
    if prec:
        for k in ("color_mlp", "endpoint_mlp"):
            pw[k] = [(W.astype(np.float16).astype(np.float64), b.astype(np.float16).astype(np.float64)) for W, b in params[k]]
    ref = ont.infer_blocks(odesc, pw)
    got = [o.cpu().numpy().reshape(-1, 8) for o in outs]
    mm, ff = mismatch(mat.formats, got, ref)
    assert mm <= (0.005 if prec == 2 else 0.001) * ff + 1, (mm, ff)
