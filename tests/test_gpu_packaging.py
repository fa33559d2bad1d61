"""Conservative packaging (Sec. 4.1): one model for the BC1 textures and one for the BC4
textures. Single-format models match the FP64 oracle like the aggressive one; the two
models of a material decode in one batched launch exactly as their own launches do; and a
conservative encode gains over its untrained networks."""
import numpy as np
import pytest
import torch

import descs
import synth
from oracle import bc as obc, ntbc as ont

nt = pytest.importorskip("paper_2407_09543_gb300")
pytestmark = pytest.mark.gpu
DEV = "cuda"


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).ravel()).to(DEV)


@pytest.mark.parametrize("kinds", [("sine_rgb", "sine_rgb"), ("sine_r", "sine_r", "sine_r")])
def test_single_format_model_matches_oracle(kinds):
    side = 64
    mat = synth.make_material("pkg", side, list(kinds), 2)
    desc, odesc = descs.case_descs(nt, mat.formats, side, 4, 4, 32, 3, "selu")
    params = synth.random_params_like(descs.init_params(odesc, 2), seed=3)
    m = nt.Model(desc)
    m.set_params(_dev(nt.configs.flatten(desc, params)))
    m.export(grid_bits=8, weight_prec=nt.PREC_FP16)
    oc, os_, oz = ont.export_grid(params["color_grid"] + params["endpoint_grid"], 8)
    deq = ont.dequantize_grid(oc, os_, oz)
    nc = desc.color_levels
    p16 = dict(params)
    for k in ("color_mlp", "endpoint_mlp"):
        p16[k] = [(W.astype(np.float16).astype(np.float64), b.astype(np.float16).astype(np.float64)) for W, b in params[k]]
    ids = np.arange(odesc.n_blocks)
    lay = m.layout
    e = torch.empty(len(ids), lay.out_endpoint, device=DEV)
    c = torch.empty(len(ids), 16, lay.out_color, device=DEV)
    m.forward(_dev(ids.astype(np.int32)), e, c)
    torch.cuda.synchronize()
    er, cr = ont.forward_blocks(odesc, p16, ids, color_grid=deq[:nc], endpoint_grid=deq[nc:])
    np.testing.assert_allclose(e.cpu().numpy(), er, rtol=1e-3, atol=1e-6)
    np.testing.assert_allclose(c.cpu().numpy(), cr, rtol=1e-3, atol=1e-6)
    outs = [torch.empty(odesc.n_blocks * 8, dtype=torch.uint8, device=DEV) for _ in mat.formats]
    m.infer_to_bc(outs)
    ref = ont.infer_blocks(odesc, p16, color_grid=deq[:nc], endpoint_grid=deq[nc:])
    torch.cuda.synchronize()
    mism = fields = 0
    for fmt, o, rb in zip(mat.formats, outs, ref):
        unpack = obc.bc1_unpack if fmt == 1 else obc.bc4_unpack
        a0, a1, ac = unpack(o.cpu().numpy().reshape(-1, 8))
        b0, b1, bc_ = unpack(rb)
        mism += int((a0 != b0).sum() + (a1 != b1).sum() + (ac != bc_).sum())
        fields += a0.size * 18
    assert mism <= 0.001 * fields


def test_conservative_encode_and_batched_decode():
    side = 128
    mat = synth.make_material("cons", side, ["sine_rgb", "sine_r", "sine_rgb", "sine_r"], 4)
    tex_d = [_dev(t) for t in mat.textures]
    refs = [torch.empty((side // 4) ** 2 * 8, dtype=torch.uint8, device=DEV) for _ in mat.formats]
    for t, fmt in enumerate(mat.formats):
        nt.bc_reference_encode(fmt, tex_d[t], side, side, refs[t])
    groups = nt.configs.packaging_groups(mat.formats, "conservative")
    assert groups == [[0, 2], [1, 3]]
    models, outs, before = [], [], {}
    for g in groups:
        fm = [mat.formats[t] for t in g]
        desc, odesc = descs.case_descs(nt, fm, side, 4, 8, 64, 3, "selu")
        p0 = descs.init_params(odesc, 7)
        m = nt.Model(desc)
        m.set_params(_dev(nt.configs.flatten(desc, p0)))
        o = [torch.empty((side // 4) ** 2 * 8, dtype=torch.uint8, device=DEV) for _ in g]
        m.export(grid_bits=8, weight_prec=nt.PREC_FP16)
        m.infer_to_bc(o)
        torch.cuda.synchronize()
        for t, oo in zip(g, o):
            before[t] = obc.psnr(obc.decode(mat.formats[t], oo.cpu().numpy(), side, side), mat.textures[t])
        material = nt.Material.make(side, side, fm, [tex_d[t] for t in g], [refs[t] for t in g])
        m.train(material, nt.TrainConfig.make(steps=800, batch_texels=4096, qat_fraction=0.1, grid_bits=8, seed=1,
                                              precision=nt.TRAIN_BF16))
        m.export(grid_bits=8, weight_prec=nt.PREC_FP16)
        models.append(m)
        outs.append(o)
    # the two models of the material in one persistent launch == their own launches
    batch = nt.Batch(models, outs)
    batch.infer()
    torch.cuda.synchronize()
    got = [[oo.clone() for oo in o] for o in outs]
    for m, o in zip(models, outs):
        m.infer_to_bc(o)
    torch.cuda.synchronize()
    for go, o in zip(got, outs):
        for a, b in zip(go, o):
            assert torch.equal(a, b)
    gains = []
    for g, o in zip(groups, outs):
        for t, oo in zip(g, o):
            after = obc.psnr(obc.decode(mat.formats[t], oo.cpu().numpy(), side, side), mat.textures[t])
            ref = obc.psnr(obc.decode(mat.formats[t], refs[t].cpu().numpy(), side, side), mat.textures[t])
            assert after > before[t] + 1.0 and after < ref, (t, before[t], after, ref)
            gains.append(after - before[t])
    assert np.mean(gains) > 4.0, gains
    batch.close()
