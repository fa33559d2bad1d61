"""The 1024^2 three-texture material (diffuse + normal BC1, roughness BC4; 8 levels 16..512,
3 x 64 SELU, FP32 grids): a 5k-step encode at 2^16 texels per step with the FP32 kernels and
with the BF16 tensor-core pass, then inference with FP32 weights (SIMT) and FP16 weights
(tensor cores) checked against the FP64 oracle on sampled blocks of the trained model."""
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


@pytest.fixture(scope="module")
def trained():
    w = nt.configs.WORKLOADS["mat1k"]
    mat = synth.material_1k(seed=0)
    side = mat.width
    desc, odesc = descs.case_descs(nt, mat.formats, side, w.levels, w.min_res, w.max_res, 3, "selu")
    p0 = descs.init_params(odesc, 0)
    tex_d = [_dev(t) for t in mat.textures]
    nblk = (side // 4) ** 2
    refs = [torch.empty(nblk * 8, dtype=torch.uint8, device=DEV) for _ in mat.formats]
    for t, fmt in enumerate(mat.formats):
        nt.bc_reference_encode(fmt, tex_d[t], side, side, refs[t])
    material = nt.Material.make(side, side, mat.formats, tex_d, refs)

    def psnrs(model, weight_prec):
        model.export(grid_bits=0, weight_prec=weight_prec)
        outs = [torch.empty(nblk * 8, dtype=torch.uint8, device=DEV) for _ in mat.formats]
        model.infer_to_bc(outs)
        torch.cuda.synchronize()
        return [obc.psnr(obc.decode(f, o.cpu().numpy(), side, side), t) for f, o, t in zip(mat.formats, outs, mat.textures)], outs

    models = {}
    untrained = None
    for prec in (nt.TRAIN_FP32, nt.TRAIN_BF16):
        m = nt.Model(desc)
        m.set_params(_dev(nt.configs.flatten(desc, p0)))
        if untrained is None:
            untrained = psnrs(m, nt.PREC_FP32)[0]
        losses = m.train(material, nt.TrainConfig.make(steps=w.steps, batch_texels=w.batch_texels, seed=0, precision=prec))
        assert all(np.isfinite(losses))
        models[prec] = m
    ref = [obc.psnr(obc.decode(f, r.cpu().numpy(), side, side), t) for f, r, t in zip(mat.formats, refs, mat.textures)]
    return dict(mat=mat, desc=desc, odesc=odesc, models=models, psnrs=psnrs, untrained=untrained, ref=ref, keep=(tex_d, refs))


def test_encode_fp32_and_bf16_gain_and_agree(trained):
    p32 = trained["psnrs"](trained["models"][nt.TRAIN_FP32], nt.PREC_FP32)[0]
    p16 = trained["psnrs"](trained["models"][nt.TRAIN_BF16], nt.PREC_FP32)[0]
    print("PSNR FP32 encode", np.round(p32, 3), "BF16 encode", np.round(p16, 3))
    for u, a, b, r in zip(trained["untrained"], p32, p16, trained["ref"]):
        assert a > u + 8.0 and b > u + 8.0
        assert a < r and b < r
        assert abs(a - b) < 0.5, (a, b)


def test_inference_fp32_and_fp16_match_oracle_on_trained_weights(trained):
    mat, desc = trained["mat"], trained["desc"]
    m = trained["models"][nt.TRAIN_BF16]
    flat = torch.empty(m.n_params, device=DEV)
    m.get_params(flat)
    odesc = trained["odesc"]
    params = descs.params_from_flat(odesc, flat.cpu().numpy())
    ids = np.sort(np.random.default_rng(1).choice(odesc.n_blocks, 500, replace=False))
    out = {}
    for prec in (nt.PREC_FP32, nt.PREC_FP16):
        psnr, outs = trained["psnrs"](m, prec)
        pw = params
        if prec == nt.PREC_FP16:
            pw = dict(params)
            for k in ("color_mlp", "endpoint_mlp"):
                pw[k] = [(W.astype(np.float16).astype(np.float64), b.astype(np.float16).astype(np.float64))
                         for W, b in params[k]]
        lay = m.layout
        e = torch.empty(len(ids), lay.out_endpoint, device=DEV)
        c = torch.empty(len(ids), 16, lay.out_color, device=DEV)
        m.forward(_dev(ids.astype(np.int32)), e, c)
        torch.cuda.synchronize()
        er, cr = ont.forward_blocks(odesc, pw, ids)
        np.testing.assert_allclose(e.cpu().numpy(), er, rtol=1e-3, atol=1e-6)
        np.testing.assert_allclose(c.cpu().numpy(), cr, rtol=1e-3, atol=1e-6)
        ref_blocks = ont.infer_blocks(odesc, pw, block_ids=ids)
        mism = fields = 0
        for t, fmt in enumerate(mat.formats):
            unpack = obc.bc1_unpack if fmt == 1 else obc.bc4_unpack
            a0, a1, ac = unpack(outs[t].cpu().numpy().reshape(-1, 8)[ids])
            b0, b1, bc_ = unpack(ref_blocks[t])
            mism += int((a0 != b0).sum() + (a1 != b1).sum() + (ac != bc_).sum())
            fields += len(ids) * 18
        assert mism <= 0.001 * fields
        out[prec] = psnr
    for a, b in zip(out[nt.PREC_FP32], out[nt.PREC_FP16]):
        assert abs(a - b) < 0.05, (a, b)
