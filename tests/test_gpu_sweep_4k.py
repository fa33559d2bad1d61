"""Inference precision sweep on trained weights of the 4096^2 four-texture material (2 BC1 +
2 BC4, 12 levels 16..2048, 3 x 64 SELU): grids u8 and u4 (each encoded with its own QAT width,
the full 20k + 2k-step schedule at 2^18 texels) x MLP weights FP32 (SIMT kernel), FP16 with
split activations, FP16 with FP16 activations (the paper's half precision, Sec. 3.3), FP8 E4M3
storage, and FP8 arithmetic (E4M3 weights and activations on kind::f8f6f4 MMAs). For each: the largest relative error of the raw outputs against the FP64 oracle with
the same stored weights, the field mismatch after quantisation and the decoded PSNR, on 2000
sampled blocks, against the bars of each mode; the error against the FP64 network on the FP32
master weights (what the storage precision gives up) is printed beside it.

The weights come from the library's own encode on the GPU (the oracle cannot train a 4k
material in test time); both sides then evaluate the same stored model. Run with -s to see
the table."""
import json

import numpy as np
import pytest
import torch

import descs
import synth
from oracle import bc as obc, ntbc as ont

nt = pytest.importorskip("paper_2407_09543_gb300")
pytestmark = pytest.mark.gpu
DEV = "cuda"
SIDE = 4096
STEPS = 20000
# largest relative output error against the FP64 oracle with the same stored weights, and the
# field-mismatch bar, per mode (the split and FP32 modes hold the 1e-3 and 0.1 % bars; FP16
# activations carry four FP16 roundings amplified by the trained network: about 1e-2 measured)
BARS = {"fp32": (1e-3, 0.001), "fp16": (1e-3, 0.001), "fp16_fast": (2.5e-2, 0.02), "fp8_e4m3": (1e-3, 0.001)}
# FP8 arithmetic (E4M3 activations, kind::f8f6f4): against the FP64 oracle of the same
# arithmetic, outputs agree within 1e-3 relative except where an FP32 value lands on the other
# side of an E4M3 rounding boundary than the FP64 one (a flip); bars: the fraction of outputs
# beyond 1e-3 relative, and the field mismatch (a flipped output moves by up to ~1e-2)
FP8_MMA_BARS = (0.005, 0.005)


@pytest.fixture(scope="module")
def material():
    mat = synth.material_4k(seed=0, side=SIDE)
    w = nt.configs.WORKLOADS["mat4k"]
    desc, od = descs.case_descs(nt, mat.formats, SIDE, w.levels, w.min_res, w.max_res, 3, "selu")
    tex_d = [torch.from_numpy(t.ravel()).to(DEV) for t in mat.textures]
    nblk = (SIDE // 4) ** 2
    refs = [torch.empty(nblk * 8, dtype=torch.uint8, device=DEV) for _ in mat.formats]
    for t, fmt in enumerate(mat.formats):
        nt.bc_reference_encode(fmt, tex_d[t], SIDE, SIDE, refs[t], refine=2)
    torch.cuda.synchronize()
    return dict(mat=mat, desc=desc, od=od, tex=tex_d, refs=refs,
                material=nt.Material.make(SIDE, SIDE, mat.formats, tex_d, refs))


def _psnr(mat, tex_d, blocks):
    """Decoded PSNR per texture (reported, not asserted): the library's decoder, bit-exact with
    the oracle's (test_gpu_codec), on the device."""
    out = []
    for f, b, src in zip(mat.formats, blocks, tex_d):
        dec = torch.empty_like(src)
        nt.bc_decode(f, b, SIDE, SIDE, dec)
        mse = float(((dec.double() - src.double()) / 255.0).pow(2).mean())
        out.append(round(10.0 * np.log10(1.0 / mse), 3))
    return out


@pytest.mark.parametrize("bits", [8, 4])
def test_precision_sweep_on_trained_4k_weights(material, bits):
    mat, desc, od = material["mat"], material["desc"], material["od"]
    nblk = (SIDE // 4) ** 2
    model = nt.Model(desc)
    model.set_params(torch.from_numpy(nt.configs.flatten(desc, descs.init_params(od, 0))).to(DEV))
    model.train(material["material"], nt.TrainConfig.make(steps=STEPS, batch_texels=1 << 18, qat_fraction=0.1,
                                                           grid_bits=bits, seed=0, precision=nt.TRAIN_BF16))
    flat = torch.empty(model.n_params, device=DEV)
    model.get_params(flat)
    params = descs.params_from_flat(od, flat.cpu().numpy())
    codes, sc, zr = ont.export_grid(params["color_grid"] + params["endpoint_grid"], bits)
    deq = ont.dequantize_grid(codes, sc, zr)
    nc = len(od.color_res)
    ids = np.sort(np.random.default_rng(0).choice(nblk, 2000, replace=False))
    er32, cr32 = ont.forward_blocks(od, params, ids, color_grid=deq[:nc], endpoint_grid=deq[nc:])
    rows = []
    for name, prec in (("fp32", nt.PREC_FP32), ("fp16", nt.PREC_FP16), ("fp16_fast", nt.PREC_FP16_FAST),
                       ("fp8_e4m3", nt.PREC_FP8), ("fp8_e4m3_mma", nt.PREC_FP8_MMA)):
        model.export(grid_bits=bits, weight_prec=prec)
        aexps = None
        if prec in (nt.PREC_FP8, nt.PREC_FP8_MMA):
            pw = ont.fp8_params(params)[0]
            if prec == nt.PREC_FP8_MMA:
                aexps = ont.fp8_activation_exponents(od, pw, color_grid=deq[:nc], endpoint_grid=deq[nc:])
        else:
            pw = dict(params)
            for k in ("color_mlp", "endpoint_mlp"):
                pw[k] = [((W.astype(np.float16) if prec else W).astype(np.float64),
                          (b.astype(np.float16) if prec else b).astype(np.float64)) for W, b in params[k]]
        er, cr = ont.forward_blocks(od, pw, ids, color_grid=deq[:nc], endpoint_grid=deq[nc:], fp8_act=aexps)
        lay = model.layout
        e = torch.empty(len(ids), lay.out_endpoint, device=DEV)
        c = torch.empty(len(ids), 16, lay.out_color, device=DEV)
        model.forward(torch.from_numpy(ids.astype(np.int32)).to(DEV), e, c)
        outs = [torch.empty(nblk * 8, dtype=torch.uint8, device=DEV) for _ in mat.formats]
        model.infer_to_bc(outs)
        torch.cuda.synchronize()
        eg, cg = e.cpu().numpy().astype(np.float64), c.cpu().numpy().astype(np.float64)
        rel = max(float(np.max(np.abs(eg - er) / np.abs(er))), float(np.max(np.abs(cg - cr) / np.abs(cr))))
        rel32 = max(float(np.max(np.abs(eg - er32) / np.abs(er32))), float(np.max(np.abs(cg - cr32) / np.abs(cr32))))
        flips = float(np.mean(np.concatenate([(np.abs(eg - er) > 1e-3 * np.abs(er)).ravel(),
                                              (np.abs(cg - cr) > 1e-3 * np.abs(cr)).ravel()])))
        ref_blocks = ont.infer_blocks(od, pw, block_ids=ids, color_grid=deq[:nc], endpoint_grid=deq[nc:], fp8_act=aexps)
        host = [o.cpu().numpy().reshape(-1, 8) for o in outs]
        mism = fields = 0
        for t, fmt in enumerate(mat.formats):
            unpack = obc.bc1_unpack if fmt == 1 else obc.bc4_unpack
            a, b = unpack(host[t][ids]), unpack(ref_blocks[t])
            mism += sum(int((x != y).sum()) for x, y in zip(a, b))
            fields += len(ids) * 18
        rows.append({"grid_bits": bits, "mlp": name, "max_rel_err_vs_fp64": rel,
                     "outputs_beyond_1e-3": flips, "max_rel_err_vs_fp64_fp32_weights": rel32,
                     "field_mismatch": mism / fields, "psnr_db": _psnr(mat, material["tex"], outs)})
        if prec == nt.PREC_FP8_MMA:
            assert flips <= FP8_MMA_BARS[0] and mism <= FP8_MMA_BARS[1] * fields, rows[-1]
        else:
            bar_rel, bar_mism = BARS[name]
            assert rel <= bar_rel and mism <= bar_mism * fields, rows[-1]
    model.close()
    print(json.dumps({"mode": "sweep", "workload": f"mat4k {SIDE}x{SIDE}", "train_steps": STEPS, "rows": rows}))
