"""Fused tensor-core training pass (NTBC_TRAIN_BF16) against the oracle: losses and
gradients of one step on the same weights and batch, ragged tiles, several tiles per
warpgroup, QAT, and a full encode that gains over the untrained network like the FP32 path.

The comparison is with the oracle's mode for this arithmetic: the colour network's
matrix-product operands (features, weights, biases, activations, deltas) rounded to BF16; the
endpoint network's forward on exact operands (the kernel splits each into BF16 hi + lo parts,
~2^-16 relative) and its backward on BF16 operands; products and sums exact. What is left is
FP32 against FP64 arithmetic, so the bar is 5e-3 per tensor (2e-3 on the losses). Against the
plain FP64 oracle the BF16 rounding itself shows, amplified by the straight-through argmax
(1/T inside softmax(d / T)) where it enters a forward: a few percent on the colour network at
T = 0.01, about 1 % on the endpoint network, whose forward is split (with BF16 forward operands
it reached ~30 % there). The oracle's mode reproduces those figures, so they are the
arithmetic's, not the kernel's. They are asserted too, per network and temperature, at the
bounds FP64_BOUND states (measured errors with margin), so a kernel change that makes the
arithmetic worse than the oracle's mode predicts cannot pass unnoticed.
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
TOL_GRAD = 5e-3
TOL_LOSS = 2e-3
# relative gradient error of the BF16 pass against the plain FP64 oracle, per tensor group and
# temperature: the BF16 operand rounding (2^-9) amplified by the straight-through softmax
# (the oracle's mode measures at most 0.034 on the colour network, 0.012 on the endpoint one)
FP64_BOUND = {1.0: {"color_grid": 0.06, "color_mlp": 0.06, "endpoint_grid": 0.03, "endpoint_mlp": 0.03},
              0.01: {"color_grid": 0.15, "color_mlp": 0.15, "endpoint_grid": 0.03, "endpoint_mlp": 0.03}}


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).ravel()).to(DEV)


def setup(side=32, kinds=("sine_rgb", "sine_r", "sine_r", "sine_rgb"), levels=3, lo=4, hi=9, hidden=2, act="selu",
          seed=3):
    mat = synth.make_material("trn", side, list(kinds), seed)
    desc, odesc = descs.case_descs(nt, mat.formats, side, levels, lo, hi, hidden, act)
    params = synth.random_params_like(descs.init_params(odesc, seed), seed=seed + 1, grid_scale=0.5)
    refs = [obc.encode(f, t, side, side) for f, t in zip(mat.formats, mat.textures)]
    tex_d = [_dev(t) for t in mat.textures]
    ref_d = [_dev(r) for r in refs]
    material = nt.Material.make(side, side, mat.formats, tex_d, ref_d)
    model = nt.Model(desc)
    model.set_params(_dev(nt.configs.flatten(desc, params)))
    return dict(mat=mat, desc=desc, odesc=odesc, params=params, refs=refs, material=material, model=model,
                keep=(tex_d, ref_d))


def rel_err(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def grad_errors(desc, gg, g):
    errs = {}
    for key in ("color_grid", "endpoint_grid"):
        errs[key] = max(rel_err(a, b) for a, b in zip(gg[key], g[key]))
    for key in ("color_mlp", "endpoint_mlp"):
        errs[key] = max(max(rel_err(aW, bW), rel_err(ab, bb)) for (aW, ab), (bW, bb) in zip(gg[key], g[key]))
    return errs


def check_step(s, ids, qat, T=0.01):
    model = s["model"]
    grads = torch.empty(model.n_params, device=DEV)
    losses = torch.empty(6, device=DEV)
    model.train_grads(s["material"], _dev(ids.astype(np.int32)), grads, losses, qat_bits=qat, temperature=T,
                      precision=nt.TRAIN_BF16)
    torch.cuda.synchronize()
    L, g = ont.losses_and_grads(s["odesc"], s["params"], s["mat"].textures, s["refs"], ids, T=T, qat_bits=qat, bf16=True)
    want_l = [L["L_e"], L["L_cd_endpoint"], L["L_c"], L["L_cd_color"], L["L_endpoint"], L["L_color"]]
    np.testing.assert_allclose(losses.cpu().numpy(), want_l, rtol=TOL_LOSS)
    gg = descs.params_from_flat(s["odesc"], grads.cpu().numpy())
    errs = grad_errors(s["desc"], gg, g)
    assert max(errs.values()) < TOL_GRAD, errs
    _, g64 = ont.losses_and_grads(s["odesc"], s["params"], s["mat"].textures, s["refs"], ids, T=T, qat_bits=qat)
    errs64 = grad_errors(s["desc"], gg, g64)
    for key, bound in FP64_BOUND[T].items():
        assert errs64[key] <= bound, (key, T, errs64)
    return errs, errs64


@pytest.mark.parametrize("T", [1.0, 0.01])
@pytest.mark.parametrize("act,hidden,qat", [("selu", 2, 0), ("relu", 2, 0), ("selu", 3, 8), ("selu", 1, 4)])
def test_bf16_grads_match_oracle(act, hidden, qat, T):
    s = setup(act=act, hidden=hidden)
    ids = np.array([0, 5, 17, 33, 63, 40, 5, 22, 9, 11, 60, 2, 30], np.int64)   # 208 texels: ragged second tile
    print(act, hidden, qat, T, check_step(s, ids, qat, T))


@pytest.mark.parametrize("T,qat", [(1.0, 0), (0.01, 0), (0.01, 8)])
def test_bf16_many_tiles_per_group(T, qat):
    # 4096 sampled blocks: 512 colour tiles over at most 304 warpgroups, so groups accumulate
    # weight gradients across tiles in TMEM; 32 endpoint tiles; at the training temperature too
    s = setup(side=128, levels=4, lo=8, hi=32, hidden=3)
    ids = np.random.default_rng(0).integers(0, 32 * 32, 4096)
    print(T, qat, check_step(s, ids, qat, T))


def test_bf16_training_gains_over_untrained_network():
    mat = synth.tiny_material()
    w = nt.configs.WORKLOADS["tiny256"]
    desc, odesc = descs.case_descs(nt, mat.formats, mat.width, w.levels, w.min_res, w.max_res, w.hidden_layers, "relu")
    p0 = descs.init_params(odesc, 0)
    tex_d = [_dev(t) for t in mat.textures]
    refs = [torch.empty(64 * 64 * 8, dtype=torch.uint8, device=DEV) for _ in mat.formats]
    for t, fmt in enumerate(mat.formats):
        nt.bc_reference_encode(fmt, tex_d[t], 256, 256, refs[t])
    material = nt.Material.make(256, 256, mat.formats, tex_d, refs)

    def run(precision):
        model = nt.Model(desc)
        model.set_params(_dev(nt.configs.flatten(desc, p0)))
        model.export(grid_bits=0, weight_prec=nt.PREC_FP32)
        before = psnrs(model)
        losses = model.train(material, nt.TrainConfig.make(steps=w.steps, batch_texels=w.batch_texels, seed=1,
                                                           precision=precision))
        assert all(np.isfinite(losses))
        return before, psnrs(model)

    def psnrs(model):
        model.export(grid_bits=0, weight_prec=nt.PREC_FP32)
        outs = [torch.empty(64 * 64 * 8, dtype=torch.uint8, device=DEV) for _ in mat.formats]
        model.infer_to_bc(outs)
        torch.cuda.synchronize()
        return [obc.psnr(obc.decode(f, o.cpu().numpy(), 256, 256), t) for f, o, t in zip(mat.formats, outs, mat.textures)]

    before, bf16 = run(nt.TRAIN_BF16)
    _, fp32 = run(nt.TRAIN_FP32)
    ref = [obc.psnr(obc.decode(f, r.cpu().numpy(), 256, 256), t) for f, r, t in zip(mat.formats, refs, mat.textures)]
    for b, a, f, r in zip(before, bf16, fp32, ref):
        assert a > b + 5.0 and a < r
        assert abs(a - f) < 1.0, (a, f)
