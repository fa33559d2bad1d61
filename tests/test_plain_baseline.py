"""The plain FP32 comparison path (PyTorch eager, autograd with straight-through
estimators) against the oracle, on the CPU in float64: same losses, same gradients
(an autograd cross-check of the oracle's hand-written backward) and same blocks.
Texel coordinates are FP32 in the plain path, hence agreement to ~1e-8, not 1e-15."""
import numpy as np
import pytest
import torch

import synth
from baseline import plain_fp32 as pf
from oracle import bc as obc, ntbc as ont


def _case():
    mat = synth.make_material("plain", 32, ["sine_rgb", "sine_r", "sine_r", "sine_rgb"], 3)
    cres, eres = [4, 6, 9], [4, 6]
    od = ont.ModelDesc(32, 32, mat.formats, cres, eres, hidden_layers=2, activation="selu")
    p0 = synth.init_params(cres, eres, 2, od.mlp_dims("color"), od.mlp_dims("endpoint"), 3)
    p = synth.random_params_like(p0, seed=4, grid_scale=0.5)
    refs = [obc.encode(f, t, 32, 32) for f, t in zip(mat.formats, mat.textures)]
    return mat, cres, eres, od, p, refs


@pytest.mark.parametrize("qat", [0, 8])
def test_plain_losses_and_autograd_match_oracle(qat):
    mat, cres, eres, od, p, refs = _case()
    ids = np.array([0, 5, 17, 33, 63, 40, 5, 22])
    L, g = ont.losses_and_grads(od, p, mat.textures, refs, ids, qat_bits=qat)
    p64 = {k: ([np.asarray(x, np.float64) for x in v] if "grid" in k else
               [(np.asarray(W, np.float64), np.asarray(b, np.float64)) for W, b in v]) for k, v in p.items()}
    old = torch.get_default_dtype()
    torch.set_default_dtype(torch.float64)
    try:
        pm = pf.PlainModel(32, 32, mat.formats, cres, eres, p64, "selu", "cpu")
        for lst in (pm.color_grid, pm.endpoint_grid):
            for i, x in enumerate(lst):
                lst[i] = x.double().detach().requires_grad_()
        for lst in (pm.color_mlp, pm.endpoint_mlp):
            for i, (W, b) in enumerate(lst):
                lst[i] = (W.double().detach().requires_grad_(), b.double().detach().requires_grad_())
        ref_e = [torch.tensor(obc.reference_endpoints(f, r)) for f, r in zip(mat.formats, refs)]
        le, lc = pf.losses(pm, [torch.tensor(t) for t in mat.textures], ref_e, torch.tensor(ids), qat_bits=qat)
        (le + lc).backward()
    finally:
        torch.set_default_dtype(old)
    assert le.item() == pytest.approx(L["L_endpoint"], rel=1e-6)
    assert lc.item() == pytest.approx(L["L_color"], rel=1e-6)
    for a, b in zip(pm.color_grid + pm.endpoint_grid, g["color_grid"] + g["endpoint_grid"]):
        assert np.linalg.norm(a.grad.numpy() - b) <= 1e-5 * np.linalg.norm(b)
    for (W, bb), (gW, gb) in zip(pm.color_mlp + pm.endpoint_mlp, g["color_mlp"] + g["endpoint_mlp"]):
        assert np.linalg.norm(W.grad.numpy() - gW) <= 1e-5 * np.linalg.norm(gW)
        assert np.linalg.norm(bb.grad.numpy() - gb) <= 1e-5 * max(np.linalg.norm(gb), 1e-30)


def test_plain_blocks_match_oracle():
    mat, cres, eres, od, p, refs = _case()
    pm = pf.PlainModel(32, 32, mat.formats, cres, eres, p, "selu", "cpu")
    outs = pf.infer_to_bc(pm)
    ref = ont.infer_blocks(od, p)
    mism = sum(int((o.numpy() != r).any(1).sum()) for o, r in zip(outs, ref))
    assert mism <= 1
