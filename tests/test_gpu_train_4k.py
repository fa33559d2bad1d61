"""Training-gradient parity at the encode step's launch configuration: the 4096^2 mat4k model
(2 BC1 + 2 BC4 textures, 12 colour levels 16..2048 with their endpoint levels, 3 x 64 SELU)
and one step's batch of 16,384 sampled blocks (2^18 texels: 2,048 colour tiles over the
warpgroups of a full grid, 128 endpoint tiles), at the end-of-schedule temperature T = 0.01
with 8-bit QAT, in both training arithmetics. The reference targets are the oracle encoder's,
for the sampled blocks only (a step reads no other block).

Bars. The FP32 kernels: 2e-3 per tensor against FP64. The BF16 pass against the oracle's mode
of its arithmetic: 5e-3 on the MLP tensors; on the grids, per level, 2e-2 in full and 2.5e-3
once the largest 0.1 % of the level's vertex differences are set aside. The reason is BF16
rounding flips. A colour activation whose FP32 value (kernel) and FP64 value (oracle) fall on
either side of a BF16 rounding boundary moves by one BF16 step; the straight-through softmax
amplifies that 1/T, so that texel's grid gradient moves by a large fraction. A step of 2^18
texels rounds ~50 M activations, so a handful of texels flip, and each touches four vertices
per level that few other texels touch at the fine levels. Measured: the largest 0.1 % of the
differences carry 95-100 % of each fine level's error norm, and at T = 1 the grid errors are
10-20x smaller. The small-model tests, with no flips, hold every tensor to 5e-3. Against plain
FP64 the BF16 arithmetic itself (the oracle's mode measures the same) is ~0.18 off on the
finest colour level at this batch; the bounds below carry that figure with margin.
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
T = 0.01
QAT = 8
BLOCKS = 16384
# the BF16 pass against plain FP64 at T = 0.01 on this batch (measured: colour grid 0.183,
# colour MLP 0.031, endpoint grid 0.008, endpoint MLP 0.003; the oracle's mode alike)
FP64_BOUND_BF16 = {"color_grid": 0.25, "color_mlp": 0.15, "endpoint_grid": 0.03, "endpoint_mlp": 0.03}
FLIP_SHARE = 1e-3          # the largest differences of a grid level set aside
GRID_FULL, GRID_REST, MLP_BAR = 2e-2, 2.5e-3, 5e-3


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).ravel()).to(DEV)


def rel_err(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def grad_errors(got, want):
    errs = {}
    for key in ("color_grid", "endpoint_grid"):
        errs[key] = max(rel_err(a, b) for a, b in zip(got[key], want[key]))
    for key in ("color_mlp", "endpoint_mlp"):
        errs[key] = max(max(rel_err(aW, bW), rel_err(ab, bb)) for (aW, ab), (bW, bb) in zip(got[key], want[key]))
    return errs


@pytest.fixture(scope="module")
def case():
    w = nt.configs.WORKLOADS["mat4k"]
    mat = synth.material_4k(seed=0)
    side = mat.width
    desc, odesc = descs.case_descs(nt, mat.formats, side, w.levels, w.min_res, w.max_res, 3, "selu")
    params = synth.random_params_like(descs.init_params(odesc, 0), seed=1)
    nblk = (side // 4) ** 2
    ids = np.random.default_rng(5).integers(0, nblk, BLOCKS)
    sampled = np.unique(ids)
    refs = []
    for fmt, tex in zip(mat.formats, mat.textures):
        blk = obc.to_blocks(tex, side, side)[sampled]
        full = np.zeros((nblk, 8), np.uint8)
        full[sampled] = obc.bc1_encode_blocks(blk) if fmt == obc.BC1 else obc.bc4_encode_blocks(blk[..., 0])
        refs.append(full)
    L64, g64 = ont.losses_and_grads(odesc, params, mat.textures, refs, ids, T=T, qat_bits=QAT)
    return dict(mat=mat, desc=desc, odesc=odesc, params=params, ids=ids, refs=refs, side=side, L64=L64, g64=g64)


def gpu_step(c, precision):
    side = c["side"]
    tex_d = [_dev(t) for t in c["mat"].textures]
    ref_d = [_dev(r) for r in c["refs"]]
    material = nt.Material.make(side, side, c["mat"].formats, tex_d, ref_d)
    model = nt.Model(c["desc"])
    model.set_params(_dev(nt.configs.flatten(c["desc"], c["params"])))
    grads = torch.empty(model.n_params, device=DEV)
    losses = torch.empty(6, device=DEV)
    model.train_grads(material, _dev(c["ids"].astype(np.int32)), grads, losses, qat_bits=QAT, temperature=T,
                      precision=precision)
    torch.cuda.synchronize()
    return losses.cpu().numpy(), descs.params_from_flat(c["odesc"], grads.cpu().numpy())


def grid_rest_errors(got, want, key):
    """Per level: the relative error once the largest FLIP_SHARE of the level's nonzero vertex
    differences are set aside."""
    out = []
    for a, b in zip(got[key], want[key]):
        a = np.asarray(a, np.float64).ravel()
        b = np.asarray(b, np.float64).ravel()
        d = np.sort(np.abs(a - b))
        k = int(np.ceil(FLIP_SHARE * np.count_nonzero((a != 0) | (b != 0))))
        out.append(float(np.linalg.norm(d[:d.size - k]) / max(np.linalg.norm(b), 1e-30)))
    return out


def loss_list(L):
    return [L["L_e"], L["L_cd_endpoint"], L["L_c"], L["L_cd_color"], L["L_endpoint"], L["L_color"]]


def test_fp32_gradients_at_the_encode_launch_configuration(case):
    losses, g = gpu_step(case, nt.TRAIN_FP32)
    np.testing.assert_allclose(losses, loss_list(case["L64"]), rtol=2e-4)
    errs = grad_errors(g, case["g64"])
    print("FP32 vs FP64", errs)
    assert max(errs.values()) <= 2e-3, errs


def test_bf16_gradients_at_the_encode_launch_configuration(case):
    losses, g = gpu_step(case, nt.TRAIN_BF16)
    c = case
    Lm, gm = ont.losses_and_grads(c["odesc"], c["params"], c["mat"].textures, c["refs"], c["ids"], T=T, qat_bits=QAT,
                                  bf16=True)
    np.testing.assert_allclose(losses, loss_list(Lm), rtol=2e-3)
    errs = grad_errors(g, gm)
    errs64 = grad_errors(g, c["g64"])
    rest = {key: max(grid_rest_errors(g, gm, key)) for key in ("color_grid", "endpoint_grid")}
    print("BF16 vs the oracle's mode", errs, "without the largest 0.1 %", rest, "vs FP64", errs64)
    assert errs["color_mlp"] <= MLP_BAR and errs["endpoint_mlp"] <= MLP_BAR, errs
    for key in ("color_grid", "endpoint_grid"):
        assert errs[key] <= GRID_FULL, (key, errs)
        assert rest[key] <= GRID_REST, (key, rest)
    for key, bound in FP64_BOUND_BF16.items():
        assert errs64[key] <= bound, (key, errs64)
