"""GPU training path against the FP64 oracle: losses and gradients of one step on the
same weights and batch, Adam, the Philox sampler, and the learned-part gain of a
full encode (trained network vs the same network untrained)."""
import numpy as np
import pytest
import torch

import descs
import synth
from oracle import bc as obc, ntbc as ont, philox

nt = pytest.importorskip("paper_2407_09543_gb300")
pytestmark = pytest.mark.gpu
DEV = "cuda"


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).ravel()).to(DEV)


def setup(side=32, kinds=("sine_rgb", "sine_r", "sine_r", "sine_rgb"), levels=3, lo=4, hi=9, hidden=2, act="selu",
          seed=3, grid_scale=0.5):
    mat = synth.make_material("trn", side, list(kinds), seed)
    desc, odesc = descs.case_descs(nt, mat.formats, side, levels, lo, hi, hidden, act)
    p0 = descs.init_params(odesc, seed)
    params = synth.random_params_like(p0, seed=seed + 1, grid_scale=grid_scale) if grid_scale else p0
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


@pytest.mark.parametrize("act,hidden,qat", [("selu", 2, 0), ("relu", 2, 0), ("selu", 3, 8), ("selu", 1, 4)])
def test_grads_match_oracle(act, hidden, qat):
    s = setup(act=act, hidden=hidden)
    ids = np.array([0, 5, 17, 33, 63, 40, 5, 22], np.int32)        # repeats allowed (sampling with replacement)
    model = s["model"]
    grads = torch.empty(model.n_params, device=DEV)
    losses = torch.empty(6, device=DEV)
    model.train_grads(s["material"], _dev(ids), grads, losses, qat_bits=qat)
    torch.cuda.synchronize()
    L, g = ont.losses_and_grads(s["odesc"], s["params"], s["mat"].textures, s["refs"], ids, qat_bits=qat)
    got_l = losses.cpu().numpy()
    want_l = [L["L_e"], L["L_cd_endpoint"], L["L_c"], L["L_cd_color"], L["L_endpoint"], L["L_color"]]
    np.testing.assert_allclose(got_l, want_l, rtol=2e-4)
    gg = descs.params_from_flat(s["odesc"], grads.cpu().numpy())
    for key in ("color_grid", "endpoint_grid"):
        for a, b in zip(gg[key], g[key]):
            assert rel_err(a, b) < 2e-3, key
    for key in ("color_mlp", "endpoint_mlp"):
        for (aW, ab), (bW, bb) in zip(gg[key], g[key]):
            assert rel_err(aW, bW) < 2e-3, key
            assert rel_err(ab, bb) < 2e-3, key


def test_adam_step_matches_oracle():
    s = setup()
    model = s["model"]
    n = model.n_params
    rng = np.random.default_rng(0)
    flat0 = nt.configs.flatten(s["desc"], s["params"]).astype(np.float64)
    cfg = nt.TrainConfig.make(steps=100, batch_texels=128)
    grid_n = model.layout.grid_floats
    p = flat0.copy()
    m = np.zeros(n)
    v = np.zeros(n)
    for step in range(3):
        g = rng.normal(size=n).astype(np.float32)
        model.adam_step(_dev(g), step, 100, cfg)
        lr = np.where(np.arange(n) < grid_n, ont.learning_rate(step, 100, 0.01), ont.learning_rate(step, 100, 0.005))
        p, m, v = ont.adam_update(p, g.astype(np.float64), m, v, step, lr)
    out = torch.empty(n, device=DEV)
    model.get_params(out)
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), p, rtol=1e-5, atol=1e-7)


def test_sampler_bit_exact_with_oracle():
    ids = torch.empty(100003, dtype=torch.int32, device=DEV)
    for seed, step, nb in ((0, 0, 4096), (12345678901, 777, 1 << 20), (5, 3, 1000)):
        nt.ntbc_sample_blocks(seed, step, ids.numel(), nb, ids)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ids.cpu().numpy(), philox.sample_blocks(seed, step, ids.numel(), nb))


def test_training_gains_over_untrained_network():
    # the learned part: a full encode on the GPU (500 steps, 4096 texels per step,
    # 2 x 64 ReLU, 4 levels 16..128) beats the same network at initialisation and stays
    # below the reference BC encoder (the ordering of every row of the paper's tables)
    mat = synth.tiny_material()
    w = nt.configs.WORKLOADS["tiny256"]
    desc, odesc = descs.case_descs(nt, mat.formats, mat.width, w.levels, w.min_res, w.max_res, w.hidden_layers, "relu")
    p0 = descs.init_params(odesc, 0)
    tex_d = [_dev(t) for t in mat.textures]
    refs = [torch.empty(64 * 64 * 8, dtype=torch.uint8, device=DEV) for _ in mat.formats]
    for t, fmt in enumerate(mat.formats):
        nt.bc_reference_encode(fmt, tex_d[t], 256, 256, refs[t])
    material = nt.Material.make(256, 256, mat.formats, tex_d, refs)
    model = nt.Model(desc)
    model.set_params(_dev(nt.configs.flatten(desc, p0)))

    def psnrs():
        model.export(grid_bits=0, weight_prec=nt.PREC_FP32)
        outs = [torch.empty(64 * 64 * 8, dtype=torch.uint8, device=DEV) for _ in mat.formats]
        model.infer_to_bc(outs)
        torch.cuda.synchronize()
        return [obc.psnr(obc.decode(f, o.cpu().numpy(), 256, 256), t) for f, o, t in zip(mat.formats, outs, mat.textures)]

    before = psnrs()
    cfg = nt.TrainConfig.make(steps=w.steps, batch_texels=w.batch_texels, seed=1)
    losses = model.train(material, cfg)
    after = psnrs()
    ref = [obc.psnr(obc.decode(f, r.cpu().numpy(), 256, 256), t) for f, r, t in zip(mat.formats, refs, mat.textures)]
    assert all(np.isfinite(losses))
    for b, a, r in zip(before, after, ref):
        assert a > b + 5.0 and a < r


@pytest.mark.parametrize("precision", [0, 1])
def test_checkpoint_resume_matches_uninterrupted_encode(precision):
    """An encode split at a step, its checkpoint (FP32 master parameters, Adam moments, step)
    written out and loaded into a fresh model, then resumed, ends where an uninterrupted encode
    ends, up to the rounding order of the grid scatter's floating-point atomics, which makes
    uninterrupted encodes differ too; the checkpoint round trip itself is exact. Over a long
    encode the argmax can amplify that rounding into a different trajectory (uninterrupted
    encodes of 44 steps have measured from 0 to 0.9 % apart), so this encode is short: 4 steps
    and 2 QAT steps, resumed after step 3, so the resumed range crosses into the QAT phase. The
    bar is the larger of the spread of two uninterrupted encodes (x3) and a thousandth of the
    distance the encode moves the parameters: a resume that lost the Adam moments, the step or
    the phase lands a sizeable share of that distance away."""
    s = setup(grid_scale=0)
    desc, material = s["desc"], s["material"]
    flat0 = _dev(nt.configs.flatten(desc, s["params"]))
    cfg = nt.TrainConfig.make(steps=4, batch_texels=512, qat_fraction=0.5, grid_bits=8, warmup=2, seed=5,
                              precision=precision)
    split, total = 3, 6

    def fresh():
        m = nt.Model(desc)
        m.set_params(flat0)
        return m

    def params(m):
        out = torch.empty(m.n_params, device=DEV)
        m.get_params(out)
        torch.cuda.synchronize()
        return out.cpu().numpy().astype(np.float64)

    a, c = fresh(), fresh()
    a.train(material, cfg)
    c.train(material, cfg)
    first = fresh()
    first.train_range(material, cfg, 0, split)
    ck = torch.empty(first.checkpoint_size(), dtype=torch.uint8)
    first.checkpoint_save(ck)
    b = nt.Model(desc)
    assert b.checkpoint_load(ck) == split
    ck2 = torch.empty_like(ck)
    b.checkpoint_save(ck2)
    assert torch.equal(ck, ck2)
    losses = b.train_range(material, cfg, split, total)
    assert all(np.isfinite(losses))
    p0 = flat0.cpu().numpy().astype(np.float64)
    pa, pb, pc = params(a), params(b), params(c)
    moved = np.linalg.norm(pa - p0)
    assert moved > 0
    noise = np.linalg.norm(pa - pc)
    resumed = min(np.linalg.norm(pb - pa), np.linalg.norm(pb - pc))
    bar = max(3 * noise, 1e-3 * moved)
    assert resumed <= bar, (resumed, noise, moved)
    # control: the split's parameters resumed with other Adam moments (those of a one-step
    # history) land far outside the bar, so it tells a resume that lost the optimizer state
    flat_split = torch.empty(first.n_params, device=DEV)
    first.get_params(flat_split)
    stale = fresh()
    stale.train_range(material, cfg, 0, 1)
    stale.set_params(flat_split)
    stale.train_range(material, cfg, split, total)
    lost = np.linalg.norm(params(stale) - pa)
    print("resumed", resumed / moved, "noise", noise / moved, "other moments", lost / moved)
    assert lost > 10 * bar, (lost, bar)
    # a checkpoint of another model, or with a damaged header, is refused
    other = nt.Model(nt.configs.model_desc(list(s["mat"].formats), 64, 3, 4, 9, 2, nt.ACT_SELU))
    with pytest.raises(nt.NTBCError):
        other.checkpoint_load(ck)
    bad = ck.clone()
    bad[0] = 0
    with pytest.raises(nt.NTBCError):
        b.checkpoint_load(bad)
