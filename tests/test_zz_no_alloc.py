"""The allocation-free training-gradient entry point (ntbc_train_grads_noalloc).

It serves callers that may not allocate device memory, such as an engine's
texture-streaming thread bound to a pre-reserved VRAM budget, or a real-time
thread that cannot take cudaMalloc's device-wide synchronisation. Its scratch is
a fixed device array inside libntbc, shared by every call. These tests call it
through the C ABI and compare it with the allocating ntbc_train_grads on the
same inputs, twice in a row (the second call must not see the first call's
leftovers), within the gradient tolerance the other training tests use.
Kept in its own file, collected last."""
import numpy as np
import pytest
import torch

import descs
import synth
from oracle import bc as obc

nt = pytest.importorskip("paper_2407_09543_gb300")
pytestmark = pytest.mark.gpu
DEV = "cuda"
REL = 2e-3


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).ravel()).to(DEV)


def _case(seed=3):
    mat = synth.make_material("noalloc", 64, ["sine_rgb", "sine_r", "sine_r", "sine_rgb"], seed)
    desc, odesc = descs.case_descs(nt, mat.formats, 64, 3, 4, 16, 3, "selu")
    p0 = descs.init_params(odesc, seed)
    params = synth.random_params_like(p0, seed=seed + 1, grid_scale=0.5)
    refs = [obc.encode(f, t, 64, 64) for f, t in zip(mat.formats, mat.textures)]
    tex_d = [_dev(t) for t in mat.textures]
    ref_d = [_dev(r) for r in refs]
    material = nt.Material.make(64, 64, mat.formats, tex_d, ref_d)
    flat = _dev(nt.configs.flatten(desc, params))
    return desc, material, flat, (tex_d, ref_d)


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_noalloc_matches_allocating_path_twice():
    desc, material, flat, keep = _case()
    model = nt.Model(desc)
    model.set_params(flat)
    n = model.n_params
    rng = np.random.default_rng(0)
    for call, (nb, qat) in enumerate([(nt.NOALLOC_MAX_BLOCKS, 8), (37, 0)]):
        ids = _dev(rng.integers(0, 256, nb).astype(np.int32))
        g_ref = torch.empty(n, device=DEV)
        l_ref = torch.empty(6, device=DEV)
        model.train_grads(material, ids, g_ref, l_ref, qat_bits=qat)
        g = torch.full((n,), float("nan"), device=DEV)
        l = torch.full((6,), float("nan"), device=DEV)
        nt.ntbc_train_grads_noalloc(desc, flat, material, ids, g, l, qat_bits=qat)
        torch.cuda.synchronize()
        assert torch.isfinite(g).all() and torch.isfinite(l).all(), call
        np.testing.assert_allclose(l.cpu().numpy(), l_ref.cpu().numpy(), rtol=2e-4)
        lay = model.layout
        assert _rel(g[:lay.grid_floats], g_ref[:lay.grid_floats]) < REL, call
        assert _rel(g[lay.grid_floats:], g_ref[lay.grid_floats:]) < REL, call
    model.close()


def test_noalloc_rejects_batches_beyond_its_scratch():
    desc, material, flat, keep = _case()
    lay = nt.ntbc_model_layout(desc)
    ids = torch.zeros(nt.NOALLOC_MAX_BLOCKS + 1, dtype=torch.int32, device=DEV)
    g = torch.empty(lay.total, device=DEV)
    l = torch.empty(6, device=DEV)
    with pytest.raises(nt.NTBCError) as e:
        nt.ntbc_train_grads_noalloc(desc, flat, material, ids, g, l)
    assert e.value.status == 1 and "allocation-free limit" in str(e.value)
