"""The network as a torch.autograd.Function (forward and hand-written backward through
ntbc_vjp) against the FP64 oracle's vector-Jacobian product and against finite
differences of the GPU forward; the full 4096^2 / 12-level model checked on the blocks of a
64x64 texel crop."""
import numpy as np
import pytest
import torch

import descs
import synth
from oracle import ntbc as ont

nt = pytest.importorskip("paper_2407_09543_gb300")
pytestmark = pytest.mark.gpu
DEV = "cuda"


def rel_err(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def case(side=32, kinds=("sine_rgb", "sine_r", "sine_rgb"), levels=3, lo=4, hi=9, hidden=2, act="selu", seed=3):
    mat = synth.make_material("vjp", side, list(kinds), seed)
    desc, odesc = descs.case_descs(nt, mat.formats, side, levels, lo, hi, hidden, act)
    params = synth.random_params_like(descs.init_params(odesc, seed), seed=seed + 1)
    return desc, odesc, params


def run_function(desc, params, ids, g_e, g_c, qat):
    model = nt.Model(desc)
    p = torch.from_numpy(nt.configs.flatten(desc, params)).to(DEV).requires_grad_(True)
    idt = torch.from_numpy(np.asarray(ids, np.int32)).to(DEV)
    e, c = nt.NTBCFunction.apply(p, model, idt, qat)
    f = (e * torch.from_numpy(g_e).float().to(DEV)).sum() + (c * torch.from_numpy(g_c).float().to(DEV)).sum()
    f.backward()
    torch.cuda.synchronize()
    return e.detach().cpu().numpy(), c.detach().cpu().numpy(), p.grad.cpu().numpy(), model


def compare_grads(desc, gflat, want):
    gg = nt.configs.unflatten(desc, gflat)
    for key in ("color_grid", "endpoint_grid"):
        for a, b in zip(gg[key], want[key]):
            assert rel_err(a, b) < 2e-3, key
    for key in ("color_mlp", "endpoint_mlp"):
        for (aW, ab), (bW, bb) in zip(gg[key], want[key]):
            assert rel_err(aW, bW) < 2e-3, key
            assert rel_err(ab, bb) < 2e-3, key


@pytest.mark.parametrize("act,hidden,qat", [("selu", 2, 0), ("relu", 2, 0), ("selu", 3, 8), ("selu", 1, 4)])
def test_function_matches_oracle_vjp(act, hidden, qat):
    desc, odesc, params = case(act=act, hidden=hidden)
    rng = np.random.default_rng(0)
    ids = np.array([0, 5, 17, 33, 63, 40, 5, 22])
    g_e = rng.standard_normal((len(ids), odesc.out_endpoint))
    g_c = rng.standard_normal((len(ids), 16, odesc.out_color))
    e, c, g, _ = run_function(desc, params, ids, g_e, g_c, qat)
    er, cr, want = ont.outputs_vjp(odesc, params, ids, g_e, g_c, qat_bits=qat)
    np.testing.assert_allclose(e, er, rtol=2e-5, atol=1e-7)
    np.testing.assert_allclose(c, cr, rtol=2e-5, atol=1e-7)
    compare_grads(desc, g, want)


def test_backward_matches_finite_differences_of_the_gpu_forward():
    # central differences of f = <g_e, e_hat> + <g_c, c_hat> through the GPU forward (FP32,
    # deterministic, host sum in FP64) at the MLP weights and grid entries with the largest
    # gradients. h = 1e-3 keeps the FP32 noise below 1e-3 absolute; SELU's derivative jumps
    # at 0 (lambda vs lambda alpha), so a difference quotient that straddles a kink is off by
    # O(h): 0.8% at most on this case in FP64, hence the 2% bound.
    desc, odesc, params = case(hidden=3)
    rng = np.random.default_rng(1)
    ids = np.arange(0, 64, 3)
    g_e = rng.standard_normal((len(ids), odesc.out_endpoint))
    g_c = rng.standard_normal((len(ids), 16, odesc.out_color))
    _, _, g, model = run_function(desc, params, ids, g_e, g_c, 0)
    flat = nt.configs.flatten(desc, params).astype(np.float64)
    idt = torch.from_numpy(ids.astype(np.int32)).to(DEV)
    lay = model.layout

    def f(x):
        model.set_params(torch.from_numpy(x.astype(np.float32)).to(DEV))
        e = torch.empty(len(ids), lay.out_endpoint, device=DEV)
        c = torch.empty(len(ids), 16, lay.out_color, device=DEV)
        model.vjp(idt, 0, e_hat=e, c_hat=c)
        torch.cuda.synchronize()
        return float(np.sum(g_e * e.cpu().numpy().astype(np.float64)) + np.sum(g_c * c.cpu().numpy().astype(np.float64)))

    grid_n = lay.grid_floats
    mlp = np.arange(grid_n, flat.size)
    grid = np.arange(grid_n)
    picks = list(mlp[np.argsort(-np.abs(g[mlp]))[:8]]) + list(grid[np.argsort(-np.abs(g[grid]))[:4]])
    h = 1e-3
    for i in picks:
        d = np.zeros(flat.size)
        d[i] = h
        fd = (f(flat + d) - f(flat - d)) / (2 * h)
        assert abs(fd - g[i]) <= 2e-2 * abs(g[i]) + 1e-3, (i, fd, g[i])


def test_full_model_on_a_64x64_crop():
    # the 4096^2 material model (12 levels 16..2048, 10 endpoint levels, 3 x 64 SELU,
    # 2 BC1 + 2 BC4, 8-bit QAT) at the 16 x 16 blocks covering texels [1024, 1088)^2
    w = nt.configs.WORKLOADS["mat4k"]
    formats = [1, 1, 4, 4]
    desc, odesc = descs.case_descs(nt, formats, 4096, w.levels, w.min_res, w.max_res, 3, "selu")
    params = synth.random_params_like(descs.init_params(odesc, 9), seed=10)
    bx, by = np.meshgrid(np.arange(256, 272), np.arange(256, 272))
    ids = (by * 1024 + bx).ravel()
    rng = np.random.default_rng(2)
    g_e = rng.standard_normal((len(ids), odesc.out_endpoint))
    g_c = rng.standard_normal((len(ids), 16, odesc.out_color))
    e, c, g, _ = run_function(desc, params, ids, g_e, g_c, 8)
    er, cr, want = ont.outputs_vjp(odesc, params, ids, g_e, g_c, qat_bits=8)
    np.testing.assert_allclose(e, er, rtol=2e-5, atol=1e-7)
    np.testing.assert_allclose(c, cr, rtol=2e-5, atol=1e-7)
    compare_grads(desc, g, want)
