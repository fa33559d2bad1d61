"""Batched load-time inference: materials of uneven size and texture mix, each with its
own model, in one persistent launch (replayed from a CUDA graph); every material's blocks
must equal those of its own single-material launch (same kernels, same arithmetic)."""
import numpy as np
import pytest
import torch

import descs
import synth

nt = pytest.importorskip("paper_2407_09543_gb300")
pytestmark = pytest.mark.gpu
DEV = "cuda"

SPECS = [(64, [1, 4]), (132, [4, 1, 1]), (256, [1, 1, 4, 4, 4]), (96, [4, 4])]


def _models(prec):
    models, outs, dlist = [], [], []
    for i, (side, formats) in enumerate(SPECS):
        desc, odesc = descs.case_descs(nt, formats, side, 4, 8, max(side // 2, 16), 3, "selu")
        p0 = descs.init_params(odesc, i)
        params = synth.random_params_like(p0, seed=10 + i)
        m = nt.Model(desc)
        m.set_params(torch.from_numpy(nt.configs.flatten(desc, params)).to(DEV))
        m.export(grid_bits=8, weight_prec=prec)
        nb = (side // 4) ** 2
        models.append(m)
        outs.append([torch.full((nb * 8,), 0xAB, dtype=torch.uint8, device=DEV) for _ in formats])
        dlist.append(desc)
    return models, outs, dlist


@pytest.mark.parametrize("prec", [1, 2])
def test_batch_equals_single_launches_and_replays(prec):
    models, outs, dlist = _models(prec)
    batch = nt.Batch(models, outs)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.infer()
    ms = batch.times_ms(stream)
    assert all(t > 0 for t in ms) and max(ms) < 1000.0
    first = [[o.clone() for o in mo] for mo in outs]
    for mo in outs:
        for o in mo:
            o.fill_(0xCD)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        batch.infer()
    g.replay()
    torch.cuda.synchronize()
    for m, mo, fo in zip(models, outs, first):
        single = [torch.empty_like(o) for o in mo]
        m.infer_to_bc(single)
        torch.cuda.synchronize()
        for a, b, c in zip(single, mo, fo):
            assert torch.equal(a, b) and torch.equal(a, c)
    batch.close()


def test_batch_rejects_fp32_models():
    models, outs, dlist = _models(1)
    models[1].export(grid_bits=8, weight_prec=nt.PREC_FP32)
    with pytest.raises(nt.NTBCError):
        nt.Batch(models, outs)
