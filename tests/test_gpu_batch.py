"""Batched load-time inference: materials of uneven size and texture mix, each with its
own model, in one persistent launch (replayed from a CUDA graph). Every material's blocks are
checked against the FP64 oracle on the same stored model (u8 QAT grids, FP16 weights: at most
0.1 % of fields differ with split activations) and must equal those of its own single-material
launch (same kernels, same arithmetic). The launch's work queue gives up with NTBC_ETIMEOUT
when its ticket counter is corrupted (host-side fault injection), and the next launch works."""
import os

import numpy as np
import pytest
import torch

import descs
import synth
from oracle import bc as obc, ntbc as ont

nt = pytest.importorskip("paper_2407_09543_gb300")
pytestmark = pytest.mark.gpu
DEV = "cuda"

SPECS = [(64, [1, 4]), (132, [4, 1, 1]), (256, [1, 1, 4, 4, 4]), (96, [4, 4])]


def _models(prec):
    models, outs, dlist = [], [], []
    for i, (side, formats) in enumerate(SPECS):
        desc, odesc = descs.case_descs(nt, formats, side, 4, 8, max(side // 2, 16), 3, "selu")
        p0 = descs.init_params(odesc, i)
        params = descs.as_float32(synth.random_params_like(p0, seed=10 + i))
        m = nt.Model(desc)
        m.set_params(torch.from_numpy(nt.configs.flatten(desc, params)).to(DEV))
        m.export(grid_bits=8, weight_prec=prec)
        nb = (side // 4) ** 2
        models.append(m)
        outs.append([torch.full((nb * 8,), 0xAB, dtype=torch.uint8, device=DEV) for _ in formats])
        dlist.append((desc, odesc, params))
    return models, outs, dlist


def _oracle_blocks(odesc, params):
    """The oracle's inference to blocks on the stored model: its own u8 export of the grids,
    MLP weights rounded to FP16."""
    codes, sc, zr = ont.export_grid(params["color_grid"] + params["endpoint_grid"], 8)
    deq = ont.dequantize_grid(codes, sc, zr)
    nc = len(odesc.color_res)
    p16 = dict(params)
    for k in ("color_mlp", "endpoint_mlp"):
        p16[k] = [(W.astype(np.float16).astype(np.float64), b.astype(np.float16).astype(np.float64))
                  for W, b in params[k]]
    return ont.infer_blocks(odesc, p16, color_grid=deq[:nc], endpoint_grid=deq[nc:])


def _field_mismatch(formats, got, ref):
    mism = total = 0
    for fmt, g, r in zip(formats, got, ref):
        unpack = obc.bc1_unpack if fmt == 1 else obc.bc4_unpack
        a, b = unpack(g), unpack(r)
        mism += sum(int((x != y).sum()) for x, y in zip(a, b))
        total += 18 * len(g)
    return mism, total


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
    for m, mo, fo, (side, formats), (desc, odesc, params) in zip(models, outs, first, SPECS, dlist):
        single = [torch.empty_like(o) for o in mo]
        m.infer_to_bc(single)
        torch.cuda.synchronize()
        for a, b, c in zip(single, mo, fo):
            assert torch.equal(a, b) and torch.equal(a, c)
        got = [o.cpu().numpy().reshape(-1, 8) for o in mo]
        mism, total = _field_mismatch(formats, got, _oracle_blocks(odesc, params))
        assert mism <= (0.001 if prec == 1 else 0.005) * total, (side, mism, total)
    batch.close()


def test_batch_work_queue_timeout_and_recovery():
    models, outs, dlist = _models(1)
    batch = nt.Batch(models, outs)
    stream = torch.cuda.Stream()
    os.environ["NTBC_FAULT"] = "ticket"
    try:
        with torch.cuda.stream(stream):
            batch.infer()
        with pytest.raises(nt.NTBCError) as e:
            batch.times_ms(stream)
        assert e.value.status == 4 and "gave up" in str(e.value)
    finally:
        del os.environ["NTBC_FAULT"]
    # the context stays usable and the next launch delivers every material
    for mo in outs:
        for o in mo:
            o.fill_(0xCD)
    with torch.cuda.stream(stream):
        batch.infer()
    ms = batch.times_ms(stream)
    assert all(t > 0 for t in ms)
    for m, mo in zip(models, outs):
        single = [torch.empty_like(o) for o in mo]
        m.infer_to_bc(single)
        torch.cuda.synchronize()
        for a, b in zip(single, mo):
            assert torch.equal(a, b)
    batch.close()


def test_batch_rejects_fp32_models():
    models, outs, dlist = _models(1)
    models[1].export(grid_bits=8, weight_prec=nt.PREC_FP32)
    with pytest.raises(nt.NTBCError):
        nt.Batch(models, outs)
