"""Batched load-time inference: materials of uneven size and texture mix, each with its
own model, decoded by one call (replayed from a CUDA graph), in both batch modes: chained
single-material launches (programmatic dependent launch) and one persistent work-queue launch.
Every material's blocks are checked against the FP64 oracle on the same stored model (u8 QAT
grids, FP16 weights: at most 0.1 % of fields differ with split activations) and must equal
those of its own single-material launch (same arithmetic). The work queue gives up with
NTBC_ETIMEOUT when its ticket counter is corrupted (host-side fault injection), and the next
launch works; overlapping outputs and unknown modes are refused on the host."""
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
    torch.cuda.synchronize()            # the exports ran on the current stream
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


MODES = [nt.BATCH_CHAINED, nt.BATCH_QUEUE]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("prec", [1, 2])
def test_batch_equals_single_launches_and_replays(prec, mode):
    models, outs, dlist = _models(prec)
    batch = nt.Batch(models, outs, mode=mode)
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
    batch = nt.Batch(models, outs, mode=nt.BATCH_QUEUE)
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


@pytest.mark.parametrize("mode", MODES)
def test_batch_rejects_fp32_models_overlapping_outputs_and_unknown_modes(mode):
    models, outs, dlist = _models(1)
    models[1].export(grid_bits=8, weight_prec=nt.PREC_FP32)
    with pytest.raises(nt.NTBCError):
        nt.Batch(models, outs, mode=mode)
    models, outs, dlist = _models(1)
    shifted = [list(o) for o in outs]
    shifted[3][1] = outs[0][0][8:]              # overlaps material 0's first texture
    with pytest.raises(nt.NTBCError) as e:
        nt.Batch(models, shifted, mode=mode)
    assert e.value.status == 1 and "overlap" in str(e.value)
    with pytest.raises(nt.NTBCError) as e:
        nt.Batch(models, outs, mode=7)
    assert e.value.status == 1


def test_chained_batch_mixes_precisions():
    """Chained launches run each material's own kernel: split FP16, pure FP16 and FP8
    arithmetic in one batch, each equal to its single-material launch."""
    models, outs, dlist = _models(1)
    models[1].export(grid_bits=8, weight_prec=nt.PREC_FP16_FAST)
    models[2].export(grid_bits=8, weight_prec=nt.PREC_FP8_MMA)
    torch.cuda.synchronize()
    with pytest.raises(nt.NTBCError):
        nt.Batch(models, outs, mode=nt.BATCH_QUEUE)
    batch = nt.Batch(models, outs)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.infer()
    assert all(t > 0 for t in batch.times_ms(stream))
    for m, mo in zip(models, outs):
        single = [torch.empty_like(o) for o in mo]
        m.infer_to_bc(single)
        torch.cuda.synchronize()
        for a, b in zip(single, mo):
            assert torch.equal(a, b)
    batch.close()


def test_batches_and_single_launches_with_different_shared_memory_coexist():
    """Two five-texture materials (64-block work units, the same kernel instance) whose weight
    images differ in size (12 vs 4 grid levels): a single launch of the smaller one between two
    launches of the larger one's batch must not shrink the shared-memory allowance the batch
    was created with."""
    made = []
    for i, levels in enumerate((12, 4)):
        formats = [1, 1, 4, 4, 4]
        desc, odesc = descs.case_descs(nt, formats, 256, levels, 8, 128, 3, "selu")
        params = descs.as_float32(synth.random_params_like(descs.init_params(odesc, 20 + i), seed=30 + i))
        m = nt.Model(desc)
        m.set_params(torch.from_numpy(nt.configs.flatten(desc, params)).to(DEV))
        m.export(grid_bits=8, weight_prec=nt.PREC_FP16)
        made.append((m, [torch.empty((256 // 4) ** 2 * 8, dtype=torch.uint8, device=DEV) for _ in formats]))
    (big, big_out), (small, small_out) = made
    batch = nt.Batch([big], [big_out], mode=nt.BATCH_QUEUE)
    batch.infer()
    torch.cuda.synchronize()
    first = [o.clone() for o in big_out]
    small.infer_to_bc(small_out)
    other = nt.Batch([small], [small_out], mode=nt.BATCH_QUEUE)
    other.infer()
    torch.cuda.synchronize()
    for o in big_out:
        o.fill_(0)
    batch.infer()
    torch.cuda.synchronize()
    for a, b in zip(first, big_out):
        assert torch.equal(a, b)
    single = [torch.empty_like(o) for o in big_out]
    big.infer_to_bc(single)
    torch.cuda.synchronize()
    for a, b in zip(single, big_out):
        assert torch.equal(a, b)
    batch.close()
    other.close()
    for m, _ in made:
        m.close()
