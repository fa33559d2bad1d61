"""Inference precision sweep on trained 4096^2 weights: grids u8 / u4 (each trained with its
QAT width) x MLP weights FP32 (SIMT) / FP16 split / FP16 fast / FP8 E4M3, reporting for each
the error against the FP64 oracle with the same stored weights (kernel parity), against the
FP64 network on the FP32 master weights (what the storage precision gives up), the field
mismatch after quantisation and the decoded PSNR.

A GPU script beside the tests (it needs the oracle, which the benchmark does not run):
    python tests/precision_sweep.py [--train-steps 20000]
prints one JSON line.
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402

BATCH_TEXELS = bench.BATCH_TEXELS
build_workload = bench.build_workload


def run_sweep(args):
    """Inference precision sweep on trained 4k weights (one encode per grid width)."""
    import torch
    import paper_2407_09543_gb300 as nt
    from oracle import bc as obc, ntbc as ont
    dev = torch.device("cuda", 0)
    side = args.side
    nblk = (side // 4) ** 2
    mat, desc, p0, tex_d, refs = build_workload(nt, torch, side, seed=0, dev=dev)
    for t, fmt in enumerate(mat.formats):
        nt.bc_reference_encode(fmt, tex_d[t], side, side, refs[t], refine=bench.REF_REFINE)
    torch.cuda.synchronize()
    ref_psnr = bench.psnr_list(nt, torch, mat, refs, side)
    material = nt.Material.make(side, side, mat.formats, tex_d, refs)
    cres, eres = nt.configs.res_lists(desc)
    od = ont.ModelDesc(side, side, mat.formats, cres, eres, hidden_layers=desc.hidden_layers, activation="selu")
    ids = np.sort(np.random.default_rng(0).choice(nblk, 2000, replace=False))
    rows = []
    for bits in (8, 4):
        model = nt.Model(desc)
        model.set_params(torch.from_numpy(nt.configs.flatten(desc, p0)).to(dev))
        model.train(material, nt.TrainConfig.make(steps=args.train_steps, batch_texels=BATCH_TEXELS, qat_fraction=0.1,
                                                  grid_bits=bits, seed=0, precision=nt.TRAIN_BF16))
        flat = torch.empty(model.n_params, device=dev)
        model.get_params(flat)
        params = nt.configs.unflatten(desc, flat.cpu().numpy())
        codes, sc, zr = ont.export_grid(params["color_grid"] + params["endpoint_grid"], bits)
        deq = ont.dequantize_grid(codes, sc, zr)
        nc = desc.color_levels
        # the FP64 network on the FP32 master weights: what each stored precision gives up
        er32, cr32 = ont.forward_blocks(od, params, ids, color_grid=deq[:nc], endpoint_grid=deq[nc:])
        for name, prec in (("fp32", nt.PREC_FP32), ("fp16", nt.PREC_FP16), ("fp16_fast", nt.PREC_FP16_FAST),
                           ("fp8_e4m3", nt.PREC_FP8)):
            model.export(grid_bits=bits, weight_prec=prec)
            if prec == nt.PREC_FP8:
                pw = ont.fp8_params(params)[0]
            else:
                pw = dict(color_grid=params["color_grid"], endpoint_grid=params["endpoint_grid"])
                for k in ("color_mlp", "endpoint_mlp"):
                    pw[k] = [((W.astype(np.float16) if prec else W).astype(np.float64),
                              (b.astype(np.float16) if prec else b).astype(np.float64)) for W, b in params[k]]
            er, cr = ont.forward_blocks(od, pw, ids, color_grid=deq[:nc], endpoint_grid=deq[nc:])
            idt = torch.from_numpy(ids.astype(np.int32)).to(dev)
            lay = model.layout
            e = torch.empty(len(ids), lay.out_endpoint, device=dev)
            c = torch.empty(len(ids), 16, lay.out_color, device=dev)
            model.forward(idt, e, c)
            outs = [torch.empty(nblk * 8, dtype=torch.uint8, device=dev) for _ in mat.formats]
            model.infer_to_bc(outs)
            torch.cuda.synchronize()
            eg, cg = e.cpu().numpy(), c.cpu().numpy()
            rel = max(float(np.max(np.abs(eg - er) / np.abs(er))), float(np.max(np.abs(cg - cr) / np.abs(cr))))
            rel32 = max(float(np.max(np.abs(eg - er32) / np.abs(er32))), float(np.max(np.abs(cg - cr32) / np.abs(cr32))))
            ref_blocks = ont.infer_blocks(od, pw, block_ids=ids, color_grid=deq[:nc], endpoint_grid=deq[nc:])
            mism = fields = 0
            for t, fmt in enumerate(mat.formats):
                got = outs[t].cpu().numpy().reshape(-1, 8)[ids]
                unpack = obc.bc1_unpack if fmt == 1 else obc.bc4_unpack
                a0, a1, ac = unpack(got)
                b0, b1, bc_ = unpack(ref_blocks[t])
                mism += int((a0 != b0).sum() + (a1 != b1).sum() + (ac != bc_).sum())
                fields += len(ids) * 18
            rows.append({"grid_bits": bits, "mlp": name, "max_rel_err_vs_fp64": rel,
                         "max_rel_err_vs_fp64_fp32_weights": rel32,
                         "field_mismatch": mism / fields, "psnr_db": bench.psnr_list(nt, torch, mat, outs, side)})
        model.close()
    print(json.dumps({"mode": "sweep", "workload": f"mat4k {side}x{side}", "train_steps": args.train_steps,
                      "reference_bc_psnr_db": ref_psnr, "rows": rows}), flush=True)
    return 0


KIND_FORMAT = {"diffuse": 1, "normal": 1, "roughness": 4, "ao": 4}


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-steps", type=int, default=bench.FULL_MAIN_STEPS)
    ap.add_argument("--side", type=int, default=4096)
    sys.exit(run_sweep(ap.parse_args()))
