"""Benchmark: NTBC inference (Mblocks/s) and 4k-material encode time on one GB300 per rank.

Workload (default): the 4096^2 material with diffuse + normal (BC1) and roughness + AO
(BC4) textures and crack overlay, 12 grid levels 16..2048, 8-bit QAT grids,
3 x 64 SELU MLPs, FP16 inference weights. Synthetic, seeded (no dataset exists here).

One timed step = one NTBC inference pass over the whole material (all 4 textures,
1,048,576 block positions, 4,194,304 texture blocks) through the C ABI, inputs
resident in HBM; the L2 is flushed (256 MiB write) between timed iterations, each
iteration bracketed by its own CUDA events on the launching stream.
Also reported: the roofline of the inference kernel against the exp2 rate measured in the
same run; the encode (training) time per step and the full-schedule encode seconds (BF16
tensor-core training; the FP32-kernel encode beside it for decoded-PSNR parity); the same
metric end to end with host buffers (model blob H2D, blocks D2H) and its parts; the plain
FP32 PyTorch path on the same GPU; the 16-material batched launch; the FP64 oracle over the
whole material on all host cores (cpu_baseline) with the accuracy bars checked on the GPU's
blocks against it; and a quality / storage study (Fig. average: mean decoded PSNR and SSIM as
ratios of the reference BC's against stored bytes, aggressive and conservative packaging,
8-bit and 4-bit QAT grids). The reference BC targets are the range-fit encoder with two
least-squares endpoint refits.

--impl reference times the FP64 oracle alone on all host cores (the paper has no code, so its
reference arm is the oracle): runs of block rows of the same workload, no product code.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

FULL_MAIN_STEPS = 20000
FULL_QAT_STEPS = 2000
BATCH_TEXELS = 1 << 18
FORMATS = [1, 1, 4, 4]
# the reference BC targets: range fit + two least-squares endpoint refits (the paper's
# reference encoder runs two refinement steps, Sec. 4.1)
REF_REFINE = 2
# end-to-end leg: blocks delivered to pinned host memory in this many ranges, each range's
# copy overlapping the inference of the next
E2E_CHUNKS = 4
KIND_FORMAT = {"diffuse": 1, "normal": 1, "roughness": 4, "ao": 4}
METRIC = "NTBC infer Mblocks/s (4k material, 4 textures) + 4k-material encode s, vs plain FP32 GPU, at decoded-PSNR parity"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--train-steps", type=int, default=FULL_MAIN_STEPS,
                    help="main-phase encode steps actually run (the QAT phase adds 10 %%)")
    ap.add_argument("--side", type=int, default=4096)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp32-train", action="store_true", help="skip the FP32-kernel encode (PSNR comparison)")
    ap.add_argument("--no-conservative", action="store_true", help="skip the conservative-packaging encode and decode")
    ap.add_argument("--no-study", action="store_true",
                    help="skip the quality / storage study (4-bit-grid encodes of both packagings)")
    ap.add_argument("--prec", type=int, default=1, help="1: FP16 weights, split FP16 activations; 2: pure FP16; 3: FP8 E4M3 weights, split activations; 4: FP8 arithmetic (E4M3 activations, kind::f8f6f4)")
    ap.add_argument("--batch", action="store_true",
                    help="batched load-time inference: 16 uneven materials in one persistent launch (CUDA graph)")
    ap.add_argument("--quick", action="store_true",
                    help="inference only on random-init weights (no material, training, plain path or oracle)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_material_seed(rank):
    """Each rank encodes and decodes its own material (weak scaling, no data exchange)."""
    return int(rank)


def max_over_ranks(value, world, device=None):
    """Time of the slowest rank (the whole job ends when it ends)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, ms):
    """Units processed by all ranks per second, in millions."""
    return world * units_per_rank / (ms * 1e-3) / 1e6


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.out = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def wait_first_sample(self, timeout_s=5.0):
        """Block until nvidia-smi has written its first sample (it takes a moment to start)."""
        t0 = time.perf_counter()
        while self.proc is not None and time.perf_counter() - t0 < timeout_s:
            if os.path.getsize(self.path) > 0:
                return
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            if self.out is not None:
                self.out.close()
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, val in zip(names, r[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ----------------------------------------------------------------------------
# workload setup
# ----------------------------------------------------------------------------

def build_workload(nt, torch, side, seed, dev):
    mat = synth.material_4k(seed=seed, side=side)
    w = nt.configs.WORKLOADS["mat4k"]
    desc = nt.configs.desc_for(w, mat.formats, side=side)
    cres, eres = nt.configs.res_lists(desc)
    p0 = synth.init_params(cres, eres, 2, nt.configs.mlp_dims(desc, "color"), nt.configs.mlp_dims(desc, "endpoint"), seed)
    tex_d = [torch.from_numpy(t.ravel()).to(dev) for t in mat.textures]
    nblk = (side // 4) ** 2
    refs = [torch.empty(nblk * 8, dtype=torch.uint8, device=dev) for _ in mat.formats]
    return mat, desc, p0, tex_d, refs


def time_events(torch, fn, iters, flush=None, stream=None):
    """Per-iteration CUDA-event timing on the launching stream; optional L2 flush between."""
    times = []
    for _ in range(iters):
        if flush is not None:
            flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    return times


def ssim_gpu(torch, a, b):
    """Mean SSIM (Wang et al. 2004; Sec. 4.1 reports it beside PSNR) of two H x W x C uint8
    images on the GPU: 11 x 11 Gaussian window (sigma 1.5), C1 = 0.01^2, C2 = 0.03^2 on values
    in [0, 1], valid region only, averaged over the channels."""
    g = torch.exp(-((torch.arange(11, device=a.device, dtype=torch.float64) - 5.0) ** 2) / (2 * 1.5 ** 2))
    g = g / g.sum()
    taps = [float(w) for w in g.cpu()]

    def blur(t, dim):                # one 11-tap pass along `dim`, valid region (FP64 adds)
        n = t.shape[dim] - 10
        acc = t.narrow(dim, 0, n) * taps[0]
        for k in range(1, 11):
            acc = acc + t.narrow(dim, k, n) * taps[k]
        return acc

    def win(t):                      # the separable 11 x 11 Gaussian window
        return blur(blur(t, 3), 2)

    x = a.double().permute(2, 0, 1)[:, None] / 255.0
    y = b.double().permute(2, 0, 1)[:, None] / 255.0
    mx, my = win(x), win(y)
    sxx = win(x * x) - mx * mx
    syy = win(y * y) - my * my
    sxy = win(x * y) - mx * my
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    m = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
    return float(m.mean(dim=(1, 2, 3)).mean())


def ssim_list(nt, torch, mat, blocks, side):
    """Decoded SSIM per texture (GPU decoder, GPU SSIM)."""
    out = []
    dev = torch.device("cuda", torch.cuda.current_device())
    for t, fmt in enumerate(mat.formats):
        src = torch.from_numpy(np.ascontiguousarray(mat.textures[t]).ravel()).to(dev)
        dec = torch.empty_like(src)
        nt.bc_decode(fmt, torch.as_tensor(blocks[t]).reshape(-1).to(dev), side, side, dec)
        shape = (side, side, 3 if fmt == 1 else 1)
        out.append(round(ssim_gpu(torch, dec.reshape(shape), src.reshape(shape)), 4))
    return out


def psnr_list(nt, torch, mat, blocks, side):
    """Decoded PSNR per texture (Sec. 4.1: 10 log10(1 / MSE) over all channels in [0, 1]):
    the blocks decoded by the library's GPU decoder, compared with the source texels."""
    out = []
    dev = torch.device("cuda", torch.cuda.current_device())
    for t, fmt in enumerate(mat.formats):
        src = torch.from_numpy(np.ascontiguousarray(mat.textures[t]).ravel()).to(dev)
        dec = torch.empty_like(src)
        b = torch.as_tensor(blocks[t]).reshape(-1).to(dev)          # host results are copied over first
        nt.bc_decode(fmt, b, side, side, dec)
        mse = float(((dec.double() - src.double()) / 255.0).pow(2).mean())
        out.append(round(float("inf") if mse == 0 else 10.0 * float(np.log10(1.0 / mse)), 3))
    return out


# ----------------------------------------------------------------------------
# the CPU oracle across the host cores (cpu_baseline, full-material parity, reference arm)
# ----------------------------------------------------------------------------

def workload_spec(side, seed=0, params_path=None, grid_bits=8):
    """What an oracle worker needs to rebuild the model on its own: the 4k workload's shape
    (Sec. 3.4 model configuration) and either a file of flat FP32 parameters or a seed."""
    return dict(formats=list(FORMATS), side=side, levels=12, lo=16, hi=2048, hidden=3, act="selu",
                grid_bits=grid_bits, params=params_path, seed=seed)


def oracle_desc_of(spec):
    from oracle import ntbc as ont
    cres = ont.level_resolutions(spec["levels"], spec["lo"], spec["hi"])
    eres = ont.endpoint_resolutions(cres, spec["side"] // 4)
    return ont.ModelDesc(spec["side"], spec["side"], spec["formats"], cres, eres, hidden_layers=spec["hidden"],
                         activation=spec["act"])


def oracle_random_params(od, seed):
    """The seeded random-init weights (Sec. 3.4 initialisation, then spread over (0, 1) outputs)."""
    p0 = synth.init_params(od.color_res, od.endpoint_res, od.features, od.mlp_dims("color"),
                           od.mlp_dims("endpoint"), seed)
    return synth.random_params_like(p0, seed=seed + 1)


_ORACLE = {}


def _oracle_init(spec, compare=None):
    """Worker set-up: the exported model as the oracle computes it (its own QAT export of the
    grids, MLP weights rounded to FP16), and for the comparison pass memory maps of the source
    textures and of both block sets."""
    from oracle import ntbc as ont
    od = oracle_desc_of(spec)
    if spec["params"]:
        p = ont.params_from_flat(od, np.load(spec["params"], mmap_mode="r"))
    else:
        p = oracle_random_params(od, spec["seed"])
    nc = len(od.color_res)
    codes, sc, zr = ont.export_grid(p["color_grid"] + p["endpoint_grid"], spec["grid_bits"])
    deq = ont.dequantize_grid(codes, sc, zr)
    p16 = dict(color_grid=[], endpoint_grid=[])
    for k in ("color_mlp", "endpoint_mlp"):
        p16[k] = [(W.astype(np.float16).astype(np.float64), b.astype(np.float16).astype(np.float64)) for W, b in p[k]]
    _ORACLE.update(od=od, p16=p16, cgrid=deq[:nc], egrid=deq[nc:])
    if compare:
        _ORACLE["cmp"] = {k: [np.load(p, mmap_mode="r") for p in v] if isinstance(v, list) else np.load(v, mmap_mode="r")
                          for k, v in compare.items()}


def _oracle_blocks(rng):
    """NTBC inference to blocks (Sec. 3.2) of block ids [start, stop): [textures, n, 8] uint8."""
    from oracle import ntbc as ont
    start, stop = rng
    o = _ORACLE
    blocks = ont.infer_blocks(o["od"], o["p16"], block_ids=np.arange(start, stop), color_grid=o["cgrid"],
                              endpoint_grid=o["egrid"])
    return start, np.stack(blocks)


def _oracle_compare(rng):
    """Per texture, over whole block rows [start, stop): squared error of the decoded oracle and
    GPU blocks against the source (in [0, 1] units), and mismatched endpoint / index fields."""
    from oracle import bc as obc
    start, stop = rng
    od, c = _ORACLE["od"], _ORACLE["cmp"]
    bw = od.blocks_x
    y0, y1 = 4 * (start // bw), 4 * (stop // bw)
    out = []
    for t, fmt in enumerate(od.formats):
        ours = np.asarray(c["gpu"][t, start:stop])
        ref = np.asarray(c["oracle"][t, start:stop])
        src = np.asarray(c["tex"][t][y0:y1], np.float64) / 255.0
        unpack = obc.bc1_unpack if fmt == 1 else obc.bc4_unpack
        fo, fr = unpack(ours), unpack(ref)
        ep = int((fo[0] != fr[0]).sum() + (fo[1] != fr[1]).sum())
        ix = int((fo[2] != fr[2]).sum())
        sse = []
        for b in (ours, ref):
            d = obc.decode(fmt, b, od.width, y1 - y0).astype(np.float64) / 255.0
            sse.append(float(((d - src.reshape(d.shape)) ** 2).sum()))
        out.append((sse[0], sse[1], ep, ix))
    return start, out


class OraclePool:
    """The FP64 oracle in one spawned process per host core (spawn: safe after CUDA is up;
    single-threaded BLAS in every worker so the processes do not oversubscribe the cores)."""

    def __init__(self, spec, compare=None, cores=None):
        import multiprocessing as mp
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        self.cores = cores or len(os.sched_getaffinity(0))
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_init, initargs=(spec, compare))
        self.od = oracle_desc_of(spec)
        # every worker finished its set-up before anything is timed
        self.pool.map(_oracle_blocks, [(0, 1)] * self.cores, chunksize=1)

    def ranges(self, start_row, rows, rows_per_task=1):
        bw = self.od.blocks_x
        return [(r * bw, min(start_row + rows, r + rows_per_task) * bw)
                for r in range(start_row, start_row + rows, rows_per_task)]

    def blocks(self, start_row=0, rows=None):
        """Oracle blocks of block rows [start_row, start_row + rows): ([T, n, 8], wall seconds)."""
        rows = self.od.blocks_y - start_row if rows is None else rows
        rngs = self.ranges(start_row, rows)
        out = np.empty((len(self.od.formats), rows * self.od.blocks_x, 8), np.uint8)
        base = start_row * self.od.blocks_x
        t0 = time.perf_counter()
        for s, b in self.pool.imap_unordered(_oracle_blocks, rngs):
            out[:, s - base:s - base + b.shape[1]] = b
        return out, time.perf_counter() - t0

    def compare(self):
        res = [r for _, r in sorted(self.pool.imap_unordered(_oracle_compare, self.ranges(0, self.od.blocks_y, 4)))]
        return [tuple(sum(r[t][k] for r in res) for k in range(4)) for t in range(len(self.od.formats))]

    def close(self):
        self.pool.close()
        self.pool.join()


def full_material_oracle(side, flat_params, gpu_blocks, textures):
    """The oracle over every block of the material with the GPU arm's exported model (u8 QAT
    grids, FP16 MLP weights): timed across the host cores (the CPU baseline), then checked
    against the GPU blocks on the accuracy bars: decoded PSNR within 0.05 dB of the FP64-oracle
    network per texture and at most 0.1 % of endpoint or index fields differing."""
    tmp = tempfile.mkdtemp(prefix="ntbc_oracle_")
    paths = {"params": os.path.join(tmp, "params.npy"), "gpu": os.path.join(tmp, "gpu.npy"),
             "oracle": os.path.join(tmp, "oracle.npy")}
    try:
        np.save(paths["params"], np.asarray(flat_params, np.float32))
        np.save(paths["gpu"], np.stack([np.asarray(b).reshape(-1, 8) for b in gpu_blocks]))
        tex_paths = []
        for t, tex in enumerate(textures):
            tex_paths.append(os.path.join(tmp, f"tex{t}.npy"))
            np.save(tex_paths[-1], np.ascontiguousarray(tex))
        spec = workload_spec(side, params_path=paths["params"])
        compare = {"gpu": paths["gpu"], "oracle": paths["oracle"], "tex": tex_paths}
        # the comparison reads the oracle's blocks from a file the first pass writes
        pool = OraclePool(spec)
        blocks, dt = pool.blocks()
        pool.close()
        np.save(paths["oracle"], blocks)
        pool = OraclePool(spec, compare=compare, cores=pool.cores)
        sums = pool.compare()
        pool.close()
    finally:
        for p in list(paths.values()) + [os.path.join(tmp, f) for f in os.listdir(tmp) if f.startswith("tex")]:
            if os.path.exists(p):
                os.unlink(p)
        os.rmdir(tmp)
    od = oracle_desc_of(spec)
    n = od.n_blocks
    psnr_g, psnr_o, diff = [], [], []
    ep_m = ix_m = ep_f = ix_f = 0
    for t, (sse_g, sse_o, ep, ix) in enumerate(sums):
        vals = side * side * od.channels[t]
        pg, po = (10.0 * np.log10(vals / s) if s > 0 else float("inf") for s in (sse_g, sse_o))
        psnr_g.append(round(float(pg), 4))
        psnr_o.append(round(float(po), 4))
        diff.append(round(float(pg - po), 4))
        ep_m, ix_m = ep_m + ep, ix_m + ix
        ep_f, ix_f = ep_f + 2 * n, ix_f + 16 * n
    rate = (ep_m + ix_m) / (ep_f + ix_f)
    parity = {"blocks": n, "textures": len(od.formats), "psnr_db_gpu": psnr_g, "psnr_db_oracle": psnr_o,
              "psnr_diff_db": diff, "endpoint_field_mismatch": ep_m, "index_field_mismatch": ix_m,
              "field_mismatch_rate": round(rate, 7),
              "bar": "|PSNR diff| <= 0.05 dB per texture and <= 0.1 % fields differ",
              "pass": bool(max(abs(d) for d in diff) <= 0.05 and rate <= 0.001)}
    cpu = {"value": round(n * len(od.formats) / dt / 1e6, 6), "unit": "Mblocks/s", "cores": pool.cores,
           "kind": "oracle",
           "sample": f"the whole {side}x{side} material ({n} block positions x {len(od.formats)} textures), "
                     f"FP64 numpy, {pool.cores} processes, {dt:.1f} s"}
    return parity, cpu


# ----------------------------------------------------------------------------
# reference arm: the CPU oracle
# ----------------------------------------------------------------------------

def workload_config(side, world):
    return {"workload": f"mat4k {side}x{side}, 4 textures (2 BC1 + 2 BC4), 12 levels 16..2048 u8 QAT, "
                        f"3x64 SELU, FP16 weights", "texture_blocks": (side // 4) ** 2 * len(FORMATS),
            "block_positions": (side // 4) ** 2, "l2": "flushed (256 MiB write) between timed iterations",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    """The oracle (FP64 numpy, no product code) on the host cores: every step decodes a run of
    block rows of the 4k material to BC blocks, sized from the warm-up rate so the whole run
    takes about two minutes (the whole material per step when the cores allow it)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    side = args.side
    pool = OraclePool(workload_spec(side, seed=0))
    od = pool.od
    rows_total = od.blocks_y
    rows = max(1, min(rows_total, 2 * pool.cores))
    rates = []
    for i in range(args.warmup):
        _, dt = pool.blocks((i * rows) % max(1, rows_total - rows + 1), rows)
        rates.append(rows / dt)
    per_step_s = 120.0 / max(1, args.steps)
    rows = int(max(1, min(rows_total, (np.median(rates) if rates else rows) * per_step_s)))
    times = []
    for i in range(args.steps):
        start = (i * rows) % max(1, rows_total - rows + 1)
        _, dt = pool.blocks(start, rows)
        times.append(dt)
    pool.close()
    ms = 1e3 * float(np.mean(times))
    tex_blocks = rows * od.blocks_x * len(FORMATS)
    value = tex_blocks / (ms * 1e-3) / 1e6
    sample = (f"{rows} of {rows_total} block rows per step ({rows * od.blocks_x} block positions x {len(FORMATS)} "
              f"textures), FP64 numpy, {pool.cores} processes")
    line = {
        "metric": METRIC, "value": round(value, 6), "unit": "Mblocks/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": workload_config(side, world),
        "weights": "seeded random-init (the timed work does not depend on the weight values)",
        "cpu_baseline": {"value": round(value, 6), "unit": "Mblocks/s", "cores": pool.cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 6), "unit": "Mblocks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# exp2 results per clock per SM: measured on GB300 by ntbc_ex2_rate_probe (31.9 at 2.07 GHz);
# used only when no live measurement is given
MUFU_PER_SM_PER_CLK = 32
SM_COUNT = 152
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one inference pass of the split
# FP16 kernel on the 4096^2 four-texture material (its full-rounds launch and its split tail
# launch, summed), from one ncu capture of the current kernels; None for any other workload or
# precision
INFER_TC_DRAM_BYTES_MAT4K = 16_368_896 + 6_144 + 794_368     # full rounds (read + write), tail (read)
SM_MAX_GHZ = 2.07


def measured_peaks():
    """The measured HBM copy and bf16 GEMM peaks of these GPUs (MEASURED_PEAKS.json), else fallback figures."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if not os.path.exists(path):
        return {"bf16_tflops": 1900.0, "hbm_gbs": 6800.0}
    with open(path) as f:
        return json.load(f)


def encode_roofline(nt, desc, ms_step):
    """Bounds of one encode step at BATCH_TEXELS: tensor time of the forward + backward MLP
    FLOPs (3x the forward, BF16 dense peak) and HBM time of the dense Adam pass (read p, g,
    m, v; write p, m, v) and one read of both FP32 grids. The gradients need no dense clear:
    the step's Adam zeroes the entries it read, a few million of them."""
    lay = nt.ntbc_model_layout(desc)
    hl = desc.hidden_layers
    mac_c = lay.in_color * 64 + (hl - 1) * 64 * 64 + 64 * lay.out_color
    mac_e = lay.in_endpoint * 64 + (hl - 1) * 64 * 64 + 64 * lay.out_endpoint
    flops = 3 * 2.0 * (BATCH_TEXELS * mac_c + BATCH_TEXELS // 16 * mac_e)
    bytes_ = lay.total * 4.0 * (7 + 1)
    peaks = measured_peaks()
    t_tc = flops / (peaks["bf16_tflops"] * 1e12) * 1e3
    t_hbm = bytes_ / (peaks["hbm_gbs"] * 1e9) * 1e3
    return {"flop_per_step": flops, "hbm_bytes_per_step": bytes_, "t_tensor_ms": round(t_tc, 4),
            "t_hbm_ms": round(t_hbm, 4), "bound": "hbm" if t_hbm > t_tc else "tensor",
            "frac_of_measured": round(max(t_tc, t_hbm) / ms_step, 4)}


def inference_roofline(nt, desc, ms, traffic=None, mufu_peak=None):
    """Governing roofline of one inference pass: max of tensor (FP16 dense), MUFU (one exp2 per
    SELU unit and per sigmoid output) and HBM (grid codes read once + blocks written) times.
    mufu_peak: exp2 per second measured on the device (ntbc_ex2_rate_probe), else the per-SM
    rate measured on GB300 at the maximum SM clock."""
    lay = nt.ntbc_model_layout(desc)
    n_pos = (desc.width // 4) * (desc.height // 4)
    hl = desc.hidden_layers
    mac_c = lay.in_color * 64 + (hl - 1) * 64 * 64 + 64 * lay.out_color
    mac_e = lay.in_endpoint * 64 + (hl - 1) * 64 * 64 + 64 * lay.out_endpoint
    flops = 2.0 * (16 * mac_c + mac_e) * n_pos
    exps = (16 * (hl * 64 + lay.out_color) + hl * 64 + lay.out_endpoint) * float(n_pos)
    bytes_ = lay.grid_floats * 1 + 8.0 * n_pos * desc.n_textures
    peaks = measured_peaks()
    measured = mufu_peak is not None
    if not measured:
        mufu_peak = SM_COUNT * MUFU_PER_SM_PER_CLK * SM_MAX_GHZ * 1e9
    t_tc = flops / (peaks["bf16_tflops"] * 1e12)
    t_xu = exps / mufu_peak
    t_hbm = bytes_ / (peaks["hbm_gbs"] * 1e9)
    sec = ms * 1e-3
    kind = ("MUFU exp2 measured live by ntbc_ex2_rate_probe" if measured else
            "MUFU exp2: 152 SM x 32/clk (measured per-SM rate) x 2.07 GHz")
    roofline = {"bound": "alu", "achieved": round(exps / sec / 1e12, 4), "peak": round(mufu_peak / 1e12, 4),
                "unit": "Texp/s", "frac": round(t_xu / sec, 4), "traffic": traffic,
                "kernel": "infer_tc_kernel<split FP16> (full rounds of 128-block units + a chained tail of 64-block units; per pass)",
                "peak_kind": kind + "; tensor / HBM terms against MEASURED_PEAKS (of measured)"}
    terms = {"t_tensor_ms": round(t_tc * 1e3, 4), "t_mufu_ms": round(t_xu * 1e3, 4), "t_hbm_ms": round(t_hbm * 1e3, 4),
             "tensor_frac_of_measured": round(t_tc / sec, 4), "hbm_frac_of_measured": round(t_hbm / sec, 4),
             "flop_per_pass": flops, "exp_per_pass": exps, "hbm_bytes_per_pass": bytes_}
    return roofline, terms


def batch_leg(nt, torch, dev, steps, warmup, prec, flush):
    """16 materials of uneven size (sides 512..4096, 2..5 textures), each with its own 12-level
    grid (16 .. side/2) and 3 x 64 SELU MLPs, random-init weights, decoded to BC blocks by one
    batch call replayed from a CUDA graph: chained single-material launches (programmatic
    dependent launch, largest material first); beside it the work-queue mode (one persistent
    launch) and the same materials as 16 plain back-to-back single-material launches."""
    spec = synth.material_batch_spec(seed=0, count=16)
    models, outs, blocks = [], [], 0
    for i, (side, kinds) in enumerate(spec):
        formats = [KIND_FORMAT[k] for k in kinds]
        desc = nt.configs.model_desc(formats, side, 12, 16, side // 2, 3, nt.ACT_SELU)
        cres, eres = nt.configs.res_lists(desc)
        p0 = synth.init_params(cres, eres, 2, nt.configs.mlp_dims(desc, "color"), nt.configs.mlp_dims(desc, "endpoint"), i)
        m = nt.Model(desc)
        m.set_params(torch.from_numpy(nt.configs.flatten(desc, synth.random_params_like(p0, seed=100 + i))).to(dev))
        m.export(grid_bits=8, weight_prec=prec)
        nb = (side // 4) ** 2
        blocks += nb * len(formats)
        models.append(m)
        outs.append([torch.empty(nb * 8, dtype=torch.uint8, device=dev) for _ in formats])
    stream = torch.cuda.Stream()

    def graphed(batch):
        with torch.cuda.stream(stream):
            batch.infer()
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            batch.infer()
        for _ in range(warmup):
            g.replay()
        torch.cuda.synchronize()
        return g

    batch = nt.Batch(models, outs)                              # chained launches
    queue = nt.Batch(models, outs, mode=nt.BATCH_QUEUE)         # one persistent work-queue launch
    g = graphed(batch)
    times = time_events(torch, g.replay, steps, flush=flush)
    per_mat = batch.times_ms(torch.cuda.current_stream())
    gq = graphed(queue)
    times_q = time_events(torch, gq.replay, steps, flush=flush)
    seq = time_events(torch, lambda: [m.infer_to_bc(o) for m, o in zip(models, outs)], max(3, steps // 2), flush=flush)
    ms = float(np.mean(times))
    out = {"materials": [{"side": side, "textures": len(kinds), "done_ms": round(t, 4)} for (side, kinds), t in
                         zip(spec, per_mat)],
           "texture_blocks": blocks, "mode": "chained (programmatic dependent launch)", "launches": len(models),
           "ms_per_batch": round(ms, 4),
           "value": round(blocks / (ms * 1e-3) / 1e6, 3), "unit": "Mblocks/s",
           "work_queue_single_launch_ms": round(float(np.mean(times_q)), 4),
           "sequential_single_launch_ms": round(float(np.mean(seq)), 4), "graph": True}
    batch.close()
    queue.close()
    for m in models:
        m.close()
    return out


def run_batch(args):
    import torch
    import paper_2407_09543_gb300 as nt
    dev = torch.device("cuda", 0)
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    out = batch_leg(nt, torch, dev, args.steps, args.warmup, args.prec, lambda: flush_buf.fill_(1))
    print(json.dumps(dict(bench="batch", gpu_launches=out["launches"], **out)), flush=True)
    return 0


def run_quick(args):
    """Inference-only timing on random-init 4k weights (for profiling captures)."""
    import torch
    import paper_2407_09543_gb300 as nt
    dev = torch.device("cuda", 0)
    side = args.side
    nblk = (side // 4) ** 2
    w = nt.configs.WORKLOADS["mat4k"]
    desc = nt.configs.desc_for(w, FORMATS, side=side)
    cres, eres = nt.configs.res_lists(desc)
    p0 = synth.init_params(cres, eres, 2, nt.configs.mlp_dims(desc, "color"), nt.configs.mlp_dims(desc, "endpoint"), 0)
    params = synth.random_params_like(p0, seed=1)
    model = nt.Model(desc)
    model.set_params(torch.from_numpy(nt.configs.flatten(desc, params)).to(dev))
    model.export(grid_bits=8, weight_prec=args.prec)
    outs = [torch.empty(nblk * 8, dtype=torch.uint8, device=dev) for _ in FORMATS]
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        model.infer_to_bc(outs)
    torch.cuda.synchronize()
    times = time_events(torch, lambda: model.infer_to_bc(outs), args.steps, flush=lambda: flush_buf.fill_(1))
    ms = float(np.mean(times))
    print(json.dumps({"mode": "quick", "prec": args.prec, "workload": f"mat4k {side}x{side} random-init", "ms_per_step": round(ms, 4),
                      "value": round(nblk * len(FORMATS) / (ms * 1e-3) / 1e6, 3), "unit": "Mblocks/s",
                      "times_ms": [round(t, 4) for t in times]}), flush=True)
    return 0


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.quick:
        return run_quick(args)
    if args.batch:
        return run_batch(args)
    import torch
    import paper_2407_09543_gb300 as nt
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    torch.backends.cuda.matmul.allow_tf32 = False
    stream = torch.cuda.current_stream()
    side = args.side
    nblk = (side // 4) ** 2
    tex_blocks = nblk * len(FORMATS)

    mat, desc, p0, tex_d, refs = build_workload(nt, torch, side, seed=rank_material_seed(rank), dev=dev)

    # ---- reference BC targets (timed separately); the unrefined range fit for comparison
    for t, fmt in enumerate(mat.formats):
        nt.bc_reference_encode(fmt, tex_d[t], side, side, refs[t])
    torch.cuda.synchronize()
    ref_psnr_unrefined = psnr_list(nt, torch, mat, refs, side)
    ref_ms = time_events(torch, lambda: [nt.bc_reference_encode(f, tex_d[t], side, side, refs[t], refine=REF_REFINE)
                                         for t, f in enumerate(mat.formats)], 3)
    ref_psnr = psnr_list(nt, torch, mat, refs, side)
    ref_ssim = ssim_list(nt, torch, mat, refs, side)

    # ---- encode (training) on the GPU: measured steps, full schedule extrapolated
    model = nt.Model(desc)
    flat0 = torch.from_numpy(nt.configs.flatten(desc, p0)).to(dev)
    model.set_params(flat0)
    model.export(grid_bits=8, weight_prec=nt.PREC_FP16)
    untrained = [torch.empty(nblk * 8, dtype=torch.uint8, device=dev) for _ in FORMATS]
    model.infer_to_bc(untrained)
    untrained_psnr = psnr_list(nt, torch, mat, untrained, side)
    material = nt.Material.make(side, side, mat.formats, tex_d, refs)
    main_steps = args.train_steps
    total_steps = main_steps + int(np.ceil(0.1 * main_steps))

    def encode(m, precision):
        cfg = nt.TrainConfig.make(steps=main_steps, batch_texels=BATCH_TEXELS, qat_fraction=0.1, grid_bits=8,
                                  seed=rank, precision=precision)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        losses = m.train(material, cfg)
        return time.perf_counter() - t0, losses

    # headline encode: the fused BF16 tensor-core training pass
    train_s, last_losses = encode(model, nt.TRAIN_BF16)
    ms_per_train_step = 1e3 * train_s / total_steps
    encode_full_s = ms_per_train_step * (FULL_MAIN_STEPS + FULL_QAT_STEPS) / 1e3
    model.export(grid_bits=8, weight_prec=nt.PREC_FP16)
    # the same encode with the FP32 layer-by-layer kernels (decoded-PSNR parity of the BF16 encode)
    fp32_encode = None
    if not args.no_fp32_train:
        m32 = nt.Model(desc)
        m32.set_params(flat0)
        t32, _ = encode(m32, nt.TRAIN_FP32)
        m32.export(grid_bits=8, weight_prec=nt.PREC_FP16)
        o32 = [torch.empty(nblk * 8, dtype=torch.uint8, device=dev) for _ in FORMATS]
        m32.infer_to_bc(o32)
        fp32_encode = {"measured_s": round(t32, 2), "ms_per_step": round(1e3 * t32 / total_steps, 3),
                       "psnr_db": psnr_list(nt, torch, mat, o32, side)}
        m32.close()
        del o32

    # ---- inference timing (device-resident inputs)
    outs = [torch.empty(nblk * 8, dtype=torch.uint8, device=dev) for _ in FORMATS]
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def flush():
        flush_buf.fill_(1)

    def infer():
        model.infer_to_bc(outs)

    clocks = ClockSampler(local)
    clocks.start()
    clocks.wait_first_sample()
    for _ in range(args.warmup):
        flush()
        infer()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    times = time_events(torch, infer, args.steps, flush=flush)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    ms = max_over_ranks(float(np.mean(times)), world, dev)
    launches_per_pass = model.infer_plan()[0]                  # the full rounds, and a split tail
    headline_blocks = [o.cpu().numpy() for o in outs]          # for the full-material oracle check
    ours_psnr = psnr_list(nt, torch, mat, outs, side)
    ours_ssim = ssim_list(nt, torch, mat, outs, side)
    value = job_throughput(tex_blocks, world, ms)

    # ---- end to end through the C ABI with host buffers: blob H2D, then the inference with the
    # blocks delivered to pinned host memory (ntbc_infer_to_host)
    blob = torch.empty(model.blob_size(), dtype=torch.uint8).pin_memory()
    model.save(blob)
    host_out = [torch.empty(nblk * 8, dtype=torch.uint8).pin_memory() for _ in FORMATS]
    e2e_model = nt.Model(desc)

    def e2e():
        e2e_model.load(blob)
        e2e_model.infer_to_host(host_out, chunks=E2E_CHUNKS)

    for _ in range(max(1, args.warmup)):
        e2e()
    torch.cuda.synchronize()
    e2e_times = time_events(torch, e2e, args.steps, flush=flush)
    e2e_ms = max_over_ranks(float(np.mean(e2e_times)), world, dev)
    e2e_value = job_throughput(tex_blocks, world, e2e_ms)
    # where the end-to-end time goes: the blob upload, the inference with the blocks delivered
    # to host memory (copies overlapping the compute), and the raw copy rates of the same bytes
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    up, rest = [], []
    for _ in range(max(3, args.steps // 4)):
        flush()
        ev[0].record(stream)
        e2e_model.load(blob)
        ev[1].record(stream)
        e2e_model.infer_to_host(host_out, chunks=E2E_CHUNKS)
        ev[2].record(stream)
        ev[2].synchronize()
        up.append(ev[0].elapsed_time(ev[1]))
        rest.append(ev[1].elapsed_time(ev[2]))
    blob_dev = torch.empty(blob.numel(), dtype=torch.uint8, device=dev)
    raw_h2d = time_events(torch, lambda: blob_dev.copy_(blob, non_blocking=True), 5, flush=flush)
    raw_d2h = time_events(torch, lambda: [h.copy_(o, non_blocking=True) for h, o in zip(host_out, outs)], 5,
                          flush=flush)
    d2h_bytes = nblk * 8 * len(FORMATS)
    e2e_parts = {"blob_upload_ms": round(float(np.median(up)), 4),
                 "infer_and_delivery_ms": round(float(np.median(rest)), 4),
                 "raw_h2d_gbs": round(blob.numel() / (float(np.median(raw_h2d)) * 1e-3) / 1e9, 1),
                 "raw_d2h_gbs": round(d2h_bytes / (float(np.median(raw_d2h)) * 1e-3) / 1e9, 1),
                 "e2e_ms_min_median_max": [round(float(np.min(e2e_times)), 4), round(float(np.median(e2e_times)), 4),
                                           round(float(np.max(e2e_times)), 4)],
                 "chunks": E2E_CHUNKS}
    del blob_dev
    e2e_psnr = psnr_list(nt, torch, mat, host_out, side)

    # ---- roofline of the inference kernel (algorithmic counts per block position)
    mufu_peak = nt.ntbc_ex2_rate_probe()
    roofline, terms = inference_roofline(
        nt, desc, ms, INFER_TC_DRAM_BYTES_MAT4K if side == 4096 and args.prec == 1 else None, mufu_peak=mufu_peak)
    encode_terms = encode_roofline(nt, desc, ms_per_train_step)

    # ---- the same inference in the other modes (pure FP16 activations; FP8 arithmetic with
    # E4M3 activations on kind::f8f6f4 MMAs; FP32 SIMT kernel)
    modes = {}
    for name, prec in (("fp16_fast", nt.PREC_FP16_FAST), ("fp8_e4m3_mma", nt.PREC_FP8_MMA), ("fp32_simt", nt.PREC_FP32)):
        model.export(grid_bits=8, weight_prec=prec)
        model.infer_to_bc(outs)
        torch.cuda.synchronize()
        t_m = float(np.mean(time_events(torch, infer, max(3, args.steps // 4), flush=flush)))
        modes[name] = {"ms": round(t_m, 4), "value": round(tex_blocks / (t_m * 1e-3) / 1e6, 3),
                       "psnr_db": psnr_list(nt, torch, mat, outs, side)}
    model.export(grid_bits=8, weight_prec=nt.PREC_FP16)
    # the roughness and AO textures written as one BC5 texture (16-byte blocks, interleaved)
    bc5 = torch.empty(nblk * 16, dtype=torch.uint8, device=dev)
    bc5_ptrs = [outs[0].data_ptr(), outs[1].data_ptr(), bc5.data_ptr(), bc5.data_ptr() + 8]
    model.infer_to_bc(bc5_ptrs, strides=[8, 8, 16, 16])
    torch.cuda.synchronize()
    t_b5 = float(np.mean(time_events(torch, lambda: model.infer_to_bc(bc5_ptrs, strides=[8, 8, 16, 16]),
                                     max(3, args.steps // 4), flush=flush)))
    modes["bc5_layout"] = {"ms": round(t_b5, 4), "value": round(tex_blocks / (t_b5 * 1e-3) / 1e6, 3),
                           "note": "roughness + AO as one BC5 texture (strided 16-byte blocks)"}
    del bc5

    # ---- batched load-time inference: 16 uneven materials in one launch (work queue, graph)
    batch16 = batch_leg(nt, torch, dev, max(5, args.steps // 2), 3, nt.PREC_FP16, flush)

    # ---- packagings (Sec. 4.1): aggressive = one model for all textures, conservative = one
    # model for the BC1 textures and one for the BC4 textures; each encoded with the BF16 pass
    # at the given QAT grid width and exported with grids of that width and FP16 weights
    wl = nt.configs.WORKLOADS["mat4k"]

    def encode_package(packaging, grid_bits):
        groups = nt.configs.packaging_groups(FORMATS, packaging)
        models, outs_g, enc_s, nbytes = [], [], 0.0, 0
        for gi, g in enumerate(groups):
            fm = [FORMATS[t] for t in g]
            d = nt.configs.desc_for(wl, fm, side=side)
            cres, eres = nt.configs.res_lists(d)
            seed = rank_material_seed(rank) + (0 if packaging == "aggressive" else 17 * (gi + 1))
            pc = synth.init_params(cres, eres, 2, nt.configs.mlp_dims(d, "color"), nt.configs.mlp_dims(d, "endpoint"),
                                   seed)
            mc = nt.Model(d)
            mc.set_params(torch.from_numpy(nt.configs.flatten(d, pc)).to(dev))
            mat_g = nt.Material.make(side, side, fm, [tex_d[t] for t in g], [refs[t] for t in g])
            cfg_g = nt.TrainConfig.make(steps=main_steps, batch_texels=BATCH_TEXELS, qat_fraction=0.1,
                                        grid_bits=grid_bits, seed=rank, precision=nt.TRAIN_BF16)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mc.train(mat_g, cfg_g)
            enc_s += time.perf_counter() - t0
            mc.export(grid_bits=grid_bits, weight_prec=nt.PREC_FP16)
            nbytes += mc.blob_size()
            models.append(mc)
            outs_g.append([torch.empty(nblk * 8, dtype=torch.uint8, device=dev) for _ in g])
        by_tex = [None] * len(FORMATS)
        for g, o in zip(groups, outs_g):
            for t, oo in zip(g, o):
                by_tex[t] = oo
        return groups, models, outs_g, by_tex, enc_s, nbytes

    def quality(by_tex):
        return psnr_list(nt, torch, mat, by_tex, side), ssim_list(nt, torch, mat, by_tex, side)

    packages = {"aggressive_u8": {"storage_bytes": int(model.blob_size()), "encode_s": round(train_s, 2),
                                  "psnr_db": ours_psnr, "ssim": ours_ssim}}
    conservative = None
    if not args.no_conservative:
        groups, c_models, c_outs, by_tex, c_train_s, c_bytes = encode_package("conservative", 8)
        c_batch = nt.Batch(c_models, c_outs)
        c_batch.infer()
        torch.cuda.synchronize()
        c_times = time_events(torch, c_batch.infer, max(3, args.steps // 2), flush=flush)
        c_ms = float(np.mean(c_times))
        c_psnr, c_ssim = quality(by_tex)
        conservative = {"models": len(groups), "textures_per_model": [len(g) for g in groups],
                        "encode_s_measured": round(c_train_s, 2), "infer_ms": round(c_ms, 4),
                        "infer_value": round(tex_blocks / (c_ms * 1e-3) / 1e6, 3), "unit": "Mblocks/s",
                        "psnr_db": c_psnr, "ssim": c_ssim,
                        "storage_bytes": int(c_bytes), "aggressive_storage_bytes": int(model.blob_size())}
        packages["conservative_u8"] = {"storage_bytes": int(c_bytes), "encode_s": round(c_train_s, 2),
                                       "psnr_db": c_psnr, "ssim": c_ssim}
        c_batch.close()
        for mc in c_models:
            mc.close()

    # ---- quality / storage study (Fig. average): each packaging's mean decoded PSNR and SSIM
    # as a ratio of the reference BC's, against its stored bytes; 8-bit and 4-bit QAT grids
    study = None
    if not args.no_study:
        for packaging in ("aggressive", "conservative"):
            if packaging == "conservative" and args.no_conservative:
                continue
            groups, ms_, outs_g, by_tex, enc_s, nbytes = encode_package(packaging, 4)
            for mm, o in zip(ms_, outs_g):
                mm.infer_to_bc(o)
            torch.cuda.synchronize()
            q_psnr, q_ssim = quality(by_tex)
            packages[packaging + "_u4"] = {"storage_bytes": int(nbytes), "encode_s": round(enc_s, 2),
                                           "psnr_db": q_psnr, "ssim": q_ssim}
            for mm in ms_:
                mm.close()
        ref_bytes = nblk * 8 * len(FORMATS)
        p_ref, s_ref = float(np.mean(ref_psnr)), float(np.mean(ref_ssim))
        study = {"reference_bc": {"storage_bytes": int(ref_bytes), "psnr_db_mean": round(p_ref, 3),
                                  "ssim_mean": round(s_ref, 4), "refine_steps": REF_REFINE}}
        for name, e in packages.items():
            study[name] = dict(e, storage_ratio=round(e["storage_bytes"] / ref_bytes, 4),
                               psnr_ratio=round(float(np.mean(e["psnr_db"])) / p_ref, 4),
                               ssim_ratio=round(float(np.mean(e["ssim"])) / s_ref, 4))

    # ---- plain FP32 PyTorch path on the same GPU and weights
    plain = None
    if not args.no_plain:
        from baseline import plain_fp32 as pf
        flat = torch.empty(model.n_params, device=dev)
        model.get_params(flat)
        params = nt.configs.unflatten(desc, flat.cpu().numpy())
        cres, eres = nt.configs.res_lists(desc)
        pm = pf.PlainModel(side, side, mat.formats, cres, eres, params, "selu", dev)
        qf = pf._qat_fn(8)
        with torch.no_grad():
            grids = ([qf(g) for g in pm.color_grid], [qf(g) for g in pm.endpoint_grid])
        for W, b in pm.color_mlp + pm.endpoint_mlp:
            with torch.no_grad():
                W.copy_(W.half().float())
                b.copy_(b.half().float())
        pf.infer_to_bc(pm, grids=grids)
        torch.cuda.synchronize()
        p_times = time_events(torch, lambda: pf.infer_to_bc(pm, grids=grids), 2, flush=flush)
        p_ms = float(np.mean(p_times))
        p_outs = pf.infer_to_bc(pm, grids=grids)
        plain_psnr = psnr_list(nt, torch, mat, [o.reshape(-1) for o in p_outs], side)
        # training step of the plain path
        ref_e = [pf.reference_endpoints(f, r) for f, r in zip(mat.formats, refs)]
        texs = [torch.from_numpy(t).to(dev) for t in mat.textures]
        trainer = pf.PlainTrainer(pm, FULL_MAIN_STEPS + FULL_QAT_STEPS)
        ids = torch.randint(0, nblk, (BATCH_TEXELS // 16,), device=dev)
        for _ in range(2):
            trainer.step(texs, ref_e, ids)
        torch.cuda.synchronize()
        pt = time_events(torch, lambda: trainer.step(texs, ref_e, ids), 5)
        p_train_ms = float(np.mean(pt))
        plain = {"infer_value": round(tex_blocks / (p_ms * 1e-3) / 1e6, 3), "unit": "Mblocks/s",
                 "infer_ms": round(p_ms, 3), "psnr_db": plain_psnr,
                 "train_ms_per_step": round(p_train_ms, 3),
                 "encode_s_extrapolated": round(p_train_ms * (FULL_MAIN_STEPS + FULL_QAT_STEPS) / 1e3, 1)}

    # ---- the CPU oracle over the whole material on the host cores: the CPU baseline, and the
    # accuracy parity of the headline blocks (PSNR per texture, field mismatch)
    cpu = oracle_parity = None
    if not args.no_cpu and rank == 0 and world == 1:
        flat = torch.empty(model.n_params, device=dev)
        model.get_params(flat)
        oracle_parity, cpu = full_material_oracle(side, flat.cpu().numpy(), headline_blocks, mat.textures)

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "Mblocks/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp16 tensor-core MMA (split hi+lo activations), fp32 accumulate; u8 grids", "data": "synthetic",
        "config": workload_config(side, world),
        "block_positions_per_s_M": round(nblk * world / (ms * 1e-3) / 1e6, 3),
        "ssim": {"ntbc": ours_ssim, "reference_bc": ref_ssim},
        "psnr_db": {"ntbc": ours_psnr, "untrained": untrained_psnr, "reference_bc": ref_psnr,
                    "reference_bc_unrefined": ref_psnr_unrefined,
                    "e2e": e2e_psnr, "plain_fp32": plain["psnr_db"] if plain else None},
        "encode": {"precision": "bf16 tensor-core MMA operands, fp32 accumulate / loss / Adam",
                   "ms_per_step": round(ms_per_train_step, 3), "steps_run": total_steps,
                   "batch_texels": BATCH_TEXELS, "measured_s": round(train_s, 2),
                   "full_schedule_s_extrapolated": round(encode_full_s, 1),
                   "full_schedule_steps": FULL_MAIN_STEPS + FULL_QAT_STEPS,
                   "last_losses": [round(x, 6) for x in last_losses],
                   "roofline_terms": encode_terms,
                   "reference_bc_encode_ms": round(float(np.mean(ref_ms)), 3),
                   "fp32_kernels": fp32_encode},
        "plain_fp32_gpu": plain,
        "conservative": conservative,
        "batch16": batch16,
        "quality_storage": study,
        "storage": {"ntbc_blob_bytes": int(model.blob_size()), "bc_bytes": int(nblk * 8 * len(FORMATS)),
                    "weights": "FP16", "grids": "u8"},
        "roofline": roofline,
        "roofline_terms": terms,
        "other_modes": modes,
        "cpu_baseline": cpu,
        "oracle_parity": oracle_parity,
        "e2e": {"value": round(e2e_value, 3), "unit": "Mblocks/s", "ms_per_step": round(e2e_ms, 4),
                "h2d_bytes_per_step": int(blob.numel()), "d2h_bytes_per_step": int(nblk * 8 * len(FORMATS)),
                **e2e_parts},
        "clocks": clk,
        "gpu_launches": args.steps * launches_per_pass,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
