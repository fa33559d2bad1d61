"""The bench's full-material oracle leg on the CPU: the oracle, spread over spawned worker
processes, compared with a planted set of "GPU" blocks. Identical blocks meet the bars, a
flipped index field is counted, a corrupted texture breaks the PSNR bar. No GPU and no product
code are involved (the planted blocks come from the oracle itself)."""
import numpy as np

import bench
import synth
from oracle import ntbc as ont


def _case(side=64):
    mat = synth.material_4k(seed=0, side=side)
    spec = bench.workload_spec(side, seed=0)
    od = bench.oracle_desc_of(spec)
    p = bench.oracle_random_params(od, 0)
    flat = np.concatenate([np.asarray(a, np.float32).ravel() for a in ont.flatten_params(p)])
    pool = bench.OraclePool(spec, cores=2)
    blocks, _ = pool.blocks()
    pool.close()
    return mat, od, flat, blocks


def test_full_material_oracle_leg_counts_and_bars():
    side = 64
    mat, od, flat, blocks = _case(side)
    par, cpu = bench.full_material_oracle(side, flat, [b.copy() for b in blocks], mat.textures)
    assert par["blocks"] == od.n_blocks and par["pass"]
    assert par["endpoint_field_mismatch"] == 0 and par["index_field_mismatch"] == 0
    assert all(d == 0 for d in par["psnr_diff_db"])
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] > 0
    # one flipped code bit of block 5 in texture 0 (BC1: byte 4 holds texels 0..3)
    g = [b.copy() for b in blocks]
    g[0][5, 4] ^= 1
    par, _ = bench.full_material_oracle(side, flat, g, mat.textures)
    assert par["index_field_mismatch"] == 1 and par["endpoint_field_mismatch"] == 0
    # a texture decoded from garbage misses the PSNR bar
    g = [b.copy() for b in blocks]
    g[2][:] = np.random.default_rng(1).integers(0, 256, g[2].shape, dtype=np.uint8)
    par, _ = bench.full_material_oracle(side, flat, g, mat.textures)
    assert not par["pass"] and abs(par["psnr_diff_db"][2]) > 0.05
