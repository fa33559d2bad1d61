"""Roofline arithmetic of the benchmark, pinned to the per-block counts derived by hand for
the 4096^2 four-texture material (Sec. 3.4 network: 3 x 64 SELU; 12 colour levels, 10
endpoint levels, 2 features each; outputs 3 + 3 + 1 + 1 colour, 6 + 6 + 2 + 2 endpoint)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

nt = pytest.importorskip("paper_2407_09543_gb300")
import bench  # noqa: E402


def _desc():
    return nt.configs.desc_for(nt.configs.WORKLOADS["mat4k"], [nt.BC1, nt.BC1, nt.BC4, nt.BC4], side=4096)


def test_inference_counts_per_block():
    # colour MLP per texel: 24*64 + 64*64 + 64*64 + 64*8 = 10,240 MAC; endpoint per block:
    # 20*64 + 64*64 + 64*64 + 64*16 = 10,496 MAC -> 2 * (16 * 10,240 + 10,496) = 348,672 FLOP
    # per block position; exponentials 16 * (3*64 + 8) + 3*64 + 16 = 3,408
    roof, terms = bench.inference_roofline(nt, _desc(), 2.0)
    n_pos = 1024 * 1024
    assert terms["flop_per_pass"] == 348_672 * n_pos
    assert terms["exp_per_pass"] == 3_408 * n_pos
    # grid codes read once (one byte per feature) + 8-byte blocks of four textures
    lay = nt.ntbc_model_layout(_desc())
    assert terms["hbm_bytes_per_pass"] == lay.grid_floats + 32 * n_pos
    # MUFU peak without a live measurement: 152 SMs x 32 exp2 per clock (the rate measured on
    # GB300) x 2.07 GHz; a live measurement replaces it
    assert roof["peak"] == pytest.approx(152 * 32 * 2.07e9 / 1e12, rel=1e-4)
    assert bench.inference_roofline(nt, _desc(), 2.0, mufu_peak=9.5e12)[0]["peak"] == pytest.approx(9.5)
    assert roof["bound"] == "alu" and roof["unit"] == "Texp/s"
    assert roof["achieved"] == pytest.approx(3_408 * n_pos / 2.0e-3 / 1e12, rel=1e-3)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"], rel=1e-3)


def test_encode_counts_per_step():
    # forward + backward ~ 3x the forward MACs over 2^18 texels and 2^14 blocks
    terms = bench.encode_roofline(nt, _desc(), 0.4)
    assert terms["flop_per_step"] == 3 * 2 * ((1 << 18) * 10_240 + (1 << 14) * 10_496)
    # dense Adam (read p, g, m, v; write p, m, v) + one read of the grids (no dense gradient clear)
    lay = nt.ntbc_model_layout(_desc())
    assert terms["hbm_bytes_per_step"] == lay.total * 4 * 8


def test_job_throughput_is_whole_job():
    # texture blocks of every rank over the slowest rank's time, in millions per second
    assert bench.job_throughput(4_194_304, 1, 2.0) == pytest.approx(4_194_304 / 2e-3 / 1e6)
    assert bench.job_throughput(4_194_304, 8, 2.0) == pytest.approx(8 * 4_194_304 / 2e-3 / 1e6)
