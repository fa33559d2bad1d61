"""C ABI checks that need no GPU: the library loads, exports every entry point that
include/ntbc.h declares, validates arguments on the host (no launch), and its host-
side configuration logic agrees with the oracle."""
import ctypes
import os
import re
import subprocess
import sys

import numpy as np
import pytest

import descs
from conftest import ROOT, golden
from oracle import ntbc as ont

nt = pytest.importorskip("paper_2407_09543_gb300")


def declared_functions():
    with open(os.path.join(ROOT, "include", "ntbc.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(\w+)\s*\([^;{]*\)\s*;", text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert "ntbc_infer_to_bc" in names and "bc_reference_encode" in names and len(names) >= 20
    for n in names:
        assert hasattr(nt.lib, n), n


def test_enum_values_match_the_header():
    with open(os.path.join(ROOT, "include", "ntbc.h")) as f:
        text = f.read()
    values = {k: int(v) for k, v in re.findall(r"\b(NTBC_(?:PREC|ACT|BC|TRAIN|BATCH)_?\w*)\s*=\s*(\d+)", text)}
    for name in ("PREC_FP32", "PREC_FP16", "PREC_FP16_FAST", "PREC_FP8", "PREC_FP8_MMA", "ACT_SELU", "ACT_RELU",
                 "TRAIN_FP32", "TRAIN_BF16", "BATCH_CHAINED", "BATCH_QUEUE"):
        assert values["NTBC_" + name] == getattr(nt, name), name


def test_level_resolutions_agree_with_oracle():
    for L, lo, hi in ((8, 16, 2048), (12, 16, 2048), (4, 16, 128), (8, 16, 512), (5, 7, 333), (1, 16, 16)):
        assert nt.ntbc_level_resolutions(L, lo, hi) == ont.level_resolutions(L, lo, hi)


def test_layout_counts_agree_with_oracle_storage():
    g = golden("paper_numbers.txt")
    for formats in ([1, 1, 4, 4, 4, 4], [1, 1], [4, 4, 4, 4], [1, 4]):
        desc, od = descs.case_descs(nt, formats, 4096, 8, 16, 2048, 3, "selu")
        lay = nt.ntbc_model_layout(desc)
        # FP32 everywhere: storage_bytes with 32-bit grids and 4-byte weights is 4 * layout.total
        assert ont.storage_bytes(od, grid_bits=32, weight_bytes=4) == 4 * lay.total
        assert lay.in_color == int(g["color_input_dims"][0])
        assert lay.in_endpoint == int(g["endpoint_input_dims"][0])


def test_host_validation_errors():
    with pytest.raises(nt.NTBCError) as e:
        nt.bc_reference_encode(1, 1, 10, 8, 1, stream=0)
    assert e.value.status == 1 and "multiples of 4" in str(e.value)
    with pytest.raises(nt.NTBCError) as e:
        nt.bc_decode(2, 1, 8, 8, 1, stream=0)
    assert e.value.status == 1
    with pytest.raises(nt.NTBCError) as e:
        nt.bc_decode(1, 0, 8, 8, 1, stream=0)
    assert e.value.status == 1
    nt.ntbc_outputs_to_bc(1, 1, 1, 0, 1, stream=0)             # empty input: nothing to do
    d = nt.configs.model_desc([1, 4], 64, 3, 4, 16)
    d.hidden_width = 32
    with pytest.raises(nt.NTBCError) as e:
        nt.ntbc_model_layout(d)
    assert e.value.status == 6
    d = nt.configs.model_desc([1, 4], 64, 3, 4, 16)
    d.n_textures = 9
    with pytest.raises(nt.NTBCError):
        nt.ntbc_model_layout(d)
    d = nt.configs.model_desc([1, 4], 64, 3, 4, 16)
    d.color_res[1] = 1
    with pytest.raises(nt.NTBCError):
        nt.ntbc_model_layout(d)
    with pytest.raises(nt.NTBCError):
        nt.ntbc_level_resolutions(0, 16, 32)
    with pytest.raises(nt.NTBCError):
        nt.ntbc_sample_blocks(0, 0, 10, 0, 1, stream=0)
    # refinement steps outside 0..16 (valid dummy pointers: nothing is launched)
    with pytest.raises(nt.NTBCError) as e:
        nt.bc_reference_encode(1, 16, 8, 8, 16, stream=0, refine=17)
    assert e.value.status == 1 and "0..16" in str(e.value)
    # the bounded-wait probe's poll count is checked before anything runs
    for bad in (0, (1 << 18) + 1):
        status, _ = nt.ntbc_wait_probe(bad)
        assert status == 1
    # host delivery: no model
    arr = (ctypes.c_void_p * 1)(16)
    assert nt.lib.ntbc_infer_to_host(None, arr, 4, None) == 1


def test_injected_allocation_failure_reports_enomem():
    # host-side fault injection: the allocator fails before any device call
    code = ("import paper_2407_09543_gb300 as nt\n"
            "d = nt.configs.model_desc([1, 4], 64, 3, 4, 16)\n"
            "try:\n    nt.Model(d)\nexcept nt.NTBCError as e:\n    print(e.status)\n")
    env = dict(os.environ, NTBC_FAULT="alloc", PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=120)
    assert out.stdout.strip().splitlines()[-1] == "2", out.stdout + out.stderr


def test_smallest_material():
    # one 4x4 block leaves the endpoint grid no level (every level has res >= 2 > 1 block per
    # side), so the description is refused before anything is allocated; 8x8 (2x2 blocks) is the
    # smallest material with an endpoint grid
    with pytest.raises(nt.NTBCError) as e:
        nt.ntbc_model_layout(nt.configs.model_desc([1, 4], 4, 2, 2, 4, 2, nt.ACT_SELU))
    assert e.value.status == 1
    d = nt.configs.model_desc([1, 4], 8, 2, 2, 8, 2, nt.ACT_SELU)
    assert d.endpoint_levels == 1 and nt.ntbc_model_layout(d).in_endpoint == 2
