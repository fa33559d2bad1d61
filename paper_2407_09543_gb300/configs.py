"""Workload presets (host-side configuration only) and parameter flattening.

Five workloads:
  tiny256  256^2 BC1 + BC4, 4 colour levels 16..128, 2 x 64 ReLU MLPs, FP32,
           500 Adam steps at 4096 texels per step
  mat1k    1024^2 diffuse / normal BC1 + roughness BC4, 8 levels 16..512,
           3 x 64 SELU, 5000 steps at 2^16 texels, FP16 inference
  mat4k    4096^2 diffuse / normal BC1 + roughness / AO BC4, 12 levels
           16..2048, 8-bit QAT grids, 3 x 64 SELU, 20000 + 2000 QAT steps at 2^18
  sweep    mat4k weights with u8 / u4 grids and FP32 / FP16 MLPs
  batch16  16 materials of uneven size (sides 512..4096, 2..5 textures)
The endpoint grid keeps the colour-grid levels whose resolution does not exceed
the number of blocks per side (Sec. 3.4: 7 of the 8 levels for a 4096^2 texture).
Packaging (Sec. 4.1): aggressive = one model per material, conservative = one model for
the BC1 textures and one for the BC4 textures (`packaging_groups`).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from ._abi import ACT_RELU, ACT_SELU, ModelDesc, ntbc_level_resolutions, ntbc_model_layout


@dataclass
class Workload:
    name: str
    side: int
    levels: int
    min_res: int
    max_res: int
    hidden_layers: int
    activation: int
    steps: int
    batch_texels: int
    qat_fraction: float
    grid_bits: int          # exported grid: 0 = FP32, 8 / 4 = QAT codes
    weight_prec: int        # 0 FP32, 1 FP16


WORKLOADS = {
    "tiny256": Workload("tiny256", 256, 4, 16, 128, 2, ACT_RELU, 500, 4096, 0.0, 0, 0),
    "mat1k": Workload("mat1k", 1024, 8, 16, 512, 3, ACT_SELU, 5000, 1 << 16, 0.0, 0, 1),
    "mat4k": Workload("mat4k", 4096, 12, 16, 2048, 3, ACT_SELU, 20000, 1 << 18, 0.1, 8, 1),
}


def packaging_groups(formats, packaging="aggressive"):
    """Texture indices per model (Sec. 4.1): aggressive packaging trains one model for all
    textures of the material; conservative packaging trains one model for the RGB (BC1)
    textures and one for the single-channel (BC4) textures."""
    formats = list(formats)
    if packaging == "aggressive":
        return [list(range(len(formats)))]
    if packaging != "conservative":
        raise ValueError(f"unknown packaging {packaging!r}")
    groups = [[t for t, f in enumerate(formats) if f == 1], [t for t, f in enumerate(formats) if f == 4]]
    return [g for g in groups if g]


def grid_levels(levels, min_res, max_res, side):
    color = ntbc_level_resolutions(levels, min_res, max_res)
    endpoint = [r for r in color if r <= side // 4]
    return color, endpoint


def model_desc(formats, side, levels, min_res, max_res, hidden_layers=3, activation=ACT_SELU, height=None):
    color, endpoint = grid_levels(levels, min_res, max_res, side)
    return ModelDesc.make(side, height or side, list(formats), color, endpoint, hidden_layers, activation)


def desc_for(workload: Workload, formats, side=None):
    side = side or workload.side
    return model_desc(formats, side, workload.levels, workload.min_res, workload.max_res,
                      workload.hidden_layers, workload.activation)


def mlp_dims(desc: ModelDesc, which: str):
    lay = ntbc_model_layout(desc)
    hidden = [desc.hidden_width] * desc.hidden_layers
    if which == "color":
        return [lay.in_color] + hidden + [lay.out_color]
    return [lay.in_endpoint] + hidden + [lay.out_endpoint]


def res_lists(desc: ModelDesc):
    return ([desc.color_res[i] for i in range(desc.color_levels)],
            [desc.endpoint_res[i] for i in range(desc.endpoint_levels)])


def flatten(desc: ModelDesc, params: dict) -> np.ndarray:
    """dict(color_grid=[...], endpoint_grid=[...], color_mlp=[(W, b)], endpoint_mlp=[...]) -> flat FP32
    in the layout order of include/ntbc.h."""
    lay = ntbc_model_layout(desc)
    flat = np.zeros(lay.total, np.float32)

    def put(span, arr):
        a = np.asarray(arr, np.float32).ravel()
        assert a.size == span.count, (a.size, span.count)
        flat[span.offset:span.offset + span.count] = a

    for l, g in enumerate(params["color_grid"]):
        put(lay.color_grid[l], g)
    for l, g in enumerate(params["endpoint_grid"]):
        put(lay.endpoint_grid[l], g)
    for l, (W, b) in enumerate(params["color_mlp"]):
        put(lay.color_w[l], W)
        put(lay.color_b[l], b)
    for l, (W, b) in enumerate(params["endpoint_mlp"]):
        put(lay.endpoint_w[l], W)
        put(lay.endpoint_b[l], b)
    return flat


def unflatten(desc: ModelDesc, flat) -> dict:
    lay = ntbc_model_layout(desc)
    flat = np.asarray(flat)
    cres, eres = res_lists(desc)

    def get(span, shape):
        return flat[span.offset:span.offset + span.count].reshape(shape)

    out = dict(color_grid=[get(lay.color_grid[l], (r, r, 2)) for l, r in enumerate(cres)],
               endpoint_grid=[get(lay.endpoint_grid[l], (r, r, 2)) for l, r in enumerate(eres)],
               color_mlp=[], endpoint_mlp=[])
    for which, ws, bs in (("color", lay.color_w, lay.color_b), ("endpoint", lay.endpoint_w, lay.endpoint_b)):
        dims = mlp_dims(desc, which)
        for l in range(len(dims) - 1):
            out[which + "_mlp"].append((get(ws[l], (dims[l + 1], dims[l])), get(bs[l], (dims[l + 1],))))
    return out
