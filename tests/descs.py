"""Model descriptions for the parity tests: the oracle's from oracle/ alone, the library's
checked against it.

The oracle's grid-level ladder (geometric from the coarsest to the finest resolution,
Sec. 3.4), its endpoint-grid levels (the colour levels not finer than the blocks per side)
and its MLP sizes come from oracle/ntbc.py; the library's description of the same model is
built through the library and must agree with it exactly, so no oracle input is taken from
the product.
"""
import synth
from oracle import ntbc as ont


def oracle_desc(formats, width, levels, lo, hi, hidden=3, act="selu", height=None):
    cres = ont.level_resolutions(levels, lo, hi)
    eres = ont.endpoint_resolutions(cres, width // 4)
    return ont.ModelDesc(width, height or width, list(formats), cres, eres, hidden_layers=hidden, activation=act)


def product_desc(nt, od, levels, lo, hi):
    """The library's description (its own level ladder) of the oracle's model, asserted equal."""
    acti = nt.ACT_SELU if od.activation == "selu" else nt.ACT_RELU
    desc = nt.configs.model_desc(od.formats, od.width, levels, lo, hi, od.hidden_layers, acti, height=od.height)
    assert nt.configs.res_lists(desc) == (list(od.color_res), list(od.endpoint_res)), "grid ladders differ"
    for which in ("color", "endpoint"):
        assert nt.configs.mlp_dims(desc, which) == od.mlp_dims(which), f"{which} MLP sizes differ"
    return desc


def case_descs(nt, formats, width, levels, lo, hi, hidden=3, act="selu", height=None):
    """(library desc, oracle desc) of one test model."""
    od = oracle_desc(formats, width, levels, lo, hi, hidden, act, height)
    return product_desc(nt, od, levels, lo, hi), od


def init_params(od, seed):
    """Initial parameters (Sec. 3.4 initialisation) sized by the oracle's description."""
    return synth.init_params(od.color_res, od.endpoint_res, od.features, od.mlp_dims("color"),
                             od.mlp_dims("endpoint"), seed)


def params_from_flat(od, flat):
    """A flat parameter vector (the C ABI's order) split by the oracle's own reader."""
    return ont.params_from_flat(od, flat)


def as_float32(params):
    """The same parameters rounded to FP32 (what the library stores), kept as float64 arrays."""
    import numpy as np

    f = lambda a: np.asarray(a, np.float32).astype(np.float64)
    out = dict(color_grid=[f(g) for g in params["color_grid"]], endpoint_grid=[f(g) for g in params["endpoint_grid"]])
    for k in ("color_mlp", "endpoint_mlp"):
        out[k] = [(f(W), f(b)) for W, b in params[k]]
    return out
