"""Python binding of libntbc (the C ABI in include/ntbc.h).

Argument marshalling only: every step of the compression path runs in the CUDA
kernels of libntbc.so. PyTorch supplies device memory and streams. Importing
this package fails loudly when the library has not been built (there is no CPU
fallback); build it with `python -m paper_2407_09543_gb300.build` or
`__graft_entry__.build()`.

Entry points keep the C names: bc_reference_encode, bc_decode,
ntbc_outputs_to_bc, ntbc_infer_to_bc, ntbc_forward, ntbc_train_grads,
ntbc_adam_step, ntbc_sample_blocks, ntbc_train, plus the Model wrapper around
the opaque ntbc_model handle.
"""
from __future__ import annotations

import ctypes
import os

from ._abi import (  # noqa: F401
    BC1, BC3, BC4, BC5, ACT_RELU, ACT_SELU, PREC_FP16, PREC_FP16_FAST, PREC_FP32, PREC_FP8, PREC_FP8_MMA, TRAIN_FP32, TRAIN_BF16, MAX_LEVELS, MAX_TEXTURES,
    MAX_MLP_LAYERS, BATCH_CHAINED, BATCH_QUEUE,
    NTBCError, ModelDesc, Layout, Material, TrainConfig, lib, library_path,
    bc_reference_encode, bc_decode, ntbc_outputs_to_bc, ntbc_level_resolutions, ntbc_model_layout,
    ntbc_sample_blocks, ntbc_train_grads_noalloc, ntbc_wait_probe, ntbc_ex2_rate_probe, NOALLOC_MAX_BLOCKS, Model, Batch, STATUS_NAMES,
)
from . import configs  # noqa: F401
from .autograd import NTBCFunction, ntbc_apply  # noqa: F401
