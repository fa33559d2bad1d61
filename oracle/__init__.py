"""CPU oracle for the NTBC hot path: a plain, slow, FP64 restatement of the paper.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package; the product path never does, and it
shares no code with the CUDA path (only the seeded generators in `synth` feed both).

  bc      -- BC1 / BC4 codec, reference encoder, PSNR   (Sec. 2.1, Sec. 4.1, Sec. 4.3)
  ntbc    -- grids, MLPs, inference to blocks, losses + straight-through backward,
             QAT, Adam and LR schedule                 (Sec. 2.3, Sec. 3, Sec. 3.4, App. A)
  philox  -- Philox4x32-10 batch sampler               (Salmon et al. 2011)

Parity status of each function is recorded with its tests; every function here
is pinned by a test against values the paper prints, closed forms, invariants or
brute force.
"""
from . import bc, ntbc, philox  # noqa: F401
