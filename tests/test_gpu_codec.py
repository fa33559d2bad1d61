"""GPU parity of the BC codec and of the output-to-block stage (bit-exact vs the oracle)."""
import numpy as np
import pytest
import torch

import synth
from oracle import bc as obc, ntbc as ont

nt = pytest.importorskip("paper_2407_09543_gb300")
pytestmark = pytest.mark.gpu
DEV = "cuda"


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).ravel()).to(DEV)


def gpu_encode(fmt, tex, w, h):
    blocks = torch.empty((w // 4) * (h // 4) * 8, dtype=torch.uint8, device=DEV)
    nt.bc_reference_encode(fmt, _dev(tex), w, h, blocks)
    torch.cuda.synchronize()
    return blocks.cpu().numpy().reshape(-1, 8)


def gpu_decode(fmt, blocks, w, h):
    ch = 3 if fmt == nt.BC1 else 1
    out = torch.empty(w * h * ch, dtype=torch.uint8, device=DEV)
    nt.bc_decode(fmt, _dev(blocks), w, h, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape((h, w, 3) if ch == 3 else (h, w))


@pytest.mark.parametrize("fmt", [1, 4])
def test_reference_encode_bit_exact_material(fmt):
    mat = synth.tiny_material()
    tex = mat.textures[0 if fmt == 1 else 1]
    got = gpu_encode(fmt, tex, 256, 256)
    assert (got == obc.encode(fmt, tex, 256, 256)).all()


@pytest.mark.parametrize("fmt", [1, 4])
@pytest.mark.parametrize("n", [1, 127, 1000, 4099])
def test_reference_encode_bit_exact_mixed_blocks(fmt, n):
    # uniform noise, two-colour, solid and gradient blocks; block counts around the
    # launch's 128-thread tiles (ragged tails)
    tex = synth.random_blocks_texels(n, fmt, seed=n)
    assert (gpu_encode(fmt, tex, 4 * n, 4) == obc.encode(fmt, tex, 4 * n, 4)).all()


@pytest.mark.parametrize("fmt", [1, 4])
def test_reference_encode_non_square_ragged(fmt):
    m = synth.make_material("ragged", 264, ["sine_rgb", "sine_r"], 2)
    tex = m.textures[0 if fmt == 1 else 1][:132]
    assert (gpu_encode(fmt, tex, 264, 132) == obc.encode(fmt, tex, 264, 132)).all()


@pytest.mark.parametrize("fmt", [1, 4])
def test_decode_bit_exact_all_modes(fmt):
    rng = np.random.default_rng(fmt)
    n = 20000
    blocks = rng.integers(0, 256, (n, 8), dtype=np.uint8)
    if fmt == 1:
        blocks[: n // 4, 0:2] = blocks[: n // 4, 2:4]          # c0 == c1 (3-colour mode)
    else:
        blocks[: n // 4, 0] = blocks[: n // 4, 1]              # r0 == r1
    assert (gpu_decode(fmt, blocks, 4 * n, 4) == obc.decode(fmt, blocks, 4 * n, 4)).all()


@pytest.mark.parametrize("fmt", [1, 4])
def test_full_size_4k_sampled(fmt):
    # full 4096^2 texture encoded in one launch; oracle checks a seeded sample of blocks
    mat = synth.material_4k()
    tex = mat.textures[1 if fmt == 1 else 2]
    got = gpu_encode(fmt, tex, 4096, 4096)
    blk = obc.to_blocks(tex, 4096, 4096)
    idx = np.random.default_rng(0).choice(1024 * 1024, 20000, replace=False)
    want = obc.bc1_encode_blocks(blk[idx]) if fmt == 1 else obc.bc4_encode_blocks(blk[idx, :, 0])
    assert (got[idx] == want).all()
    dec = gpu_decode(fmt, got, 4096, 4096)
    assert obc.psnr(dec, tex) == pytest.approx(obc.psnr(obc.decode(fmt, got, 4096, 4096), tex), abs=0)


@pytest.mark.parametrize("fmt", [1, 4])
def test_outputs_to_bc_bit_exact(fmt):
    rng = np.random.default_rng(10 + fmt)
    n = 5000
    C = 3 if fmt == 1 else 1
    e = rng.random((n, 2 * C)).astype(np.float32)
    c = rng.random((n, 16, C)).astype(np.float32)
    e[:50] = e[:50, :C].repeat(2, axis=1) if C == 1 else np.concatenate([e[:50, :3], e[:50, :3]], 1)  # equal endpoints
    c[50:100] = np.round(c[50:100] * 255) / 255                       # on-palette-ish colours
    e[100:120] = np.round(e[100:120] * 31) / 31                        # quantisation boundaries
    out = torch.empty(n * 8, dtype=torch.uint8, device=DEV)
    nt.ntbc_outputs_to_bc(fmt, _dev(e), _dev(c), n, out)
    torch.cuda.synchronize()
    assert (out.cpu().numpy().reshape(-1, 8) == ont.outputs_to_blocks(fmt, e, c)).all()


def test_invalid_arguments_launch_nothing():
    with pytest.raises(nt.NTBCError) as ei:
        nt.bc_reference_encode(1, torch.zeros(30, dtype=torch.uint8, device=DEV), 10, 1,
                               torch.zeros(8, dtype=torch.uint8, device=DEV))
    assert ei.value.status == 1


# ----------------------------------------------------------------------------
# BC3 / BC5: compositions of BC1 and BC4 (16-byte blocks)
# ----------------------------------------------------------------------------

def _comp_texture(fmt, w, h, seed):
    mat = synth.make_material("comp", max(w, h), ["sine_rgb", "sine_r", "sine_r"], seed)
    if fmt == nt.BC3:
        return np.concatenate([mat.textures[0][:h, :w], mat.textures[1][:h, :w, None]], axis=-1)
    return np.stack([mat.textures[1][:h, :w], mat.textures[2][:h, :w]], axis=-1)


@pytest.mark.parametrize("fmt", [3, 5])
def test_composed_formats_encode_and_decode_bit_exact(fmt):
    w, h = 72, 40
    tex = np.ascontiguousarray(_comp_texture(fmt, w, h, 5))
    blocks = torch.empty((w // 4) * (h // 4) * 16, dtype=torch.uint8, device=DEV)
    nt.bc_reference_encode(fmt, _dev(tex), w, h, blocks)
    torch.cuda.synchronize()
    got = blocks.cpu().numpy().reshape(-1, 16)
    np.testing.assert_array_equal(got, obc.encode(fmt, tex, w, h))
    # decode random blocks too (BC3 colour blocks with colour0 <= colour1 included)
    rnd = np.random.default_rng(7).integers(0, 256, got.shape, dtype=np.uint8)
    for b in (got, rnd):
        out = torch.empty(w * h * tex.shape[-1], dtype=torch.uint8, device=DEV)
        nt.bc_decode(fmt, _dev(b), w, h, out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy().reshape(h, w, -1), obc.decode(fmt, b, w, h))


@pytest.mark.parametrize("fmt,refine", [(1, 1), (1, 2), (4, 2), (4, 4)])
def test_refined_reference_encode_bit_exact(fmt, refine):
    mat = synth.tiny_material()
    tex = mat.textures[0 if fmt == 1 else 1]
    blocks = torch.empty(64 * 64 * 8, dtype=torch.uint8, device=DEV)
    nt.bc_reference_encode(fmt, _dev(tex), 256, 256, blocks, refine=refine)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(blocks.cpu().numpy().reshape(-1, 8), obc.encode_refined(fmt, tex, 256, 256, refine))


def test_refined_reference_encode_4k_sampled_and_better():
    # the 4096^2 material: sampled blocks bit-exact, and a higher decoded PSNR than unrefined
    mat = synth.material_4k(seed=0)
    for t, fmt in enumerate(mat.formats):
        tex = mat.textures[t]
        base = torch.empty(1024 * 1024 * 8, dtype=torch.uint8, device=DEV)
        ref2 = torch.empty_like(base)
        d = _dev(tex)
        nt.bc_reference_encode(fmt, d, 4096, 4096, base)
        nt.bc_reference_encode(fmt, d, 4096, 4096, ref2, refine=2)
        torch.cuda.synchronize()
        got = ref2.cpu().numpy().reshape(-1, 8)
        rows = np.random.default_rng(t).choice(1024, 8, replace=False)
        for by in rows:                                   # whole block rows: 16 texel rows x 4096
            sub = tex[4 * by:4 * by + 4]
            want = obc.encode_refined(fmt, sub, 4096, 4, 2)
            np.testing.assert_array_equal(got[by * 1024:(by + 1) * 1024], want)
        p0 = obc.psnr(obc.decode(fmt, base.cpu().numpy(), 4096, 4096), tex)
        p2 = obc.psnr(obc.decode(fmt, got, 4096, 4096), tex)
        assert p2 > p0
