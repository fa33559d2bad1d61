"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds no arithmetic of the compression method itself. It only draws
data: procedural texture content standing in for the paper's 4096^2 ambientCG /
Poly Haven materials (Sec. 4.2; the dataset is not available here), and the
random initial parameters of a model (He-normal MLP weights, zero biases, and
U[-1e-4, 1e-4] grid features, Sec. 3.4), which both sides receive as inputs.

Every array is a deterministic function of a string key and an integer seed
(SHA-256 of the key feeds numpy's SeedSequence), so the same call gives the same
bytes on x86 and on Arm.

Texture recipes (all uint8, row-major, H x W x C):
  * diffuse (RGB): 8 sinusoids with random frequency (1..64 cycles per side),
    orientation and phase, plus 4-octave value noise (octave cell W/8/2^o,
    amplitude 0.5^o, smoothstep interpolation), mixed per channel.
  * normal (RGB): tangent-space normal of a seeded fBm height field h,
    n = normalize(-k dh/du, -k dh/dv, 1), stored as (n + 1) / 2 * 255.
  * roughness (R): smooth noise pushed through its empirical CDF and then the
    inverse CDF of Beta(2, 5).
  * ao (R): 1 - normalised cavity of h.
  * cracks (4k material only): ~64 random-walk polylines, 1-2 px wide, that
    darken diffuse and AO, raise roughness and carve into h.
"""
from __future__ import annotations

import hashlib
from dataclasses import dataclass, field

import numpy as np

BC1 = 1
BC4 = 4


def _rng(*key) -> np.random.Generator:
    digest = hashlib.sha256(repr(key).encode()).digest()
    words = [int.from_bytes(digest[i:i + 4], "little") for i in range(0, 32, 4)]
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(words)))


# ----------------------------------------------------------------------------
# procedural fields (float64 in [0, 1]-ish, shape H x W)
# ----------------------------------------------------------------------------

def _smoothstep(t):
    return t * t * (3.0 - 2.0 * t)


def value_noise(rng: np.random.Generator, w: int, h: int, cell: float) -> np.ndarray:
    """Lattice value noise with smoothstep interpolation; lattice spacing `cell` texels."""
    cell = max(float(cell), 1.0)
    gx = int(np.ceil(w / cell)) + 2
    gy = int(np.ceil(h / cell)) + 2
    lat = rng.random((gy, gx))
    x = (np.arange(w) + 0.5) / cell
    y = (np.arange(h) + 0.5) / cell
    ix = np.floor(x).astype(np.int64)
    iy = np.floor(y).astype(np.int64)
    sx = _smoothstep(x - ix)
    sy = _smoothstep(y - iy)
    rows = lat[:, ix] * (1.0 - sx) + lat[:, ix + 1] * sx          # gy x w
    return rows[iy] * (1.0 - sy)[:, None] + rows[iy + 1] * sy[:, None]


def octave_noise(rng, w, h, base_cell, octaves=4):
    acc = np.zeros((h, w))
    norm = 0.0
    for o in range(octaves):
        amp = 0.5 ** o
        acc += amp * value_noise(rng, w, h, base_cell / 2 ** o)
        norm += amp
    return acc / norm


def sinusoids(rng, w, h, count=8):
    x = (np.arange(w) + 0.5) / w
    y = (np.arange(h) + 0.5) / h
    acc = np.zeros((h, w))
    for _ in range(count):
        freq = rng.uniform(1.0, 64.0)
        theta = rng.uniform(0.0, np.pi)
        phase = rng.uniform(0.0, 2 * np.pi)
        amp = rng.uniform(0.3, 1.0)
        # separable evaluation of sin(a*x + b*y + phase) = sin(ax)cos(by+p) + cos(ax)sin(by+p)
        ax = 2 * np.pi * freq * np.cos(theta) * x
        by = 2 * np.pi * freq * np.sin(theta) * y + phase
        acc += amp * (np.outer(np.cos(by), np.sin(ax)) + np.outer(np.sin(by), np.cos(ax)))
    return acc


def _normalise(f):
    lo, hi = f.min(), f.max()
    return (f - lo) / (hi - lo) if hi > lo else np.zeros_like(f)


def _to_u8(f):
    return np.clip(np.floor(f * 255.0 + 0.5), 0, 255).astype(np.uint8)


def fbm_height(rng, w, h, octaves=6):
    return _normalise(octave_noise(rng, w, h, w / 16.0, octaves))


def box_blur(f, radius):
    """Separable box blur with clamped borders (summed-area along each axis)."""
    r = max(int(radius), 1)
    out = f
    for axis in (0, 1):
        pad = [(0, 0), (0, 0)]
        pad[axis] = (r + 1, r)
        p = np.pad(out, pad, mode="edge")
        c = np.cumsum(p, axis=axis)
        n = out.shape[axis]
        hi = np.take(c, np.arange(2 * r + 1, 2 * r + 1 + n), axis=axis)
        lo = np.take(c, np.arange(0, n), axis=axis)
        out = (hi - lo) / (2 * r + 1)
    return out


def beta25_inverse_cdf(p: np.ndarray) -> np.ndarray:
    """Inverse CDF of Beta(2,5), F(x) = 1 - (1-x)^6 - 6x(1-x)^5, by bisection on a table."""
    q = np.linspace(0.0, 1.0, 4097)
    lo = np.zeros_like(q)
    hi = np.ones_like(q)
    for _ in range(48):
        mid = 0.5 * (lo + hi)
        F = 1.0 - (1.0 - mid) ** 6 - 6.0 * mid * (1.0 - mid) ** 5
        below = F < q
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return np.interp(p, q, 0.5 * (lo + hi))


def crack_mask(rng, w, h, count=64):
    mask = np.zeros((h, w), dtype=bool)
    steps = max(w // 8, 16)
    for _ in range(count):
        x0, y0 = rng.uniform(0, w), rng.uniform(0, h)
        ang = rng.uniform(0, 2 * np.pi) + np.cumsum(rng.normal(0.0, 0.25, steps))
        xs = x0 + np.cumsum(np.cos(ang))
        ys = y0 + np.cumsum(np.sin(ang))
        width = int(rng.integers(1, 3))
        xi = np.clip(np.round(xs).astype(np.int64), 0, w - 1)
        yi = np.clip(np.round(ys).astype(np.int64), 0, h - 1)
        mask[yi, xi] = True
        if width == 2:
            mask[yi, np.minimum(xi + 1, w - 1)] = True
            mask[np.minimum(yi + 1, h - 1), xi] = True
    return mask


# ----------------------------------------------------------------------------
# textures
# ----------------------------------------------------------------------------

def diffuse_texture(rng, w, h, channels=3):
    sines = _normalise(sinusoids(rng, w, h, 8))
    noise = octave_noise(rng, w, h, w / 8.0, 4)
    out = np.empty((h, w, channels), dtype=np.float64)
    for c in range(channels):
        a, b = rng.uniform(0.2, 0.8, 2)
        base = rng.uniform(0.0, 0.3)
        gain = rng.uniform(0.5, 1.0)
        out[..., c] = base + gain * _normalise(a * sines + b * noise)
    return np.clip(out, 0.0, 1.0)


def normal_texture(height, strength=1.0 / 16.0):
    h, w = height.shape
    dhdv, dhdu = np.gradient(height)
    dhdu = dhdu * w
    dhdv = dhdv * h
    n = np.stack([-strength * dhdu, -strength * dhdv, np.ones_like(height)], axis=-1)
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    return (n + 1.0) * 0.5


def roughness_texture(rng, w, h):
    field_ = octave_noise(rng, w, h, w / 8.0, 4)
    ranks = np.empty(field_.size, dtype=np.float64)
    ranks[np.argsort(field_, axis=None, kind="stable")] = (np.arange(field_.size) + 0.5) / field_.size
    return beta25_inverse_cdf(ranks.reshape(h, w))


def ao_texture(height, w):
    cavity = np.maximum(box_blur(height, max(w // 128, 2)) - height, 0.0)
    top = np.percentile(cavity, 99.0)
    cavity = np.minimum(cavity / top, 1.0) if top > 0 else cavity
    return 1.0 - 0.7 * cavity


@dataclass
class Material:
    """A material: same-size textures, each with its BC format (1 = BC1 RGB, 4 = BC4 R)."""
    name: str
    width: int
    height: int
    formats: list = field(default_factory=list)
    textures: list = field(default_factory=list)   # uint8 arrays, H x W x 3 (BC1) or H x W (BC4)
    kinds: list = field(default_factory=list)

    @property
    def blocks_per_texture(self):
        return (self.width // 4) * (self.height // 4)


def make_material(name: str, side: int, kinds, seed: int = 0, cracks: bool = False) -> Material:
    """Build a material from texture kinds: 'diffuse', 'normal', 'roughness', 'ao',
    'sine_rgb' / 'sine_r' (sinusoids + value noise, RGB or single channel)."""
    w = h = int(side)
    rng = _rng("material", name, side, tuple(kinds), seed, cracks)
    height = fbm_height(rng, w, h)
    mask = crack_mask(rng, w, h) if cracks else None
    if mask is not None:
        height = np.where(mask, height - 0.35, height)
    mat = Material(name=name, width=w, height=h)
    for kind in kinds:
        if kind in ("diffuse", "sine_rgb"):
            tex = diffuse_texture(rng, w, h, 3)
            if mask is not None:
                tex = np.where(mask[..., None], tex * 0.35, tex)
            fmt = BC1
        elif kind == "sine_r":
            tex = diffuse_texture(rng, w, h, 1)[..., 0]
            fmt = BC4
        elif kind == "normal":
            tex = normal_texture(height)
            fmt = BC1
        elif kind == "roughness":
            tex = roughness_texture(rng, w, h)
            if mask is not None:
                tex = np.where(mask, 0.95, tex)
            fmt = BC4
        elif kind == "ao":
            tex = ao_texture(height, w)
            if mask is not None:
                tex = np.where(mask, tex * 0.4, tex)
            fmt = BC4
        else:
            raise ValueError(f"unknown texture kind {kind!r}")
        mat.formats.append(fmt)
        mat.textures.append(np.ascontiguousarray(_to_u8(tex)))
        mat.kinds.append(kind)
    return mat


# Named workloads.  Sizes and texture mixes follow the five benchmark
# configurations: a 256^2 BC1+BC4 pair, a 1024^2 three-texture material, the
# full 4096^2 four-texture material with cracks, and a batch of 16 materials of
# uneven size.
def tiny_material(seed=0):
    return make_material("tiny256", 256, ["sine_rgb", "sine_r"], seed)


def material_1k(seed=0):
    return make_material("mat1k", 1024, ["diffuse", "normal", "roughness"], seed)


def material_4k(seed=0, side=4096):
    return make_material("mat4k", side, ["diffuse", "normal", "roughness", "ao"], seed, cracks=True)


def material_batch_spec(seed=0, count=16):
    """(side, kinds) of each material of an uneven batch: sides from {512, 1024, 2048,
    4096}, 2 to 5 textures each, at least one RGB texture."""
    rng = _rng("batch", seed, count)
    pool = ["diffuse", "normal", "roughness", "ao"]
    spec = []
    for _ in range(count):
        side = int(rng.choice([512, 1024, 2048, 4096]))
        n = int(rng.integers(2, 6))
        kinds = [pool[int(k)] for k in rng.integers(0, 4, n)]
        if all(k in ("roughness", "ao") for k in kinds):
            kinds[0] = "diffuse"
        spec.append((side, kinds))
    return spec


def material_batch(seed=0, count=16):
    return [make_material(f"batch{seed}_{i}", side, kinds, seed + 1000 * i, cracks=(side == 4096))
            for i, (side, kinds) in enumerate(material_batch_spec(seed, count))]


# ----------------------------------------------------------------------------
# initial parameters (Sec. 3.4): He-normal weights, zero biases, U[-1e-4, 1e-4] grids
# ----------------------------------------------------------------------------

def init_params(grid_res_color, grid_res_endpoint, features, mlp_color_dims, mlp_endpoint_dims, seed=0):
    """Random initial parameters as float32 arrays.

    grid_res_*: per-level resolutions; each level is a res x res x features array.
    mlp_*_dims: [in, hidden..., out]; layer i has weight [dims[i+1], dims[i]] and bias [dims[i+1]].
    Returns dict(color_grid=[...], endpoint_grid=[...], color_mlp=[(W, b), ...], endpoint_mlp=[...]).
    """
    rng = _rng("init", tuple(grid_res_color), tuple(grid_res_endpoint), features,
               tuple(mlp_color_dims), tuple(mlp_endpoint_dims), seed)

    def grid(res_list):
        return [rng.uniform(-1e-4, 1e-4, (r, r, features)).astype(np.float32) for r in res_list]

    def mlp(dims):
        layers = []
        for i in range(len(dims) - 1):
            fan_in = dims[i]
            wgt = (rng.standard_normal((dims[i + 1], fan_in)) * np.sqrt(2.0 / fan_in)).astype(np.float32)
            layers.append((wgt, np.zeros(dims[i + 1], dtype=np.float32)))
        return layers

    return dict(color_grid=grid(grid_res_color), endpoint_grid=grid(grid_res_endpoint),
                color_mlp=mlp(mlp_color_dims), endpoint_mlp=mlp(mlp_endpoint_dims))


def random_params_like(params, seed=0, grid_scale=0.5, weight_scale=1.0):
    """Random non-trivial parameters of the same shapes (grids U[-grid_scale, grid_scale]),
    used where a test needs a network whose outputs spread over [0, 1]."""
    rng = _rng("random_like", seed, grid_scale, weight_scale)
    out = dict(color_grid=[], endpoint_grid=[], color_mlp=[], endpoint_mlp=[])
    for k in ("color_grid", "endpoint_grid"):
        out[k] = [rng.uniform(-grid_scale, grid_scale, g.shape).astype(np.float32) for g in params[k]]
    for k in ("color_mlp", "endpoint_mlp"):
        for wgt, b in params[k]:
            fan_in = wgt.shape[1]
            out[k].append(((rng.standard_normal(wgt.shape) * weight_scale * np.sqrt(2.0 / fan_in)).astype(np.float32),
                           (rng.standard_normal(b.shape) * 0.1).astype(np.float32)))
    return out


def random_blocks_texels(n_blocks, fmt, seed=0, kind="mixed"):
    """Random 4x4 blocks for codec tests: returns an (n_blocks*4) x 4 x C texture strip
    laid out as a 4-texel-high row of blocks, mixing uniform noise, two-colour,
    solid and smooth-gradient blocks."""
    rng = _rng("blocks", n_blocks, fmt, seed, kind)
    ch = 3 if fmt == BC1 else 1
    blk = rng.integers(0, 256, (n_blocks, 16, ch))
    if kind == "mixed":
        sel = rng.integers(0, 4, n_blocks)
        two = rng.integers(0, 256, (n_blocks, 2, ch))
        pick = rng.integers(0, 2, (n_blocks, 16))
        blk = np.where((sel == 1)[:, None, None], np.take_along_axis(two, pick[..., None].repeat(ch, -1), 1), blk)
        blk = np.where((sel == 2)[:, None, None], two[:, :1, :], blk)
        ramp = (np.arange(16) / 15.0)[None, :, None]
        grad = np.round(two[:, :1, :] * (1 - ramp) + two[:, 1:, :] * ramp)
        blk = np.where((sel == 3)[:, None, None], grad, blk)
    blk = blk.astype(np.uint8)
    # lay out as a 4 x (4*n_blocks) texture: block b covers columns 4b..4b+3
    tex = blk.reshape(n_blocks, 4, 4, ch).transpose(1, 0, 2, 3).reshape(4, n_blocks * 4, ch)
    return tex[..., 0].copy() if ch == 1 else tex.copy()
