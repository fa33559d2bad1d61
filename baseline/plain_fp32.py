"""Plain FP32 GPU path: the same NTBC algorithm written as PyTorch eager FP32 ops.

This is the comparison baseline of the benchmark, not part of the product: grid
gather by tensor indexing, torch.matmul per layer (TF32 disabled), autograd for
training with the straight-through estimators written as
`hard + (soft - soft.detach())`, torch.optim.Adam, and torch ops for endpoint
quantisation, argmax and packing. It follows the same readings of the paper as
the CUDA path (corner-aligned bilinear grids, linear-order palettes for the
losses, hardware-code order and FP32 decisions for inference).
"""
from __future__ import annotations

import math

import torch

BC1, BC4 = 1, 4


def _setup():
    torch.backends.cuda.matmul.allow_tf32 = False
    torch.backends.cudnn.allow_tf32 = False


class PlainModel:
    def __init__(self, width, height, formats, color_res, endpoint_res, params, activation="selu", device="cuda"):
        """params: dict(color_grid=[...], endpoint_grid=[...], color_mlp=[(W, b)], endpoint_mlp=[...]) of arrays."""
        _setup()
        self.w, self.h = width, height
        self.bw, self.bh = width // 4, height // 4
        self.formats = list(formats)
        self.ch = [3 if f == BC1 else 1 for f in formats]
        self.coff = [sum(self.ch[:i]) for i in range(len(formats))]
        self.act = activation
        t = lambda a: torch.tensor(a, dtype=torch.float32, device=device)  # noqa: E731
        self.color_grid = [t(g).requires_grad_() for g in params["color_grid"]]
        self.endpoint_grid = [t(g).requires_grad_() for g in params["endpoint_grid"]]
        self.color_mlp = [(t(W).requires_grad_(), t(b).requires_grad_()) for W, b in params["color_mlp"]]
        self.endpoint_mlp = [(t(W).requires_grad_(), t(b).requires_grad_()) for W, b in params["endpoint_mlp"]]
        self.device = device

    def grid_params(self):
        return self.color_grid + self.endpoint_grid

    def mlp_params(self):
        return [p for wb in self.color_mlp + self.endpoint_mlp for p in wb]

    # --- network pieces
    @staticmethod
    def lookup(levels, u, v, qat=None):
        feats = []
        for l, g in enumerate(levels):
            if qat is not None:
                g = qat[l](g)
            res = g.shape[0]
            px, py = u * (res - 1), v * (res - 1)
            ix = torch.clamp(torch.floor(px), max=res - 2).long()
            iy = torch.clamp(torch.floor(py), max=res - 2).long()
            fx, fy = (px - ix)[:, None], (py - iy)[:, None]
            f = ((1 - fx) * (1 - fy) * g[iy, ix] + fx * (1 - fy) * g[iy, ix + 1]
                 + (1 - fx) * fy * g[iy + 1, ix] + fx * fy * g[iy + 1, ix + 1])
            feats.append(f)
        return torch.cat(feats, dim=1)

    def mlp(self, layers, x):
        for i, (W, b) in enumerate(layers):
            x = torch.matmul(x, W.t()) + b
            if i + 1 < len(layers):
                x = torch.nn.functional.selu(x) if self.act == "selu" else torch.relu(x)
        return torch.sigmoid(x)

    def block_coords(self, ids):
        bx, by = (ids % self.bw).float(), (ids // self.bw).float()
        return (bx + 0.5) / self.bw, (by + 0.5) / self.bh

    def texel_xy(self, ids):
        i = torch.arange(16, device=ids.device)
        x = 4 * (ids % self.bw)[:, None] + (i % 4)[None]
        y = 4 * (ids // self.bw)[:, None] + (i // 4)[None]
        return x, y

    def forward(self, ids, grids=None):
        cg, eg = grids if grids is not None else (self.color_grid, self.endpoint_grid)
        s, t = self.block_coords(ids)
        e = self.mlp(self.endpoint_mlp, self.lookup(eg, s, t))
        x, y = self.texel_xy(ids)
        u = (x.reshape(-1).float() + 0.5) / self.w
        v = (y.reshape(-1).float() + 0.5) / self.h
        c = self.mlp(self.color_mlp, self.lookup(cg, u, v)).reshape(len(ids), 16, -1)
        return e, c


# ----------------------------------------------------------------------------
# inference to blocks (torch ops)
# ----------------------------------------------------------------------------

def _expand565(c):
    r5, g6, b5 = (c >> 11) & 31, (c >> 5) & 63, c & 31
    return torch.stack([(r5 << 3) | (r5 >> 2), (g6 << 2) | (g6 >> 4), (b5 << 3) | (b5 >> 2)], -1)


def reference_endpoints(fmt, blocks):
    """Decoded endpoints of stored blocks in [0, 1], stored order: BC1 [n, 6], BC4 [n, 2]
    (blocks: uint8 tensor [n, 8]); the L_e targets."""
    b = blocks.reshape(-1, 8).long()
    if fmt == BC1:
        c0 = b[:, 0] | (b[:, 1] << 8)
        c1 = b[:, 2] | (b[:, 3] << 8)
        return torch.cat([_expand565(c0), _expand565(c1)], 1).float() / 255.0
    return torch.stack([b[:, 0], b[:, 1]], 1).float() / 255.0


def _quant(e, levels):
    return torch.clamp(torch.floor(e * levels + 0.5), 0, levels).long()


def _pack(lo, hi):
    """lo, hi int64 words -> [n, 8] uint8 little-endian."""
    words = torch.stack([lo & 0xFFFFFFFF, hi & 0xFFFFFFFF], 1)
    shifts = torch.arange(0, 32, 8, device=lo.device)
    return ((words[:, :, None] >> shifts) & 255).reshape(-1, 8).to(torch.uint8)


def outputs_to_blocks(fmt, e, c):
    if fmt == BC1:
        def q565(x):
            return (_quant(x[:, 0], 31) << 11) | (_quant(x[:, 1], 63) << 5) | _quant(x[:, 2], 31)

        c0, c1 = q565(e[:, 0:3]), q565(e[:, 3:6])
        c0, c1 = torch.maximum(c0, c1), torch.minimum(c0, c1)
        e0, e1 = _expand565(c0), _expand565(c1)
        pal = torch.stack([e0, e1, (2 * e0 + e1 + 1) // 3, (e0 + 2 * e1 + 1) // 3], 1).float() / 255.0
        d = ((c[:, :, None, :] - pal[:, None]) ** 2)
        d = (d[..., 0] + d[..., 1]) + d[..., 2]
        codes = torch.argmin(d, -1)
        codes = torch.where((c0 == c1)[:, None], torch.zeros_like(codes), codes)
        idx = (codes << (2 * torch.arange(16, device=c.device))).sum(1)
        return _pack(c0 | (c1 << 16), idx)
    r0, r1 = _quant(e[:, 0], 255), _quant(e[:, 1], 255)
    k6 = torch.arange(1, 7, device=e.device)
    k4 = torch.arange(1, 5, device=e.device)
    v8 = ((7 - k6) * r0[:, None] + k6 * r1[:, None] + 3) // 7
    v6 = torch.cat([((5 - k4) * r0[:, None] + k4 * r1[:, None] + 2) // 5,
                    torch.zeros_like(r0)[:, None], torch.full_like(r0, 255)[:, None]], 1)
    inter = torch.where((r0 > r1)[:, None], v8, v6)
    pal = torch.cat([r0[:, None], r1[:, None], inter], 1).float() / 255.0
    codes = torch.argmin((c[:, :, 0:1] - pal[:, None]) ** 2, -1)
    idx = (codes << (3 * torch.arange(16, device=c.device))).sum(1)
    return _pack(r0 | (r1 << 8) | ((idx & 0xFFFF) << 16), idx >> 16)


@torch.no_grad()
def infer_to_bc(model: PlainModel, chunk_blocks=1 << 16, grids=None):
    n = model.bw * model.bh
    outs = [torch.empty(n, 8, dtype=torch.uint8, device=model.device) for _ in model.formats]
    for b0 in range(0, n, chunk_blocks):
        ids = torch.arange(b0, min(n, b0 + chunk_blocks), device=model.device)
        e, c = model.forward(ids, grids)
        for t, fmt in enumerate(model.formats):
            ch, co = model.ch[t], model.coff[t]
            outs[t][b0:b0 + len(ids)] = outputs_to_blocks(fmt, e[:, 2 * co:2 * co + 2 * ch], c[:, :, co:co + ch])
    return outs


# ----------------------------------------------------------------------------
# training step (autograd with straight-through estimators)
# ----------------------------------------------------------------------------

def _palette_linear(fmt, e0, e1):
    if fmt == BC1:
        w = torch.arange(4, device=e0.device, dtype=e0.dtype) / 3.0
        return (1 - w)[None, :, None] * e0[:, None] + w[None, :, None] * e1[:, None]
    n = torch.arange(8, device=e0.device, dtype=e0.dtype)
    w8 = n / 7.0
    p8 = (1 - w8)[None, :, None] * e0[:, None] + w8[None, :, None] * e1[:, None]
    w6 = torch.clamp((n - 1) / 5.0, 0, 1)
    p6 = (1 - w6)[None, :, None] * e0[:, None] + w6[None, :, None] * e1[:, None]
    p6 = torch.cat([torch.zeros_like(p6[:, :1]), p6[:, 1:7], torch.ones_like(p6[:, :1])], 1)
    return torch.where((e0[:, 0] > e1[:, 0])[:, None, None], p8, p6)


def _ste_decode(d, P, T):
    """hard decode P[argmax d] forward, softmax expectation backward."""
    sig = torch.softmax(d / T, -1)
    soft = (sig[..., None] * P).sum(-2)
    hard = torch.gather(P, -2, torch.argmax(d, -1)[..., None, None].expand(*d.shape[:-1], 1, P.shape[-1]))[..., 0, :]
    return hard + (soft - soft.detach())


def _qat_fn(bits):
    def q(g):
        a = torch.clamp(g.detach().min(), max=0.0)
        b = torch.clamp(g.detach().max(), min=0.0)
        s = (b - a) / (2 ** bits - 1)
        s = torch.where(s > 0, s, torch.ones_like(s))
        z = torch.round(-a / s)
        raw = torch.round(g / s) + z
        qv = s * (torch.clamp(raw, 0, 2 ** bits - 1) - z)
        mask = ((raw >= 0) & (raw <= 2 ** bits - 1)).float()
        return g * mask + (qv - g * mask).detach()
    return q


def losses(model: PlainModel, textures, ref_e, ids, T=0.01, qat_bits=0):
    """textures: list of uint8 device tensors [H, W(, 3)]; ref_e: list of [nblocks, 2C] float
    decoded reference endpoints. Returns (L_endpoint, L_color)."""
    qat = [_qat_fn(qat_bits)] * 64 if qat_bits else None
    s, t = model.block_coords(ids)
    e = model.mlp(model.endpoint_mlp, model.lookup(model.endpoint_grid, s, t, qat))
    x, y = model.texel_xy(ids)
    u = (x.reshape(-1).float() + 0.5) / model.w
    v = (y.reshape(-1).float() + 0.5) / model.h
    c_hat = model.mlp(model.color_mlp, model.lookup(model.color_grid, u, v, qat)).reshape(len(ids), 16, -1)
    nb = len(ids)
    n_cd = nb * 16 * c_hat.shape[-1]
    L_e = 0.0
    L_cd_e = 0.0
    L_c = 0.0
    L_cd_c = 0.0
    e_ref_all = []
    for k, fmt in enumerate(model.formats):
        ch, co = model.ch[k], model.coff[k]
        tex = textures[k]
        c = (tex[y, x].float() / 255.0).reshape(nb, 16, ch)
        er = ref_e[k][ids]
        e_ref_all.append(er)
        eh = e[:, 2 * co:2 * co + 2 * ch]
        Pr = _palette_linear(fmt, er[:, :ch], er[:, ch:])
        Ph = _palette_linear(fmt, eh[:, :ch], eh[:, ch:])
        d_e = -torch.linalg.norm(c[:, :, None, :] - Ph[:, None], dim=-1)
        dec_e = _ste_decode(d_e, Pr[:, None].expand(-1, 16, -1, -1), T)
        L_cd_e = L_cd_e + ((c - dec_e) ** 2).sum() / n_cd
        chat = c_hat[:, :, co:co + ch]
        d_c = -torch.linalg.norm(chat[:, :, None, :] - Pr[:, None], dim=-1)
        dec_c = _ste_decode(d_c, Pr[:, None].expand(-1, 16, -1, -1), T)
        L_cd_c = L_cd_c + ((c - dec_c) ** 2).sum() / n_cd
        L_c = L_c + ((chat - c) ** 2).sum()
    L_c = L_c / c_hat.numel()
    L_e = ((e - torch.cat(e_ref_all, 1)) ** 2).mean()
    return L_e + L_cd_e, L_c + L_cd_c


class PlainTrainer:
    def __init__(self, model: PlainModel, total_steps, lr_grid=0.01, lr_mlp=0.005, warmup=10):
        self.model = model
        self.opt = torch.optim.Adam([{"params": model.grid_params(), "lr": lr_grid},
                                     {"params": model.mlp_params(), "lr": lr_mlp}], betas=(0.9, 0.999), eps=1e-15)

        def sched(t):
            if t < warmup:
                return (t + 1) / warmup
            return 0.5 * (1 + math.cos(math.pi * (t - warmup) / max(total_steps - warmup, 1)))

        self.sched = torch.optim.lr_scheduler.LambdaLR(self.opt, sched)

    def step(self, textures, ref_e, ids, T=0.01, qat_bits=0):
        self.opt.zero_grad(set_to_none=True)
        le, lc = losses(self.model, textures, ref_e, ids, T, qat_bits)
        (le + lc).backward()
        self.opt.step()
        self.sched.step()
        return le.detach(), lc.detach()
