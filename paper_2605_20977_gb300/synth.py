"""Seeded synthetic inputs: latents, hyperlatents and model weights.

This module only draws random numbers and lays them out.  It computes none
of the context model's arithmetic, so both the CUDA library's tests and the
FP64 oracle can take their inputs from it.

Latents follow the stand-in for the paper's 1080p test material (Sec. 4.1 of
the paper evaluates on UVG, MCL-JCV and HEVC-B at 1920x1080, padded to
1088x1920, i.e. a 68x120 latent grid after the /16 feature transform): per
channel a separable 2D AR(1) Gaussian field with correlation ``rho`` in both
directions, scaled by a per-position sigma drawn log-uniformly from
[0.1, 8] and rounded.  P-frames mix the previous frame's field with a fresh
one (temporal AR(1), ``rho_t``).  Hyperlatents carry a coarse copy of the
local scale plus noise.  Weights are random with fan-in scaling.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, asdict, field

import numpy as np
from scipy.signal import lfilter


@dataclass(frozen=True)
class ModelConfig:
    """Sizes of one context model and one latent frame.

    H, W, C    latent grid and channels
    Hh, Wh, Ch hyperprior grid and channels, r = upsampling factor
    d, nh, F   model width, attention heads, SwiGLU hidden width
    L          blocks in each spatial module (plus one accumulator block)
    k          spatial window size (k x k)
    temporal   1: Context Transformer + temporal cross-attention (P-frames)
    Lc, Tf     Context Transformer blocks, frames in the temporal window
    mask       0: step label 2i+j; 1: cyclic s = 4 label
    Llrp       LRP Transformer blocks (0: none): the latent residual
               prediction over a decoded frame
    Nc, dc     Channel Transformer: channel groups (0: none) and width
    Lct, Fc    its blocks and the SwiGLU hidden width of each group
    hp         1: convolutional hyperprior (log2 r down / upsampling residual
               blocks, z-hat coded under a factorized prior); 0: z-hat given,
               embedded by a transposed convolution
    """
    H: int
    W: int
    C: int
    Hh: int
    Wh: int
    Ch: int
    r: int
    d: int
    nh: int
    F: int
    L: int
    k: int
    temporal: int = 0
    Lc: int = 0
    Tf: int = 3
    mask: int = 0
    Llrp: int = 0
    Nc: int = 0
    dc: int = 0
    Lct: int = 0
    Fc: int = 0
    hp: int = 0

    def with_grid(self, H: int, W: int) -> "ModelConfig":
        d = asdict(self)
        d.update(H=H, W=W, Hh=-(-H // self.r), Wh=-(-W // self.r))
        return ModelConfig(**d)

    def as_dict(self) -> dict:
        return asdict(self)


def ffn_width(d: int) -> int:
    """SwiGLU hidden width: 8d/3 rounded up to a multiple of 64."""
    return -(-(8 * d) // 192) * 64


def config(name: str) -> ModelConfig:
    """Named workloads.

    tiny      8x12x64 latent (128x192 image), hyperprior 4x6x32, d=128,
              2 blocks per spatial module, 4 heads, 5x5 window, FP32
    i1080     68x120x192 latent (1088x1920 image), hyperprior 17x30x128,
              d=384, 8 blocks per module, 6 heads, 7x7 window
    p1080     i1080 plus an 8-block Context Transformer and temporal
              cross-attention over the current and 2 previous frames
    tiny_p    tiny with the temporal path (2 context blocks)
    tiny_cyc  tiny with the cyclic s = 4 mask
    i1080_cyc i1080 with the cyclic s = 4 mask (4 steps per frame)
    tiny_lrp  tiny with a 2-block LRP Transformer
    i1080_lrp i1080 with a 4-block LRP Transformer
    tiny_p_lrp tiny_p with a 2-block time-causal LRP Transformer
    p1080_lrp p1080 with a 4-block time-causal LRP Transformer
    tiny_ct   tiny with a Channel Transformer: 4 groups, width 256, 2 blocks
    tiny_cyc_ct  tiny_ct with the cyclic s = 4 mask (16 steps per frame)
    tiny_p_ct tiny_p with the same Channel Transformer
    tiny_ct_lrp  tiny_ct with a 2-block LRP Transformer on its output
    tiny_hp, tiny_p_hp, i1080_hp, p1080_hp  the model with the convolutional
              hyperprior (z-hat produced by the analysis and coded)
    i1080_ct  i1080 with a Channel Transformer: 4 groups, width 1024, 2 blocks
    i1080_cyc_ct  i1080_ct with the cyclic s = 4 mask: s x N = 16 steps
    """
    if name == "tiny":
        return ModelConfig(H=8, W=12, C=64, Hh=4, Wh=6, Ch=32, r=2, d=128, nh=4,
                           F=ffn_width(128), L=2, k=5)
    if name == "tiny_p":
        return ModelConfig(H=8, W=12, C=64, Hh=4, Wh=6, Ch=32, r=2, d=128, nh=4,
                           F=ffn_width(128), L=2, k=5, temporal=1, Lc=2, Tf=3)
    if name == "tiny_cyc":
        return ModelConfig(H=8, W=12, C=64, Hh=4, Wh=6, Ch=32, r=2, d=128, nh=4,
                           F=ffn_width(128), L=2, k=5, mask=1)
    if name == "i1080":
        return ModelConfig(H=68, W=120, C=192, Hh=17, Wh=30, Ch=128, r=4, d=384, nh=6,
                           F=ffn_width(384), L=8, k=7)
    if name == "tiny_lrp":
        return ModelConfig(H=8, W=12, C=64, Hh=4, Wh=6, Ch=32, r=2, d=128, nh=4,
                           F=ffn_width(128), L=2, k=5, Llrp=2)
    if name == "i1080_lrp":
        return ModelConfig(H=68, W=120, C=192, Hh=17, Wh=30, Ch=128, r=4, d=384, nh=6,
                           F=ffn_width(384), L=8, k=7, Llrp=4)
    if name == "tiny_p_lrp":
        return ModelConfig(H=8, W=12, C=64, Hh=4, Wh=6, Ch=32, r=2, d=128, nh=4,
                           F=ffn_width(128), L=2, k=5, temporal=1, Lc=2, Tf=3, Llrp=2)
    if name == "p1080_lrp":
        return ModelConfig(H=68, W=120, C=192, Hh=17, Wh=30, Ch=128, r=4, d=384, nh=6,
                           F=ffn_width(384), L=8, k=7, temporal=1, Lc=8, Tf=3, Llrp=4)
    if name in ("tiny_ct", "tiny_cyc_ct", "tiny_p_ct"):
        base = config({"tiny_ct": "tiny", "tiny_cyc_ct": "tiny_cyc", "tiny_p_ct": "tiny_p"}[name])
        d = asdict(base)
        d.update(Nc=4, dc=256, Lct=2, Fc=ffn_width(64))
        return ModelConfig(**d)
    if name in ("tiny_hp", "tiny_p_hp", "i1080_hp", "p1080_hp"):
        d = asdict(config(name[:-3]))
        d.update(hp=1)
        return ModelConfig(**d)
    if name == "tiny_ct_lrp":
        d = asdict(config("tiny_ct"))
        d.update(Llrp=2)
        return ModelConfig(**d)
    if name in ("i1080_ct", "i1080_cyc_ct"):
        base = config({"i1080_ct": "i1080", "i1080_cyc_ct": "i1080_cyc"}[name])
        d = asdict(base)
        d.update(Nc=4, dc=1024, Lct=2, Fc=ffn_width(256))
        return ModelConfig(**d)
    if name == "i1080_cyc":
        return ModelConfig(H=68, W=120, C=192, Hh=17, Wh=30, Ch=128, r=4, d=384, nh=6,
                           F=ffn_width(384), L=8, k=7, mask=1)
    if name == "p1080":
        return ModelConfig(H=68, W=120, C=192, Hh=17, Wh=30, Ch=128, r=4, d=384, nh=6,
                           F=ffn_width(384), L=8, k=7, temporal=1, Lc=8, Tf=3)
    raise KeyError(name)


# --------------------------------------------------------------------------
# Weight packing order (the C-ABI documents the same order)
# --------------------------------------------------------------------------

@dataclass
class Tensor:
    name: str
    shape: tuple
    init: str          # gain | lin | lin_res | bias | relbias | normal | const
    value: float = 0.0
    fan_in: int = 1
    matrix: bool = False   # projection stored in the compute dtype


def _block(prefix: str, c: ModelConfig, cross: bool, tf_bias: bool, nblocks: int) -> list:
    d, F, kk = c.d, c.F, c.k * c.k
    res = 1.0 / math.sqrt(2.0 * nblocks)
    out = [Tensor(prefix + "g_attn", (d,), "gain")]
    for nm in ("Wq", "Wk", "Wv"):
        out.append(Tensor(prefix + nm, (d, d), "lin", fan_in=d, matrix=True))
    out.append(Tensor(prefix + "Wo", (d, d), "lin_res", value=res, fan_in=d, matrix=True))
    out.append(Tensor(prefix + "bias", (c.nh, c.Tf, c.k, c.k) if tf_bias else (c.nh, c.k, c.k), "relbias"))
    if cross:
        out.append(Tensor(prefix + "g_x", (d,), "gain"))
        for nm in ("Wxq", "Wxk", "Wxv"):
            out.append(Tensor(prefix + nm, (d, d), "lin", fan_in=d, matrix=True))
        out.append(Tensor(prefix + "Wxo", (d, d), "lin_res", value=res, fan_in=d, matrix=True))
        out.append(Tensor(prefix + "xbias", (c.nh, c.Tf, c.k, c.k), "relbias"))
    out.append(Tensor(prefix + "g_ffn", (d,), "gain"))
    out.append(Tensor(prefix + "Wg", (d, F), "lin", fan_in=d, matrix=True))
    out.append(Tensor(prefix + "Wu", (d, F), "lin", fan_in=d, matrix=True))
    out.append(Tensor(prefix + "Wd", (F, d), "lin_res", value=res, fan_in=F, matrix=True))
    return out


def weight_spec(c: ModelConfig) -> list:
    """Tensors of the flat FP32 weight vector, in packing order.

    All projections are [in][out] (used as x . W).  Order: input embedding,
    hyperprior embedding, [Context Transformer], Spatial Module 1 blocks,
    accumulator, Spatial Module 2 blocks, heads, [LRP Transformer: input
    projections of the representation and of the latents, blocks, output].
    """
    d, C, Ch, F = c.d, c.C, c.Ch, c.F
    nblocks = 2 * c.L + 1 + (c.Lc if c.temporal else 0)
    s = [Tensor("gamma_in", (C,), "const", 0.25),
         Tensor("W_in", (C, d), "lin", fan_in=C, matrix=True),
         Tensor("b_in", (d,), "bias"),
         Tensor("gamma_z", (Ch,), "const", 0.5)]
    if c.hp:
        # convolutional hyperprior: analysis RB-down blocks (d -> Ch, then
        # Ch -> Ch), synthesis RB-up blocks (Ch -> Ch, last Ch -> d), then the
        # factorized prior's per-channel parameters
        nb = int(round(math.log2(c.r)))
        s.append(Tensor("hp.g_za", (d,), "gain"))
        for b in range(nb):
            ci, co = (d if b == 0 else Ch), Ch
            s += [Tensor(f"hp.d{b}.Wa", (3, 3, ci, co), "lin", fan_in=9 * ci, matrix=True),
                  Tensor(f"hp.d{b}.ba", (co,), "bias"),
                  Tensor(f"hp.d{b}.Wb", (3, 3, co, co), "lin_res", value=0.5, fan_in=9 * co, matrix=True),
                  Tensor(f"hp.d{b}.bb", (co,), "bias"),
                  Tensor(f"hp.d{b}.Ws", (ci, co), "lin", fan_in=ci, matrix=True),
                  Tensor(f"hp.d{b}.bs", (co,), "bias")]
        for b in range(nb):
            ci, co = Ch, (d if b == nb - 1 else Ch)
            s += [Tensor(f"hp.u{b}.Wa", (3, 3, ci, 4 * co), "lin", fan_in=9 * ci, matrix=True),
                  Tensor(f"hp.u{b}.ba", (4 * co,), "bias"),
                  Tensor(f"hp.u{b}.Wb", (3, 3, co, co), "lin_res", value=0.5, fan_in=9 * co, matrix=True),
                  Tensor(f"hp.u{b}.bb", (co,), "bias"),
                  Tensor(f"hp.u{b}.Ws", (3, 3, ci, 4 * co), "lin", fan_in=9 * ci, matrix=True),
                  Tensor(f"hp.u{b}.bs", (4 * co,), "bias")]
        s += [Tensor("hp.fp_H1", (Ch, 3), "softplus_inv", 1.5), Tensor("hp.fp_b1", (Ch, 3), "bias"),
              Tensor("hp.fp_a1", (Ch, 3), "bias"),
              Tensor("hp.fp_H2", (Ch, 3, 3), "softplus_inv", 1.0 / 3.0), Tensor("hp.fp_b2", (Ch, 3), "bias"),
              Tensor("hp.fp_a2", (Ch, 3), "bias"),
              Tensor("hp.fp_H3", (Ch, 3, 3), "softplus_inv", 1.0 / 3.0), Tensor("hp.fp_b3", (Ch, 3), "bias"),
              Tensor("hp.fp_a3", (Ch, 3), "bias"),
              Tensor("hp.fp_H4", (Ch, 3), "softplus_inv", 0.2), Tensor("hp.fp_b4", (Ch,), "bias")]
    else:
        # one (Ch x d) projection per sub-pixel tap, stored in the compute
        # dtype where the tensor cores take it (Ch a multiple of 64)
        s += [Tensor("W_hp", (c.r * c.r, Ch, d), "lin", fan_in=Ch, matrix=Ch % 64 == 0),
              Tensor("b_hp", (d,), "bias")]
    if c.temporal:
        s += [Tensor("gamma_c", (C,), "const", 0.25),
              Tensor("W_c", (C, d), "lin", fan_in=C),
              Tensor("b_c", (d,), "bias"),
              Tensor("pad", (d,), "normal")]
        for l in range(c.Lc):
            s += _block(f"ctx{l}.", c, cross=False, tf_bias=True, nblocks=nblocks)
        s.append(Tensor("g_ctx", (d,), "gain"))
    for l in range(c.L):
        s += _block(f"sm1.{l}.", c, cross=bool(c.temporal), tf_bias=False, nblocks=nblocks)
    res = 1.0 / math.sqrt(2.0 * nblocks)
    s += [Tensor("acc.g_q", (d,), "gain"), Tensor("acc.g_kv", (d,), "gain"),
          Tensor("acc.Wq", (d, d), "lin", fan_in=d, matrix=True),
          Tensor("acc.Wk", (d, d), "lin", fan_in=d, matrix=True),
          Tensor("acc.Wv", (d, d), "lin", fan_in=d, matrix=True),
          Tensor("acc.Wo", (d, d), "lin_res", value=res, fan_in=d, matrix=True),
          Tensor("acc.bias", (c.nh, c.k, c.k), "relbias"),
          Tensor("acc.g_ffn", (d,), "gain"),
          Tensor("acc.Wg", (d, F), "lin", fan_in=d, matrix=True),
          Tensor("acc.Wu", (d, F), "lin", fan_in=d, matrix=True),
          Tensor("acc.Wd", (F, d), "lin_res", value=res, fan_in=F, matrix=True)]
    for l in range(c.L):
        s += _block(f"sm2.{l}.", c, cross=bool(c.temporal), tf_bias=False, nblocks=nblocks)
    if c.Nc:
        # Channel Transformer: input projection, the shifted latents' group
        # embeddings, Lct blocks of masked channel mixing and grouped SwiGLU
        G, dc = c.Nc, c.dc
        dg, Cg = dc // G, C // G
        cres = 1.0 / math.sqrt(2.0 * c.Lct)
        s += [Tensor("ct.g_in", (d,), "gain"),
              Tensor("ct.W_in", (d, dc), "lin", fan_in=d, matrix=True),
              Tensor("ct.b_in", (dc,), "bias"),
              Tensor("ct.gamma_y", (C,), "const", 0.25),
              Tensor("ct.E", (G - 1, Cg, dg), "lin", fan_in=Cg)]
        for l in range(c.Lct):
            s += [Tensor(f"ct{l}.g_mix", (dc,), "gain"),
                  Tensor(f"ct{l}.M", (dc, dc), "lin_res", value=cres, fan_in=dc, matrix=True),
                  Tensor(f"ct{l}.g_ffn", (dc,), "gain"),
                  Tensor(f"ct{l}.Wg", (G, dg, c.Fc), "lin", fan_in=dg, matrix=True),
                  Tensor(f"ct{l}.Wu", (G, dg, c.Fc), "lin", fan_in=dg, matrix=True),
                  Tensor(f"ct{l}.Wd", (G, c.Fc, dg), "lin_res", value=cres, fan_in=c.Fc, matrix=True)]
        # grouped heads
        s += [Tensor("g_head", (dc,), "gain"),
              Tensor("W1m", (G, dg, dg), "lin", fan_in=dg, matrix=True), Tensor("b1m", (dc,), "bias"),
              Tensor("W2m", (G, dg, Cg), "lin", fan_in=dg, matrix=True),
              Tensor("W1s", (G, dg, dg), "lin", fan_in=dg, matrix=True), Tensor("b1s", (dc,), "bias"),
              Tensor("W2s", (G, dg, Cg), "lin", fan_in=dg, matrix=True)]
    else:
        s += [Tensor("g_head", (d,), "gain"),
              Tensor("W1m", (d, d), "lin", fan_in=d, matrix=True), Tensor("b1m", (d,), "bias"),
              Tensor("W2m", (d, C), "lin", fan_in=d, matrix=True),
              Tensor("W1s", (d, d), "lin", fan_in=d, matrix=True), Tensor("b1s", (d,), "bias"),
              Tensor("W2s", (d, C), "lin", fan_in=d, matrix=True)]
    s += [Tensor("gamma_mu", (C,), "const", 2.0), Tensor("beta_mu", (C,), "const", 0.0),
          Tensor("gamma_sig", (C,), "const", 1.0), Tensor("beta_sig", (C,), "const", math.log(2.0))]
    if c.Llrp:
        dh = c.dc if c.Nc else d            # the heads' input width
        s += [Tensor("lrp.g_rep", (dh,), "gain"),
              Tensor("lrp.W_rep", (dh, d), "lin", fan_in=dh, matrix=True),
              Tensor("lrp.gamma_y", (C,), "const", 0.25),
              Tensor("lrp.W_y", (C, d), "lin", fan_in=C, matrix=True),
              Tensor("lrp.b_in", (d,), "bias")]
        for l in range(c.Llrp):
            s += _block(f"lrp{l}.", c, cross=False, tf_bias=bool(c.temporal), nblocks=c.Llrp)
        s += [Tensor("lrp.g_out", (d,), "gain"),
              Tensor("lrp.W_eps", (d, C), "lin_res", value=0.1, fan_in=d, matrix=True),
              Tensor("lrp.b_eps", (C,), "bias")]
    return s


def weights_count(c: ModelConfig) -> int:
    return int(sum(int(np.prod(t.shape)) for t in weight_spec(c)))


def weights(c: ModelConfig, seed: int = 42, vary_consts: bool = False) -> np.ndarray:
    """Flat FP32 weight vector in packing order (seeded PCG64).

    The channel-wise scales and offsets ("const" tensors) hold their value
    in every channel; with vary_consts each channel draws its own around it
    (value (1 + 0.2 n) + 0.05 n' from a second generator), so a wrong channel
    index or a dropped offset changes results.  The other tensors are the
    same either way."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rng_c = np.random.Generator(np.random.PCG64(seed + 1))
    parts = []
    for t in weight_spec(c):
        n = int(np.prod(t.shape))
        if t.init == "const":
            a = np.full(n, t.value, dtype=np.float64)
            if vary_consts:
                a = a * (1.0 + 0.2 * rng_c.standard_normal(n)) + 0.05 * rng_c.standard_normal(n)
        elif t.init == "gain":
            a = 1.0 + 0.1 * rng.standard_normal(n)
        elif t.init == "lin":
            a = rng.standard_normal(n) / math.sqrt(t.fan_in)
        elif t.init == "lin_res":
            a = rng.standard_normal(n) / math.sqrt(t.fan_in) * t.value
        elif t.init == "bias":
            a = 0.05 * rng.standard_normal(n)
        elif t.init == "relbias":
            a = 0.5 * rng.standard_normal(n)
        elif t.init == "normal":
            a = rng.standard_normal(n)
        elif t.init == "softplus_inv":
            # raw parameter whose softplus is about `value` (positive entries)
            a = math.log(math.expm1(t.value)) + 0.1 * rng.standard_normal(n)
        else:
            raise ValueError(t.init)
        parts.append(a.astype(np.float32))
    return np.concatenate(parts)


def matrix_mask(c: ModelConfig) -> np.ndarray:
    """Boolean mask over the flat weight vector: True for the projections a
    reduced-precision run stores in its compute dtype (block projections,
    the latent embedding and the prediction heads)."""
    out = []
    for t in weight_spec(c):
        out.append(np.full(int(np.prod(t.shape)), t.matrix, dtype=bool))
    return np.concatenate(out)


def e4m3_tensor(t: Tensor) -> bool:
    """Whether an FP8 context stores projection t as E4M3 (one power-of-two
    scale per tensor): transformer-block projections whose input width K is
    a multiple of 128, at most 512 for a normalised input and 1024 for the
    compact-row inputs of Wo, Wxo and Wd.  The latent embedding, the heads,
    the Channel Transformer and the LRP Transformer stay in the compute
    dtype."""
    if (not t.matrix or t.name in ("W_in", "W1m", "W2m", "W1s", "W2s") or t.name.startswith("lrp")
            or t.name.startswith("ct") or t.name.startswith("hp.")):
        return False
    K = t.shape[0]
    return K % 128 == 0 and K <= (1024 if t.name.split(".")[-1] in ("Wo", "Wxo", "Wd") else 512)


def e4m3_ranges(c: ModelConfig) -> list:
    """(offset, size) in the flat weight vector of each E4M3-stored tensor."""
    out, off = [], 0
    for t in weight_spec(c):
        n = int(np.prod(t.shape))
        if e4m3_tensor(t):
            out.append((off, n))
        off += n
    return out


# --------------------------------------------------------------------------
# Latents and hyperlatents
# --------------------------------------------------------------------------

def _ar1_axis(e: np.ndarray, rho: float, axis: int) -> np.ndarray:
    """Stationary unit-variance AR(1) filter along one axis: y0 = e0,
    y_n = rho y_{n-1} + sqrt(1 - rho^2) e_n."""
    s = math.sqrt(1.0 - rho * rho)
    e = np.moveaxis(e, axis, 0).copy()
    e[0] /= s
    y = lfilter([s], [1.0, -rho], e, axis=0)
    return np.moveaxis(y, 0, axis)


def ar1_field(rng: np.random.Generator, H: int, W: int, C: int, rho: float) -> np.ndarray:
    """Separable 2D AR(1) field, unit variance, corr rho^(|di|+|dj|)."""
    e = rng.standard_normal((H, W, C))
    return _ar1_axis(_ar1_axis(e, rho, 1), rho, 0)


@dataclass
class Frames:
    y: np.ndarray        # int16 [nf][H][W][C]
    z: np.ndarray        # int16 [nf][Hh][Wh][Ch]
    sigma: np.ndarray    # float64 [H][W]  per-position scale of the latents


def frames(c: ModelConfig, nf: int = 1, seed: int = 1000, rho: float = 0.8,
           rho_t: float = 0.9, sigma_lo: float = 0.1, sigma_hi: float = 8.0) -> Frames:
    """nf frames of one sequence: AR(1) latents scaled by a static
    log-uniform per-position sigma, and their hyperlatents."""
    rng = np.random.Generator(np.random.PCG64(seed))
    H, W, C = c.H, c.W, c.C
    sig = np.exp(rng.uniform(math.log(sigma_lo), math.log(sigma_hi), size=(H, W)))
    x = ar1_field(rng, H, W, C, rho)
    ys, zs = [], []
    for f in range(nf):
        if f > 0:
            x = rho_t * x + math.sqrt(1.0 - rho_t * rho_t) * ar1_field(rng, H, W, C, rho)
        y = np.clip(np.rint(sig[:, :, None] * x), -32767, 32767).astype(np.int16)
        ys.append(y)
        zs.append(_hyper(rng, c, sig))
    return Frames(y=np.stack(ys), z=np.stack(zs), sigma=sig)


def _hyper(rng: np.random.Generator, c: ModelConfig, sig: np.ndarray) -> np.ndarray:
    """Hyperlatents: the first half of the channels carry 2 log2 of the mean
    sigma of the r x r block they cover, plus unit noise; the rest is noise
    with standard deviation 2."""
    z = np.zeros((c.Hh, c.Wh, c.Ch), dtype=np.float64)
    for a in range(c.Hh):
        for b in range(c.Wh):
            blk = sig[a * c.r:(a + 1) * c.r, b * c.r:(b + 1) * c.r]
            z[a, b, :c.Ch // 2] = np.rint(2.0 * math.log2(float(blk.mean())))
    z[:, :, :c.Ch // 2] += np.rint(rng.standard_normal((c.Hh, c.Wh, c.Ch // 2)))
    z[:, :, c.Ch // 2:] = np.rint(2.0 * rng.standard_normal((c.Hh, c.Wh, c.Ch - c.Ch // 2)))
    return z.astype(np.int16)
