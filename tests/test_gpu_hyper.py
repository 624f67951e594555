"""GPU parity of the convolutional hyperprior (Fig. 1 right): the analysis
(Spatial Module 1 output through the downsampling residual blocks to z and
z-hat), the z-hat coder under the factorized prior, and the synthesis of the
hyperprior tokens (upsampling residual blocks) that the encoder's and the
decoder's passes start from.

z is a smooth function of the latents and is compared with a tolerance;
z-hat = round(z) is an integer decided in floating point, so it must equal
the oracle's wherever the oracle's z is not within the tolerance of a
rounding boundary, and elsewhere may differ by one.  Everything downstream
is compared given the GPU's z-hat (the exact input): the factorized-prior
tables and the z-hat containers bit for bit, (mu, sigma) within the
tolerance of the precision, decoding lossless and equal to the encoder.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import dev, need_gpu, oracle_weights, param_errors, torch
from paper_2605_20977_gb300 import psw, synth

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4
BF16_TOL = 5e-2
MAX_FACTOR = 10.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    need_gpu()
    from paper_2605_20977_gb300 import build
    build.build()
    O.build()
    torch.cuda.set_device(0)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def _zhat_agrees(zh, zh_o, z_o, band):
    """z-hat equal to the oracle's away from rounding boundaries (the
    oracle's z more than `band` from k + 1/2), within one elsewhere."""
    near = np.abs(np.abs(z_o - np.floor(z_o)) - 0.5) <= band
    diff = zh.astype(np.int32) - zh_o.astype(np.int32)
    assert np.all(np.abs(diff) <= 1)
    assert np.array_equal(zh[~near], zh_o[~near])
    return float(np.mean(diff != 0))


def _run(ctx, cfg, fr):
    """Per frame: z-hat and z on the GPU with its container, the latent
    container from psw_encode_params with that z-hat; then decode both
    containers with fresh sequences."""
    H, W, C = fr.y.shape[1], fr.y.shape[2], fr.y.shape[3]
    enc, dec = ctx.seq_create(H, W), ctx.seq_create(H, W)
    fd = psw.frame_desc(H, W, 0)
    Hh, Wh = -(-H // cfg.r), -(-W // cfg.r)
    res = []
    for f in range(fr.y.shape[0]):
        y = _t(fr.y[f])
        zh = torch.zeros((Hh, Wh, cfg.Ch), dtype=torch.int16, device=dev())
        z = torch.zeros((Hh, Wh, cfg.Ch), dtype=torch.float32, device=dev())
        bz = torch.zeros(ctx.bitstream_capacity(Hh, Wh) + 16 * cfg.Ch, dtype=torch.uint8, device=dev())
        nz = enc.hyper_encode(fd, y, zh, z, bz)
        mu = torch.zeros((H, W, C), dtype=torch.float32, device=dev()); sg = torch.zeros_like(mu)
        by = torch.zeros(ctx.bitstream_capacity(H, W), dtype=torch.uint8, device=dev())
        ny = enc.encode_params(fd, y, zh, mu, sg, by)
        zh2 = torch.full_like(zh, 777)
        ctx.hyper_decode(fd, bz, nz, zh2)
        y2 = torch.full_like(y, 12345)
        mu2 = torch.zeros_like(mu); sg2 = torch.zeros_like(mu)
        dec.decode_frame(fd, by, ny, zh2, y2, mu2, sg2)
        torch.cuda.synchronize()
        res.append(dict(zh=zh.cpu().numpy(), z=z.cpu().numpy(), bz=bz[:nz].cpu().numpy().tobytes(),
                        zh2=zh2.cpu().numpy(), mu=mu.cpu().numpy(), sg=sg.cpu().numpy(), y=y2.cpu().numpy(),
                        mu2=mu2.cpu().numpy(), sg2=sg2.cpu().numpy()))
    enc.close(); dec.close()
    return res


@pytest.mark.parametrize("name", ["tiny_hp", "i1080_hp"])
def test_prior_tables_byte_identical(name):
    cfg = synth.config(name)
    w = synth.weights(cfg)
    ctx = psw.Context(cfg, w, precision=psw.PSW_FP32 if name.startswith("tiny") else psw.PSW_BF16)
    for ch in range(cfg.Ch):
        assert np.array_equal(ctx.prior_table(ch), O.prior_freq(cfg, w, ch)), ch


@pytest.mark.parametrize("name,nf,vary", [("tiny_hp", 1, False), ("tiny_p_hp", 3, False), ("tiny_p_hp", 2, True)])
def test_hyperprior_fp32_vs_oracle(name, nf, vary):
    """vary: every channel-wise scale and offset differs per channel (the
    z-hat scale of the synthesis among them)."""
    cfg = synth.config(name)
    w = synth.weights(cfg, vary_consts=vary)
    fr = synth.frames(cfg, nf, seed=2301)
    ctx = psw.Context(cfg, w, precision=psw.PSW_FP32)
    res = _run(ctx, cfg, fr)
    w64 = np.asarray(w, np.float64)
    zh_o, z_o = O.hyper_analysis(cfg, w64, fr.y)
    zhs = np.stack([r["zh"] for r in res])
    scale = np.sqrt(np.mean(z_o ** 2))
    dz = np.abs(np.stack([r["z"] for r in res]) - z_o).max() / scale
    frac = _zhat_agrees(zhs, zh_o, z_o, 1e-3)
    print(f"max |dz|/rms(z) {dz:.3g}; z-hat differing {frac:.3g}")
    assert dz <= FP32_TOL
    mu_o, sg_o = O.run(cfg, w64, fr.y, zhs, driver=0)
    for f, r in enumerate(res):
        assert r["bz"] == O.hyper_encode(cfg, w64, r["zh"])
        assert np.array_equal(r["zh2"], r["zh"])
        assert np.array_equal(r["y"], fr.y[f])
        assert np.array_equal(r["mu"], r["mu2"]) and np.array_equal(r["sg"], r["sg2"])
        dmu, dls = param_errors(r["mu"], r["sg"], mu_o[f], sg_o[f])
        assert dmu.max() <= FP32_TOL and dls.max() <= FP32_TOL, (dmu.max(), dls.max())


@pytest.mark.parametrize("name,rows,nf", [("i1080_hp", 8, 1), ("p1080_hp", 4, 2)])
def test_hyperprior_bf16_1080p_width_vs_oracle(name, rows, nf):
    """BF16 at the 1080p sizes (two residual blocks each way, Ch = 128) on a
    rows x 120 grid coded as its own frame by both sides; P-frames over two
    frames."""
    base = synth.config(name)
    w = synth.weights(base)
    cfg = base.with_grid(rows, base.W)
    fr = synth.frames(cfg, nf, seed=2302)
    ctx = psw.Context(base, w, precision=psw.PSW_BF16)
    res = _run(ctx, cfg, fr)
    w64 = oracle_weights(base, w, psw.PSW_BF16)
    zh_o, z_o = O.hyper_analysis(cfg, w64, fr.y)
    zs = np.stack([r["z"] for r in res])
    err = np.abs(zs - z_o) / np.sqrt(np.mean(z_o ** 2))
    q = np.quantile(err, 0.999)
    zhs = np.stack([r["zh"] for r in res])
    frac = _zhat_agrees(zhs, zh_o, z_o, MAX_FACTOR * BF16_TOL * np.sqrt(np.mean(z_o ** 2)))
    print(f"observed |dz|/rms(z) (99.9th pct, max): {q:.3g}, {err.max():.3g}; z-hat differing {frac:.3g}")
    assert q <= BF16_TOL and err.max() <= MAX_FACTOR * BF16_TOL
    mu_o, sg_o = O.run(cfg, w64, fr.y, zhs, driver=0)
    for f, r in enumerate(res):
        assert r["bz"] == O.hyper_encode(cfg, w64, r["zh"])
        assert np.array_equal(r["zh2"], r["zh"])
        assert np.array_equal(r["y"], fr.y[f])
        assert np.array_equal(r["mu"], r["mu2"]) and np.array_equal(r["sg"], r["sg2"])
        dmu, dls = param_errors(r["mu"], r["sg"], mu_o[f], sg_o[f])
        qm = (np.quantile(dmu, 0.999), np.quantile(dls, 0.999))
        print(f"frame {f}: observed (99.9th pct, max) |dmu|/sigma {qm[0]:.3g}, {dmu.max():.3g}; "
              f"|d ln sigma| {qm[1]:.3g}, {dls.max():.3g}")
        assert qm[0] <= BF16_TOL and qm[1] <= BF16_TOL
        assert dmu.max() <= MAX_FACTOR * BF16_TOL and dls.max() <= MAX_FACTOR * BF16_TOL


def test_hyperprior_full_frame_batch_and_corruption():
    """The 68 x 120 frame, BF16: both containers round trip; two frames
    decoded in one batch (each synthesising its own hyperprior tokens in the
    prologue) equal each decoded alone; a corrupt z-hat container is
    reported and the context stays usable."""
    cfg = synth.config("i1080_hp")
    w = synth.weights(cfg)
    ctx = psw.Context(cfg, w, precision=psw.PSW_BF16)
    H, W, C = cfg.H, cfg.W, cfg.C
    fd = psw.frame_desc(H, W, 0)
    items = []
    for k in range(2):
        fr = synth.frames(cfg, 1, seed=2303 + k)
        enc = ctx.seq_create(H, W)
        y = _t(fr.y[0])
        zh = torch.zeros((cfg.Hh, cfg.Wh, cfg.Ch), dtype=torch.int16, device=dev())
        bz = torch.zeros(ctx.bitstream_capacity(cfg.Hh, cfg.Wh) + 16 * cfg.Ch, dtype=torch.uint8, device=dev())
        nz = enc.hyper_encode(fd, y, zh, None, bz)
        by = torch.zeros(ctx.bitstream_capacity(H, W), dtype=torch.uint8, device=dev())
        ny = enc.encode_params(fd, y, zh, None, None, by)
        items.append((bz, nz, by, ny, fr.y[0]))
        enc.close()
    alone = []
    for bz, nz, by, ny, y in items:
        zh = torch.zeros((cfg.Hh, cfg.Wh, cfg.Ch), dtype=torch.int16, device=dev())
        ctx.hyper_decode(fd, bz, nz, zh)
        dec = ctx.seq_create(H, W)
        y2 = torch.zeros((H, W, C), dtype=torch.int16, device=dev())
        mu2 = torch.zeros((H, W, C), dtype=torch.float32, device=dev())
        dec.decode_frame(fd, by, ny, zh, y2, mu2)
        assert np.array_equal(y2.cpu().numpy(), y)
        alone.append((zh, mu2.cpu().numpy()))
        dec.close()
    seqs = [ctx.seq_create(H, W) for _ in items]
    outs = [torch.zeros((H, W, C), dtype=torch.int16, device=dev()) for _ in items]
    mus = [torch.zeros((H, W, C), dtype=torch.float32, device=dev()) for _ in items]
    st = ctx.decode_batch(seqs, [fd, fd], [it[2] for it in items], [it[3] for it in items],
                          [a[0] for a in alone], outs, mus)
    assert st == [psw.PSW_OK, psw.PSW_OK]
    for k in range(2):
        assert np.array_equal(outs[k].cpu().numpy(), items[k][4])
        assert np.array_equal(mus[k].cpu().numpy(), alone[k][1])
    for q in seqs:
        q.close()
    bad = items[0][0].clone()
    bad[items[0][1] - 4:items[0][1]] = 0
    zh = torch.zeros((cfg.Hh, cfg.Wh, cfg.Ch), dtype=torch.int16, device=dev())
    st = ctx.hyper_decode(fd, bad, items[0][1] - 6, zh, check=False)
    assert st == psw.PSW_ERR_CORRUPT
    ctx.hyper_decode(fd, items[0][0], items[0][1], zh)
    assert torch.equal(zh, alone[0][0])
