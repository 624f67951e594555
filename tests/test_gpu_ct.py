"""GPU parity of the Channel Transformer (Sec. 3.1 Channel Transformer
paragraph; Sec. 3.2: s spatial steps times N channel groups; Sec. 4.1:
N = 4 groups, 2 blocks, width 1024) against the FP64 oracle.

The decoder runs N channel-group sub-steps after each spatial step (the
group's parameters, then its symbols); the encoder's masked pass runs the
same per-group launches over every position, so encoder and decoder give
bit-identical parameters, and the containers equal the oracle coder's given
the GPU's parameters.  The paper's own configuration is the cyclic s = 4
mask with N = 4 groups: 16 autoregressive steps per frame.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import dev, need_gpu, oracle_weights, param_errors, torch
from paper_2605_20977_gb300 import psw, synth

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4
BF16_TOL = 5e-2
FP8_TOL = 1.5e-1
MAX_FACTOR = 10.0
RATE_TOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    need_gpu()
    from paper_2605_20977_gb300 import build
    build.build()
    O.build()
    torch.cuda.set_device(0)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def _code(ctx, fr, sched=psw.PSW_SCHED_WAVEFRONT, lrp=False):
    H, W, C = fr.y.shape[1], fr.y.shape[2], fr.y.shape[3]
    enc, dec = ctx.seq_create(H, W), ctx.seq_create(H, W)
    fd = psw.frame_desc(H, W, sched)
    out = []
    for f in range(fr.y.shape[0]):
        y, z = _t(fr.y[f]), _t(fr.z[f])
        mu = torch.zeros(y.shape, dtype=torch.float32, device=dev()); sg = torch.zeros_like(mu)
        bs = torch.zeros(ctx.bitstream_capacity(H, W), dtype=torch.uint8, device=dev())
        n = enc.encode_params(fd, y, z, mu, sg, bs)
        y2 = torch.full_like(y, 12345)
        mu2 = torch.zeros_like(mu); sg2 = torch.zeros_like(mu)
        dec.decode_frame(fd, bs, n, z, y2, mu2, sg2)
        r = dict(mu=mu.cpu().numpy(), sg=sg.cpu().numpy(), bs=bs[:n].cpu().numpy().tobytes(),
                 y=y2.cpu().numpy(), mu2=mu2.cpu().numpy(), sg2=sg2.cpu().numpy())
        if lrp:
            e1 = torch.zeros((H, W, C), dtype=torch.float32, device=dev()); e2 = torch.zeros_like(e1)
            enc.lrp_residual(fd, e1)
            dec.lrp_residual(fd, e2)
            r.update(eps=e1.cpu().numpy(), eps2=e2.cpu().numpy())
        torch.cuda.synchronize()
        out.append(r)
    enc.close(); dec.close()
    return out


def _check(res, fr, cfg, mu_o, sg_o, tol, sched, pct=True):
    for f, r in enumerate(res):
        assert np.array_equal(r["y"], fr.y[f])
        assert np.array_equal(r["mu"], r["mu2"]) and np.array_equal(r["sg"], r["sg2"])
        dmu, dls = param_errors(r["mu"], r["sg"], mu_o[f], sg_o[f])
        if pct:
            q = (np.quantile(dmu, 0.999), np.quantile(dls, 0.999))
            print(f"frame {f}: observed (99.9th pct, max) |dmu|/sigma {q[0]:.3g}, {dmu.max():.3g}; "
                  f"|d ln sigma| {q[1]:.3g}, {dls.max():.3g}")
            assert q[0] <= tol and q[1] <= tol, q
            assert dmu.max() <= MAX_FACTOR * tol and dls.max() <= MAX_FACTOR * tol
        else:
            print(f"frame {f}: max |dmu|/sigma {dmu.max():.3g}, |d ln sigma| {dls.max():.3g}")
            assert dmu.max() <= tol and dls.max() <= tol
        ra = O.rate_bits(fr.y[f], r["mu"].astype(np.float64), r["sg"].astype(np.float64))
        rb = O.rate_bits(fr.y[f], mu_o[f], sg_o[f])
        assert abs(ra - rb) <= RATE_TOL * rb
        idx, m = O.quantize(r["mu"], r["sg"])
        assert r["bs"] == O.rans_encode(cfg, sched, fr.y[f], idx, m)


@pytest.mark.parametrize("name,sched", [("tiny_ct", 0), ("tiny_ct", 1), ("tiny_cyc_ct", 0), ("tiny_p_ct", 0)])
def test_ct_fp32_vs_oracle(name, sched):
    """FP32: every parameter within 1e-4 of the oracle; lossless; encoder ==
    decoder; the container equals the oracle coder's (2i+j, raster and
    cyclic schedules; P-frames over three frames)."""
    cfg = synth.config(name)
    w = synth.weights(cfg)
    fr = synth.frames(cfg, 3 if cfg.temporal else 1, seed=2201)
    ctx = psw.Context(cfg, w, precision=psw.PSW_FP32)
    res = _code(ctx, fr, sched)
    mu_o, sg_o = O.run(cfg, np.asarray(w, np.float64), fr.y, fr.z, driver=0)
    _check(res, fr, cfg, mu_o, sg_o, FP32_TOL, sched, pct=False)


def test_ct_per_channel_constants_fp32():
    """The cyclic Channel Transformer model with every channel-wise scale and
    offset different per channel (the shifted latents' scales of each group,
    the grouped heads' output scales and offsets)."""
    cfg = synth.config("tiny_cyc_ct")
    w = synth.weights(cfg, vary_consts=True)
    fr = synth.frames(cfg, 1, seed=2203)
    ctx = psw.Context(cfg, w, precision=psw.PSW_FP32)
    res = _code(ctx, fr, 0)
    mu_o, sg_o = O.run(cfg, np.asarray(w, np.float64), fr.y, fr.z, driver=0)
    _check(res, fr, cfg, mu_o, sg_o, FP32_TOL, 0, pct=False)


@pytest.mark.parametrize("name,rows,precision,vary", [("i1080_ct", 8, psw.PSW_BF16, False),
                                                      ("i1080_cyc_ct", 8, psw.PSW_BF16, False),
                                                      ("i1080_cyc_ct", 8, psw.PSW_FP8, False),
                                                      ("i1080_cyc_ct", 8, psw.PSW_BF16, True)])
def test_ct_1080p_width_vs_oracle(name, rows, precision, vary):
    """The 1080p model sizes with the Channel Transformer (4 groups, width
    1024, 2 blocks) on a rows x 120 grid coded as its own frame by both
    sides: BF16, and an FP8 context (E4M3 entropy-model blocks; the Channel
    Transformer stays BF16); vary: every channel-wise scale and offset
    differs per channel (the grouped heads' epilogues on the tensor cores)."""
    base = synth.config(name)
    w = synth.weights(base, vary_consts=vary)
    cfg = base.with_grid(rows, base.W)
    fr = synth.frames(cfg, 1, seed=2202)
    ctx = psw.Context(base, w, precision=precision)
    res = _code(ctx, fr)
    mu_o, sg_o = O.run(cfg, oracle_weights(base, w, precision), fr.y, fr.z, driver=0)
    _check(res, fr, cfg, mu_o, sg_o, BF16_TOL if precision == psw.PSW_BF16 else FP8_TOL, 0)


def test_ct_full_frame_16_steps_and_batch():
    """The paper's configuration on the full 68 x 120 frame: cyclic s = 4
    mask and 4 channel groups (16 autoregressive steps), BF16: lossless,
    encoder == decoder, and two frames decoded in one batch equal each
    decoded alone."""
    cfg = synth.config("i1080_cyc_ct")
    w = synth.weights(cfg)
    ctx = psw.Context(cfg, w, precision=psw.PSW_BF16)
    H, W, C = cfg.H, cfg.W, cfg.C
    fd = psw.frame_desc(H, W, 0)
    items = []
    for k in range(2):
        fr = synth.frames(cfg, 1, seed=2203 + k)
        enc = ctx.seq_create(H, W)
        bs = torch.zeros(ctx.bitstream_capacity(H, W), dtype=torch.uint8, device=dev())
        mu = torch.zeros((H, W, C), dtype=torch.float32, device=dev())
        z = _t(fr.z[0])
        n = enc.encode_params(fd, _t(fr.y[0]), z, mu, None, bs)
        items.append((bs, n, z, fr.y[0], mu.cpu().numpy()))
        enc.close()
    alone = []
    for bs, n, z, y, mu_enc in items:
        dec = ctx.seq_create(H, W)
        y2 = torch.zeros((H, W, C), dtype=torch.int16, device=dev())
        mu2 = torch.zeros((H, W, C), dtype=torch.float32, device=dev())
        dec.decode_frame(fd, bs, n, z, y2, mu2)
        assert np.array_equal(y2.cpu().numpy(), y)
        assert np.array_equal(mu2.cpu().numpy(), mu_enc)
        alone.append(mu2.cpu().numpy())
        dec.close()
    seqs = [ctx.seq_create(H, W) for _ in items]
    outs = [torch.zeros((H, W, C), dtype=torch.int16, device=dev()) for _ in items]
    mus = [torch.zeros((H, W, C), dtype=torch.float32, device=dev()) for _ in items]
    st = ctx.decode_batch(seqs, [fd, fd], [it[0] for it in items], [it[1] for it in items],
                          [it[2] for it in items], outs, mus)
    assert st == [psw.PSW_OK, psw.PSW_OK]
    for k in range(2):
        assert np.array_equal(outs[k].cpu().numpy(), items[k][3])
        assert np.array_equal(mus[k].cpu().numpy(), alone[k])
    for q in seqs:
        q.close()
    with pytest.raises(psw.PswError):
        ctx.set_engine(psw.ENGINE_PERSISTENT)


def test_ct_lrp_on_the_channel_transformer_output():
    """The LRP Transformer of a model with a Channel Transformer reads the
    Channel Transformer's stream (FP32): eps against the oracle, decoder's
    eps == encoder's."""
    cfg = synth.config("tiny_ct_lrp")
    w = synth.weights(cfg)
    fr = synth.frames(cfg, 1, seed=2205)
    ctx = psw.Context(cfg, w, precision=psw.PSW_FP32)
    r = _code(ctx, fr, lrp=True)[0]
    _, _, eps_o = O.run(cfg, np.asarray(w, np.float64), fr.y, fr.z, driver=0, with_eps=True)
    assert np.array_equal(r["eps"], r["eps2"])
    err = np.abs(r["eps"] - eps_o[0]) / np.sqrt(np.mean(eps_o[0] ** 2))
    print(f"max |d eps|/rms {err.max():.3g}")
    assert err.max() <= FP32_TOL
