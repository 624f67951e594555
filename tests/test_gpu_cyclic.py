"""The paper's own schedule at the 1080p model sizes: the cyclic s = 4 mask
(Fig. 2a; label ((i mod 4) + (j mod 4)) mod 4, 4 steps per frame at any
resolution, Sec. 3.2), k = 7.  Under this mask a position also sees window
positions below it whose label is smaller, so a crop is compared with the
oracle on the same cropped frame; self-attention lists up to 37 keys, so
the window attention's online softmax runs over two key chunks.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import dev, need_gpu, oracle_weights, param_errors, torch
from paper_2605_20977_gb300 import psw, synth

pytestmark = pytest.mark.gpu

TOLS = {psw.PSW_BF16: 5e-2, psw.PSW_FP8: 1.5e-1}    # 99.9th percentile of |dmu|/sigma and |d ln sigma|
MAX_FACTOR = 10.0                                    # the maximum within 10x that
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


def _encode_decode(ctx, fr):
    H, W = fr.y.shape[1], fr.y.shape[2]
    enc, dec = ctx.seq_create(H, W), ctx.seq_create(H, W)
    fd = psw.frame_desc(H, W, psw.PSW_SCHED_WAVEFRONT)
    y, z = _t(fr.y[0]), _t(fr.z[0])
    mu = torch.zeros(y.shape, dtype=torch.float32, device=dev()); sg = torch.zeros_like(mu)
    bs = torch.zeros(ctx.bitstream_capacity(H, W), dtype=torch.uint8, device=dev())
    n = enc.encode_params(fd, y, z, mu, sg, bs)
    y2 = torch.full_like(y, 12345)
    mu2 = torch.zeros_like(mu); sg2 = torch.zeros_like(mu)
    dec.decode_frame(fd, bs, n, z, y2, mu2, sg2)
    torch.cuda.synchronize()
    enc.close(); dec.close()
    return dict(mu=mu.cpu().numpy(), sg=sg.cpu().numpy(), bs=bs[:n].cpu().numpy().tobytes(), y=y2.cpu().numpy(),
                mu2=mu2.cpu().numpy(), sg2=sg2.cpu().numpy())


@pytest.mark.parametrize("precision", [psw.PSW_BF16, psw.PSW_FP8])
def test_cyclic_1080p_crop_vs_oracle(precision):
    """An 8 x 120 frame of the 1080p cyclic model (the same frame on both
    sides): lossless, decoder == encoder, parameters within tolerance, rate
    within 0.1 %, the container equal to the oracle coder's."""
    base = synth.config("i1080_cyc")
    w = synth.weights(base)
    cfg = base.with_grid(8, base.W)
    fr = synth.frames(cfg, 1, seed=1601)
    r = _encode_decode(psw.Context(base, w, precision=precision), fr)
    assert np.array_equal(r["y"], fr.y[0])
    assert np.array_equal(r["mu"], r["mu2"]) and np.array_equal(r["sg"], r["sg2"])
    mu_o, sg_o = O.run(cfg, oracle_weights(base, w, precision), fr.y, fr.z, driver=0)
    tol = TOLS[precision]
    dmu, dls = param_errors(r["mu"], r["sg"], mu_o[0], sg_o[0])
    q = (np.quantile(dmu, 0.999), np.quantile(dls, 0.999))
    assert q[0] <= tol and q[1] <= tol, q
    assert dmu.max() <= MAX_FACTOR * tol and dls.max() <= MAX_FACTOR * tol, (dmu.max(), dls.max())
    print(f"observed errors (99.9th pct, max): |dmu|/sigma {q[0]:.3g}, {dmu.max():.3g}; "
          f"|d ln sigma| {q[1]:.3g}, {dls.max():.3g}")
    ra = O.rate_bits(fr.y[0], r["mu"].astype(np.float64), r["sg"].astype(np.float64))
    rb = O.rate_bits(fr.y[0], mu_o[0], sg_o[0])
    assert abs(ra - rb) <= RATE_TOL * rb
    idx, m = O.quantize(r["mu"], r["sg"])
    assert r["bs"] == O.rans_encode(cfg, 0, fr.y[0], idx, m)


@pytest.mark.parametrize("precision", [psw.PSW_BF16, psw.PSW_FP8])
def test_cyclic_1080p_full_frame_and_batch(precision):
    """The full 68 x 120 frame in 4 steps: lossless, decoder == encoder; two
    frames decoded in one call equal each decoded alone."""
    cfg = synth.config("i1080_cyc")
    ctx = psw.Context(cfg, synth.weights(cfg), precision=precision)
    frs = [synth.frames(cfg, 1, seed=1602 + k) for k in range(2)]
    items = []
    for fr in frs:
        r = _encode_decode(ctx, fr)
        assert np.array_equal(r["y"], fr.y[0])
        assert np.array_equal(r["mu"], r["mu2"]) and np.array_equal(r["sg"], r["sg2"])
        items.append(r)
    fd = psw.frame_desc(cfg.H, cfg.W, psw.PSW_SCHED_WAVEFRONT)
    seqs = [ctx.seq_create(cfg.H, cfg.W) for _ in frs]
    bss = [torch.from_numpy(np.frombuffer(r["bs"], np.uint8).copy()).to(dev()) for r in items]
    zs = [_t(fr.z[0]) for fr in frs]
    ys = [torch.full((cfg.H, cfg.W, cfg.C), 7, dtype=torch.int16, device=dev()) for _ in frs]
    mus = [torch.zeros((cfg.H, cfg.W, cfg.C), dtype=torch.float32, device=dev()) for _ in frs]
    sgs = [torch.zeros_like(m) for m in mus]
    st = ctx.decode_batch(seqs, [fd, fd], bss, [len(r["bs"]) for r in items], zs, ys, mus, sgs)
    assert st == [psw.PSW_OK, psw.PSW_OK]
    for k, r in enumerate(items):
        assert np.array_equal(ys[k].cpu().numpy(), frs[k].y[0])
        assert np.array_equal(mus[k].cpu().numpy(), r["mu"]) and np.array_equal(sgs[k].cpu().numpy(), r["sg"])
