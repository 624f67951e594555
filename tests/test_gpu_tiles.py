"""The wide projection kernel's tile policy (tokens per tile per launch
class, chosen by the autotuner; 256-token tiles are issued by two threads)
changes no value, in BF16 and with E4M3 block projections: the encoder's masked pass
over a 34 x 120 crop of the 1080p frame (4080 tokens per launch, every
projection on the wide kernel) gives bit-identical parameters and
containers under every policy, and a decoder under one policy reproduces an
encoder under another."""
import numpy as np
import pytest

from gpu_util import dev, need_gpu, torch
from paper_2605_20977_gb300 import psw, synth

pytestmark = pytest.mark.gpu

POLICIES = [(0, 0, 0, 0), (64, 64, 64, 64), (256, 256, 256, 256), (128, 64, 256, 128), (256, 128, 64, 256)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    need_gpu()
    from paper_2605_20977_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


@pytest.mark.parametrize("precision", [psw.PSW_BF16, psw.PSW_FP8])
def test_tile_policies_are_bit_identical(precision):
    base = synth.config("i1080")
    ctx = psw.Context(base, synth.weights(base), precision=precision)
    cfg = base.with_grid(34, base.W)
    fr = synth.frames(cfg, 1, seed=2401)
    fd = psw.frame_desc(cfg.H, cfg.W, 0)
    y, z = _t(fr.y[0]), _t(fr.z[0])
    ref = None
    for pol in POLICIES:
        for k, wdt in enumerate(pol):
            ctx.set_tile_policy(k, wdt)
        assert ctx.tile_policy() == list(pol)
        q = ctx.seq_create(cfg.H, cfg.W)
        mu = torch.zeros(y.shape, dtype=torch.float32, device=dev()); sg = torch.zeros_like(mu)
        bs = torch.zeros(ctx.bitstream_capacity(cfg.H, cfg.W), dtype=torch.uint8, device=dev())
        n = q.encode_params(fd, y, z, mu, sg, bs)
        q.close()
        out = (mu.cpu().numpy(), sg.cpu().numpy(), bs[:n].cpu().numpy().tobytes())
        if ref is None:
            ref = out
        else:
            assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1]) and out[2] == ref[2], pol
    # decode under the last policy what the first encoded
    dec = ctx.seq_create(cfg.H, cfg.W)
    y2 = torch.zeros_like(y)
    mu2 = torch.zeros(y.shape, dtype=torch.float32, device=dev())
    bs = torch.from_numpy(np.frombuffer(ref[2], np.uint8).copy()).to(dev())
    dec.decode_frame(fd, bs, len(ref[2]), z, y2, mu2)
    assert np.array_equal(y2.cpu().numpy(), fr.y[0]) and np.array_equal(mu2.cpu().numpy(), ref[0])
    dec.close()
    with pytest.raises(psw.PswError):
        ctx.set_tile_policy(4, 64)
    with pytest.raises(psw.PswError):
        ctx.set_tile_policy(0, 96)
