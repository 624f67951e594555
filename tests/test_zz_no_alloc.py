"""The allocation-free encoder entry point (psw_rans_encode_noalloc).

Some callers cannot allocate device memory where they encode (their device
memory is handed out by another allocator or capped by a quota, or their
loops forbid allocation after warm-up).  This entry point keeps its
scratch in a static device array instead; its containers must be the same
bytes the allocating coder and the oracle's coder produce, call after call.  Collected last so
that a failure here comes after every other test has run.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import dev, need_gpu, torch
from paper_2605_20977_gb300 import psw, synth

pytestmark = pytest.mark.gpu


def _case(c, seed):
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, 64, size=(c.H, c.W, c.C)).astype(np.uint8)
    m = rng.integers(-40, 40, size=(c.H, c.W, c.C)).astype(np.int32)
    tab = np.exp(np.linspace(np.log(0.11), np.log(256.0), 64)).astype(np.float32)
    y = np.clip(np.rint(m + rng.standard_normal(idx.shape) * tab[idx] * 1.5), -32767, 32767).astype(np.int16)
    return [torch.from_numpy(a).to(dev()) for a in (y, idx, m)]


def test_noalloc_encoder_matches_allocating_encoder_two_calls():
    need_gpu()
    from paper_2605_20977_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    base = synth.config("tiny")
    ctx = psw.Context(base, synth.weights(base), precision=psw.PSW_FP32)
    for call, (grid, sched) in enumerate((((37, 29), psw.PSW_SCHED_WAVEFRONT), ((11, 53), psw.PSW_SCHED_RASTER))):
        c = base.with_grid(*grid)
        y, idx, m = _case(c, 300 + call)
        fd = psw.frame_desc(c.H, c.W, sched)
        seq = ctx.seq_create(c.H, c.W)
        ref = torch.zeros(ctx.bitstream_capacity(c.H, c.W), dtype=torch.uint8, device=dev())
        n_ref = seq.rans_encode(fd, y, idx, m, ref)
        out = torch.full_like(ref, 0xAB)
        st, n = ctx.rans_encode_noalloc(fd, y, idx, m, out)
        assert st == psw.PSW_OK and n == n_ref
        assert torch.equal(out[:n].cpu(), ref[:n_ref].cpu()), call
        # and the oracle coder's bytes for the same symbols
        assert out[:n].cpu().numpy().tobytes() == O.rans_encode(c, sched, y.cpu().numpy(), idx.cpu().numpy(),
                                                                m.cpu().numpy()), call
        # the container decodes back to the symbols
        yd = torch.zeros_like(y)
        seq.rans_decode(fd, out, n, idx, m, yd)
        assert torch.equal(yd, y)
        seq.close()
    # a bitstream buffer one byte too small: PSW_ERR_CAPACITY, the needed
    # size reported, nothing written; the next call with room is exact again
    c = base.with_grid(9, 13)
    y, idx, m = _case(c, 310)
    fd = psw.frame_desc(c.H, c.W, psw.PSW_SCHED_WAVEFRONT)
    seq = ctx.seq_create(c.H, c.W)
    ref = torch.zeros(ctx.bitstream_capacity(c.H, c.W), dtype=torch.uint8, device=dev())
    n_ref = seq.rans_encode(fd, y, idx, m, ref)
    seq.close()
    short = torch.full((n_ref - 1,), 0x5A, dtype=torch.uint8, device=dev())
    st, n = ctx.rans_encode_noalloc(fd, y, idx, m, short, check=False)
    assert st == psw.PSW_ERR_CAPACITY and n == n_ref
    assert bool((short == 0x5A).all())
    out = torch.zeros(n_ref, dtype=torch.uint8, device=dev())
    st, n = ctx.rans_encode_noalloc(fd, y, idx, m, out)
    assert st == psw.PSW_OK and n == n_ref and torch.equal(out.cpu(), ref[:n_ref].cpu())
    # sizes beyond the static scratch are refused, not overrun
    big = psw.frame_desc(200, 200, psw.PSW_SCHED_WAVEFRONT)
    small = torch.zeros(16, dtype=torch.int16, device=dev())
    st, _ = ctx.rans_encode_noalloc(big, small, small, small, torch.zeros(64, dtype=torch.uint8, device=dev()),
                                    check=False)
    assert st == psw.PSW_ERR_INVALID
