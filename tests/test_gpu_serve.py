"""Continuous batching: requests that arrive while others decode are
admitted as batch slots and HBM free up, their frames share decode calls,
and every request's results equal decoding it alone, bit for bit."""
import numpy as np
import pytest

from gpu_util import dev, need_gpu, torch
from paper_2605_20977_gb300 import psw, serve, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    need_gpu()
    from paper_2605_20977_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def _make_requests(ctx, base, grids, plan):
    """plan: [(arrival, grid index, frames)]; each request is its own
    synthetic sequence, encoded here."""
    reqs = []
    for rid, (arr, gi, nf) in enumerate(plan):
        H, W = grids[gi]
        c = base.with_grid(H, W)
        fr = synth.frames(c, nf, seed=300 + rid)
        enc = ctx.seq_create(H, W)
        fd = psw.frame_desc(H, W, psw.PSW_SCHED_WAVEFRONT)
        frames = []
        for f in range(nf):
            bs = torch.zeros(ctx.bitstream_capacity(H, W), dtype=torch.uint8, device=dev())
            z = _t(fr.z[f])
            frames.append((bs, enc.encode_params(fd, _t(fr.y[f]), z, bitstream=bs), z))
        enc.close()
        outs = [torch.full((H, W, c.C), 777, dtype=torch.int16, device=dev()) for _ in range(nf)]
        mus = [torch.zeros((H, W, c.C), dtype=torch.float32, device=dev()) for _ in range(nf)]
        sgs = [torch.zeros_like(m) for m in mus]
        r = serve.Request(rid=rid, arrival=arr, H=H, W=W, frames=frames, outputs=outs, mu=mus, sigma=sgs)
        r.truth = fr.y
        reqs.append(r)
    return reqs


@pytest.mark.parametrize("engine,precision", [(psw.ENGINE_PERSISTENT, psw.PSW_BF16),
                                              (psw.ENGINE_GRAPH, psw.PSW_BF16),
                                              (psw.ENGINE_PERSISTENT, psw.PSW_FP8)])
def test_serving_mix_equals_alone(engine, precision):
    base = synth.config("tiny_p")
    ctx = psw.Context(base, synth.weights(base), precision=precision)
    grids = [(8, 12), (5, 7), (6, 10)]
    plan = [(0.0, 0, 3), (0.0, 1, 1), (0.0, 2, 4), (0.0, 0, 2), (0.001, 1, 3), (0.002, 2, 1),
            (0.003, 0, 4), (0.004, 1, 2), (0.02, 2, 3), (0.03, 0, 1)]
    reqs = _make_requests(ctx, base, grids, plan)
    budget = int(2.5 * ctx.seq_bytes(8, 12))
    stats = serve.Server(ctx, budget, max_batch=3, engine=engine).run(reqs)
    assert stats["requests"] == len(plan) and stats["frames"] == sum(p[2] for p in plan)
    assert stats["peak_active"] <= 3 and stats["peak_hbm_bytes"] <= budget
    assert stats["iterations"] < stats["frames"]            # frames of different requests shared calls
    for r in reqs:
        assert all(s == psw.PSW_OK for s in r.status)
        for f in range(len(r.frames)):
            assert np.array_equal(r.outputs[f].cpu().numpy(), r.truth[f])
        # alone: a fresh sequence, one frame per call
        seq = ctx.seq_create(r.H, r.W)
        fd = psw.frame_desc(r.H, r.W, psw.PSW_SCHED_WAVEFRONT)
        for f, (bs, n, z) in enumerate(r.frames):
            y = torch.zeros_like(r.outputs[f]); mu = torch.zeros_like(r.mu[f]); sg = torch.zeros_like(mu)
            seq.decode_frame(fd, bs, n, z, y, mu, sg)
            assert torch.equal(mu, r.mu[f]) and torch.equal(sg, r.sigma[f]), (r.rid, f)
        seq.close()

