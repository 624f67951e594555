"""Host logic of the continuous-batching server, against a fake context
(no GPU): FIFO admission under the batch-slot and HBM limits, release of
finished requests, one decode call per iteration over every active
request, seeded arrival traces."""
import pytest

from paper_2605_20977_gb300 import psw, serve


class FakeSeq:
    def __init__(self, ctx, H, W):
        self.ctx, self.H, self.W, self.open = ctx, H, W, True
        ctx.live.append(self)
        ctx.created += 1

    def reset(self):
        assert self.open

    def close(self):
        assert self.open
        self.open = False
        self.ctx.live.remove(self)


class FakeCtx:
    """Sequence state costs H*W bytes; a decode call takes `dt` seconds of
    the fake clock and records which requests' frames it carried."""

    def __init__(self, clock, dt=1.0):
        self.clock, self.dt, self.live, self.calls, self.engine, self.created = clock, dt, [], [], None, 0

    def set_engine(self, e):
        self.engine = e

    def seq_bytes(self, H, W):
        return H * W

    def seq_create(self, H, W):
        return FakeSeq(self, H, W)

    def decode_batch(self, seqs, fds, bss, lens, zs, outs, mus, sigmas, check=True):
        assert len(set(map(id, seqs))) == len(seqs) and all(s.open for s in seqs)
        assert all((fd.H, fd.W) == (s.H, s.W) for fd, s in zip(fds, seqs))
        self.calls.append([b for b in bss])
        self.clock.t += self.dt
        return [psw.PSW_OK] * len(seqs)


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


def _req(rid, arrival, H, W, nf):
    return serve.Request(rid=rid, arrival=arrival, H=H, W=W,
                         frames=[((rid, f), 1, None) for f in range(nf)], outputs=[None] * nf)


def test_admission_limits_and_fifo():
    clock = Clock()
    ctx = FakeCtx(clock)
    reqs = [_req(0, 0.0, 10, 10, 3), _req(1, 0.0, 10, 10, 1), _req(2, 0.0, 20, 10, 2),
            _req(3, 0.5, 5, 5, 2), _req(4, 2.5, 10, 10, 1), _req(5, 9.0, 5, 5, 1)]
    def sleep(dt):
        assert dt > 0
        clock.t += dt

    stats = serve.Server(ctx, hbm_budget=300, max_batch=2, engine=7).run(reqs, clock=clock, sleep=sleep)
    assert ctx.engine == 7 and not ctx.live
    # every frame decoded exactly once, in order per request
    carried = [b for call in ctx.calls for b in call]
    assert sorted(carried) == sorted((r.rid, f) for r in reqs for f in range(len(r.frames)))
    for r in reqs:
        mine = [b for b in carried if b[0] == r.rid]
        assert mine == [(r.rid, f) for f in range(len(r.frames))]
    assert all(len(c) <= 2 for c in ctx.calls)
    assert stats["peak_active"] <= 2 and stats["peak_hbm_bytes"] <= 300
    # request 2 (200 bytes) waits for memory; request 3 arrives later but
    # joins once a slot is free, never ahead of an earlier arrival
    order = sorted(reqs, key=lambda r: r.admitted)
    assert [r.rid for r in order] == sorted(r.rid for r in reqs)
    assert all(r.done > r.arrival for r in reqs)
    assert stats["frames"] == 10 and stats["requests"] == 6
    # the idle gap before request 5 does not count as decode calls
    assert stats["iterations"] == len(ctx.calls)
    # finished sequence states are reused by later requests of the same grid
    assert ctx.created < len(reqs)


def test_oversized_request_is_rejected():
    clock = Clock()
    ctx = FakeCtx(clock)
    reqs = [_req(0, 0.0, 10, 10, 2), _req(1, 0.0, 100, 100, 1), _req(2, 0.1, 10, 10, 1)]
    stats = serve.Server(ctx, hbm_budget=500, max_batch=4).run(reqs, clock=clock, sleep=lambda dt: None)
    assert stats["rejected"] == 1 and stats["requests"] == 2 and stats["frames"] == 3
    assert reqs[1].done < 0 and reqs[0].done > 0 and reqs[2].done > 0


def test_poisson_trace_is_seeded():
    a = serve.poisson_trace(200.0, 1.0, [(15, 26), (30, 52)], seed=3)
    b = serve.poisson_trace(200.0, 1.0, [(15, 26), (30, 52)], seed=3)
    assert a == b and 120 < len(a) < 290
    assert all(0 <= t < 1.0 and g in (0, 1) and 1 <= n <= 16 for t, g, n in a)
