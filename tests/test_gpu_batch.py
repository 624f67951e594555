"""Batched decoding and graph replay on the GPU.

A frame decoded inside a batch (its wavefront steps sharing launches with
other frames of other sequences, grids and schedules) must give exactly the
latents and (mu, sigma) it gives when decoded alone; replays of a captured
decode must repeat bit for bit, report a corrupt container and recover.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import dev, need_gpu, torch
from paper_2605_20977_gb300 import psw, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    need_gpu()
    from paper_2605_20977_gb300 import build
    build.build()
    O.build()
    torch.cuda.set_device(0)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def _encode(ctx, cfg, fr, sched):
    """Encode every frame of fr with a fresh sequence; returns per-frame
    (bitstream tensor, length, z tensor, y numpy)."""
    H, W = fr.y.shape[1], fr.y.shape[2]
    enc = ctx.seq_create(H, W)
    fd = psw.frame_desc(H, W, sched)
    out = []
    for f in range(fr.y.shape[0]):
        bs = torch.zeros(ctx.bitstream_capacity(H, W), dtype=torch.uint8, device=dev())
        z = _t(fr.z[f])
        n = enc.encode_params(fd, _t(fr.y[f]), z, bitstream=bs)
        out.append((bs, n, z, fr.y[f]))
    enc.close()
    return out


def _alloc(H, W, C):
    y = torch.full((H, W, C), 7777, dtype=torch.int16, device=dev())
    mu = torch.zeros((H, W, C), dtype=torch.float32, device=dev())
    return y, mu, torch.zeros_like(mu)


def _alone(ctx, cfg, items, fds):
    res = []
    for (bs, n, z, y), fd in zip(items, fds):
        seq = ctx.seq_create(fd.H, fd.W)
        yo, mu, sg = _alloc(fd.H, fd.W, cfg.C)
        seq.decode_frame(fd, bs, n, z, yo, mu, sg)
        res.append((yo.cpu().numpy(), mu.cpu().numpy(), sg.cpu().numpy()))
        seq.close()
    return res


def _batched(ctx, cfg, items, fds, seqs=None):
    seqs = seqs or [ctx.seq_create(fd.H, fd.W) for fd in fds]
    outs = [_alloc(fd.H, fd.W, cfg.C) for fd in fds]
    st = ctx.decode_batch(seqs, fds, [it[0] for it in items], [it[1] for it in items], [it[2] for it in items],
                          [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs])
    assert st == [psw.PSW_OK] * len(fds)
    return [(o[0].cpu().numpy(), o[1].cpu().numpy(), o[2].cpu().numpy()) for o in outs], seqs


def _check_same(alone, batched, items):
    for (ya, ma, sa), (yb, mb, sb), it in zip(alone, batched, items):
        assert np.array_equal(ya, it[3]) and np.array_equal(yb, it[3])
        assert np.array_equal(ma, mb) and np.array_equal(sa, sb)


@pytest.mark.parametrize("precision", [psw.PSW_FP32, psw.PSW_BF16, psw.PSW_FP8])
def test_batch_equals_alone_mixed_grids_and_schedules(precision):
    base = synth.config("tiny")
    ctx = psw.Context(base, synth.weights(base), precision=precision)
    plan = [((8, 12), 0), ((5, 7), 1), ((8, 3), 0), ((1, 1), 0), ((6, 12), 0)]
    items, fds = [], []
    for k, ((H, W), sched) in enumerate(plan):
        c = base.with_grid(H, W)
        items += _encode(ctx, c, synth.frames(c, 1, seed=50 + k), sched)
        fds.append(psw.frame_desc(H, W, sched))
    alone = _alone(ctx, base, items, fds)
    batched, _ = _batched(ctx, base, items, fds)
    _check_same(alone, batched, items)


@pytest.mark.parametrize("precision", [psw.PSW_BF16, psw.PSW_FP8])
def test_batch_equals_alone_1080p(precision):
    cfg = synth.config("i1080")
    ctx = psw.Context(cfg, synth.weights(cfg), precision=precision)
    plan = [(68, 120), (12, 120), (17, 30)]
    items, fds = [], []
    for k, (H, W) in enumerate(plan):
        c = cfg.with_grid(H, W)
        items += _encode(ctx, c, synth.frames(c, 1, seed=70 + k), 0)
        fds.append(psw.frame_desc(H, W, 0))
    alone = _alone(ctx, cfg, items, fds)
    batched, _ = _batched(ctx, cfg, items, fds)
    _check_same(alone, batched, items)


def test_graph_replay_repeats_and_recovers_from_corruption():
    cfg = synth.config("tiny")
    ctx = psw.Context(cfg, synth.weights(cfg), precision=psw.PSW_BF16)
    items = _encode(ctx, cfg, synth.frames(cfg, 1, seed=90), 0)
    bs, n, z, y = items[0]
    fd = psw.frame_desc(cfg.H, cfg.W, 0)
    seq = ctx.seq_create(cfg.H, cfg.W)
    first = None
    for rep in range(4):
        seq.reset()
        yo, mu, sg = _alloc(cfg.H, cfg.W, cfg.C)
        if rep == 2:
            bad = bs.clone()
            bad[16 + 4 * (cfg.C + 1) + 300] ^= 0x3C
            st = seq.decode_frame(fd, bad, n, z, yo, mu, sg, check=False)
            assert st == psw.PSW_ERR_CORRUPT or not np.array_equal(yo.cpu().numpy(), y)
            continue
        seq.decode_frame(fd, bs, n, z, yo, mu, sg)
        got = (yo.cpu().numpy(), mu.cpu().numpy(), sg.cpu().numpy())
        assert np.array_equal(got[0], y)
        if first is None:
            first = got
        else:
            assert np.array_equal(got[1], first[1]) and np.array_equal(got[2], first[2])
    # launches are counted for replayed graphs too: one kernel per phase of
    # every step on the graph engine, the prologue plus two on the
    # persistent one
    counts = {}
    for engine in (psw.ENGINE_GRAPH, psw.ENGINE_PERSISTENT):
        ctx.set_engine(engine)
        for rep in range(2):
            l0 = ctx.launch_count()
            seq.reset()
            yo, mu, sg = _alloc(cfg.H, cfg.W, cfg.C)
            seq.decode_frame(fd, bs, n, z, yo, mu, sg)
            assert np.array_equal(yo.cpu().numpy(), y)
            counts[engine] = ctx.launch_count() - l0
    assert counts[psw.ENGINE_GRAPH] > 100
    assert 3 <= counts[psw.ENGINE_PERSISTENT] < 20


def test_temporal_sequences_in_a_batch():
    cfg = synth.config("tiny_p")
    ctx = psw.Context(cfg, synth.weights(cfg), precision=psw.PSW_FP32)
    frs = [synth.frames(cfg, 4, seed=110 + k) for k in range(2)]
    enc = [_encode(ctx, cfg, fr, 0) for fr in frs]
    fd = psw.frame_desc(cfg.H, cfg.W, 0)
    solo = [ctx.seq_create(cfg.H, cfg.W) for _ in frs]
    pair = [ctx.seq_create(cfg.H, cfg.W) for _ in frs]
    for f in range(4):
        items = [enc[k][f] for k in range(2)]
        alone = []
        for k in range(2):
            yo, mu, sg = _alloc(cfg.H, cfg.W, cfg.C)
            solo[k].decode_frame(fd, items[k][0], items[k][1], items[k][2], yo, mu, sg)
            alone.append((yo.cpu().numpy(), mu.cpu().numpy(), sg.cpu().numpy()))
        batched, _ = _batched(ctx, cfg, items, [fd, fd], seqs=pair)
        _check_same(alone, batched, items)


def _engine_run(ctx, cfg, items, fds, engine):
    ctx.set_engine(engine)
    got, seqs = _batched(ctx, cfg, items, fds)
    for s in seqs:
        s.close()
    return got, ctx.last_engine()


@pytest.mark.parametrize("precision", [psw.PSW_BF16, psw.PSW_FP8])
def test_persistent_engine_equals_graph_engine(precision):
    """The persistent decoder (one cooperative launch over every step) and
    the per-phase graph decoder give bit-identical latents and parameters."""
    base = synth.config("tiny")
    ctx = psw.Context(base, synth.weights(base), precision=precision)
    plan = [((8, 12), 0), ((5, 7), 1), ((8, 3), 0), ((1, 1), 0), ((6, 12), 0)]
    items, fds = [], []
    for k, ((H, W), sched) in enumerate(plan):
        c = base.with_grid(H, W)
        items += _encode(ctx, c, synth.frames(c, 1, seed=130 + k), sched)
        fds.append(psw.frame_desc(H, W, sched))
    g, eg = _engine_run(ctx, base, items, fds, psw.ENGINE_GRAPH)
    p, ep = _engine_run(ctx, base, items, fds, psw.ENGINE_PERSISTENT)
    assert (eg, ep) == (psw.ENGINE_GRAPH, psw.ENGINE_PERSISTENT)
    _check_same(g, p, items)
    a, ea = _engine_run(ctx, base, items, fds, psw.ENGINE_AUTO)
    assert ea == psw.ENGINE_GRAPH
    _check_same(g, a, items)


@pytest.mark.parametrize("precision", [psw.PSW_BF16, psw.PSW_FP8])
def test_persistent_engine_1080p_and_temporal(precision):
    cfg = synth.config("i1080")
    ctx = psw.Context(cfg, synth.weights(cfg), precision=precision)
    plan = [(68, 120), (9, 120), (17, 30)]
    items, fds = [], []
    for k, (H, W) in enumerate(plan):
        c = cfg.with_grid(H, W)
        items += _encode(ctx, c, synth.frames(c, 1, seed=140 + k), 0)
        fds.append(psw.frame_desc(H, W, 0))
    g, _ = _engine_run(ctx, cfg, items, fds, psw.ENGINE_GRAPH)
    p, ep = _engine_run(ctx, cfg, items, fds, psw.ENGINE_PERSISTENT)
    assert ep == psw.ENGINE_PERSISTENT
    _check_same(g, p, items)

    tcfg = synth.config("tiny_p")
    tctx = psw.Context(tcfg, synth.weights(tcfg), precision=precision)
    fr = synth.frames(tcfg, 3, seed=150)
    enc = _encode(tctx, tcfg, fr, 0)
    fd = psw.frame_desc(tcfg.H, tcfg.W, 0)
    outs = {}
    for engine in (psw.ENGINE_GRAPH, psw.ENGINE_PERSISTENT):
        tctx.set_engine(engine)
        seq = tctx.seq_create(tcfg.H, tcfg.W)
        outs[engine] = []
        for f in range(3):
            yo, mu, sg = _alloc(tcfg.H, tcfg.W, tcfg.C)
            seq.decode_frame(fd, enc[f][0], enc[f][1], enc[f][2], yo, mu, sg)
            assert tctx.last_engine() == engine
            outs[engine].append((yo.cpu().numpy(), mu.cpu().numpy(), sg.cpu().numpy()))
        seq.close()
    _check_same(outs[psw.ENGINE_GRAPH], outs[psw.ENGINE_PERSISTENT], enc)


def test_engine_selection_errors():
    cfg = synth.config("tiny")
    ctx = psw.Context(cfg, synth.weights(cfg), precision=psw.PSW_FP32)
    with pytest.raises(psw.PswError):
        ctx.set_engine(psw.ENGINE_PERSISTENT)
    with pytest.raises(psw.PswError):
        ctx.set_engine(7)
    ctx.set_engine(psw.ENGINE_AUTO)


def test_destroyed_sequences_leave_no_stale_graphs():
    """Graphs that captured a sequence's buffers are dropped with it: fresh
    sequences (which may reuse the old objects' addresses) decode correctly
    on either engine, over several create/destroy rounds."""
    base = synth.config("tiny")
    ctx = psw.Context(base, synth.weights(base), precision=psw.PSW_BF16)
    plan = [((8, 12), 0), ((5, 7), 1), ((6, 12), 0)]
    items, fds = [], []
    for k, ((H, W), sched) in enumerate(plan):
        c = base.with_grid(H, W)
        items += _encode(ctx, c, synth.frames(c, 1, seed=170 + k), sched)
        fds.append(psw.frame_desc(H, W, sched))
    ref = None
    for engine in (psw.ENGINE_GRAPH, psw.ENGINE_PERSISTENT, psw.ENGINE_GRAPH, psw.ENGINE_AUTO,
                   psw.ENGINE_PERSISTENT, psw.ENGINE_GRAPH):
        got, _ = _engine_run(ctx, base, items, fds, engine)
        if ref is None:
            ref = got
        _check_same(ref, got, items)


def test_graph_cache_is_bounded_and_records_again():
    """More batch shapes than the context keeps graphs for: the oldest are
    dropped and recorded again when needed, with the same results."""
    cfg = synth.config("tiny")
    ctx = psw.Context(cfg, synth.weights(cfg), precision=psw.PSW_BF16)
    ctx.set_engine(psw.ENGINE_GRAPH)
    items = _encode(ctx, cfg, synth.frames(cfg, 1, seed=95), 0)
    bs, n, z, y = items[0]
    fd = psw.frame_desc(cfg.H, cfg.W, 0)
    seqs = [ctx.seq_create(cfg.H, cfg.W) for _ in range(20)]
    first = None
    for rnd in range(2):
        for q in seqs:                                  # 20 single-frame batch shapes (one key each)
            q.reset()
            yo, mu, sg = _alloc(cfg.H, cfg.W, cfg.C)
            q.decode_frame(fd, bs, n, z, yo, mu, sg)
            got = (yo.cpu().numpy(), mu.cpu().numpy(), sg.cpu().numpy())
            assert np.array_equal(got[0], y)
            if first is None:
                first = got
            assert np.array_equal(got[1], first[1]) and np.array_equal(got[2], first[2])
    for q in seqs:
        q.close()


@pytest.mark.parametrize("precision", [psw.PSW_BF16, psw.PSW_FP8])
def test_wide_batch_1080p_lean_tiles(precision):
    """48 full 1080p frames in one call: the projections of the middle
    wavefront steps have more tiles than the GPU has SMs, so they run as
    lean two-CTA tiles.  Every frame decodes losslessly, and frames spread
    over the batch equal the same frames decoded alone (one-CTA tiles)."""
    cfg = synth.config("i1080")
    ctx = psw.Context(cfg, synth.weights(cfg), precision=precision)
    B = 48
    four = _encode(ctx, cfg, synth.frames(cfg, 4, seed=2100), 0)     # I-frames: each coded on its own
    items = [four[b % 4] for b in range(B)]
    fds = [psw.frame_desc(cfg.H, cfg.W, 0)] * B
    batched, seqs = _batched(ctx, cfg, items, fds)
    for s in seqs:
        s.close()
    for (yb, _, _), it in zip(batched, items):
        assert np.array_equal(yb, it[3])
    pick = [0, 17, 46, 47]
    alone = _alone(ctx, cfg, [items[k] for k in pick], [fds[k] for k in pick])
    _check_same(alone, [batched[k] for k in pick], [items[k] for k in pick])


def test_largest_batch_512_frames():
    """512 frames in one call (the largest batch; slots 256-511 set the top
    bit of the token word): 8 x 120 crops of the 1080p model, BF16.  Every
    frame decodes losslessly, frames in both halves of the slot range equal
    the same frames decoded alone, and a 513-frame batch is refused."""
    cfg = synth.config("i1080").with_grid(8, 120)
    ctx = psw.Context(synth.config("i1080"), synth.weights(synth.config("i1080")), precision=psw.PSW_BF16)
    B = 512
    four = _encode(ctx, cfg, synth.frames(cfg, 4, seed=2110), 0)
    items = [four[b % 4] for b in range(B)]
    fds = [psw.frame_desc(cfg.H, cfg.W, 0)] * B
    batched, seqs = _batched(ctx, cfg, items, fds)
    for (yb, _, _), it in zip(batched, items):
        assert np.array_equal(yb, it[3])
    pick = [0, 255, 256, 511]
    alone = _alone(ctx, cfg, [items[k] for k in pick], [fds[k] for k in pick])
    _check_same(alone, [batched[k] for k in pick], [items[k] for k in pick])
    extra = ctx.seq_create(cfg.H, cfg.W)
    outs = [_alloc(cfg.H, cfg.W, cfg.C) for _ in range(B + 1)]
    with pytest.raises(psw.PswError):
        ctx.decode_batch(seqs + [extra], fds + [fds[0]], [it[0] for it in items] + [items[0][0]],
                         [it[1] for it in items] + [items[0][1]], [it[2] for it in items] + [items[0][2]],
                         [o[0] for o in outs])
    for s in seqs + [extra]:
        s.close()


def test_bounded_wait_expires_and_the_context_stays_usable():
    """The persistent decoder's grid-barrier wait, on a barrier no block
    arrives at, expires after its limit and reports PSW_ERR_TIMEOUT through
    the status word; a decode on the same context then succeeds."""
    cfg = synth.config("tiny")
    ctx = psw.Context(cfg, synth.weights(cfg), precision=psw.PSW_BF16)
    import time
    t0 = time.perf_counter()
    assert ctx.check_wait_timeout(0.05) == psw.PSW_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert "expired" in ctx.last_error()
    items = _encode(ctx, cfg, synth.frames(cfg, 1, seed=97), 0)
    bs, n, z, y = items[0]
    seq = ctx.seq_create(cfg.H, cfg.W)
    yo, mu, sg = _alloc(cfg.H, cfg.W, cfg.C)
    seq.decode_frame(psw.frame_desc(cfg.H, cfg.W, 0), bs, n, z, yo, mu, sg)
    assert np.array_equal(yo.cpu().numpy(), y)
