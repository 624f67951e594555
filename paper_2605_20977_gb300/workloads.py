"""Batched-uneven and serving workloads of the P-frame model (1080p sizes,
d=384, 8+1+8 blocks, Context Transformer over the current and two previous
frames) over four latent grids: 15x26, 30x52, 68x120 and 135x240.

* mixed: sequences of every grid decoded together, frame f of all of them
  per round.  A small autotuner times the candidate plans -- decode engine
  (per-phase graphs or the persistent kernel) x grouping (one call per
  round over all sequences, or one call per grid) -- on the first rounds and
  decodes the rest with the fastest.
* encode: the encoder's masked parallel pass (every position of a frame in
  one pass, 8160 tokens per launch at 1080p) and its rANS coding, frame
  after frame of the I-frame model; frames/s.  Small on the device, so it
  also serves as the case for profiler captures of the wide projection
  kernel.
* serve: seeded Poisson arrivals of 1..16-frame requests through the
  continuous-batching server (serve.Server), batched (in the chosen
  precision, E4M3 block projections by default) against one frame per call
  in BF16.

Frames come from a pool of seeded synthetic sequences per grid, encoded
once; a request or sequence decodes a pool sequence's first frames.

    python -m paper_2605_20977_gb300.workloads mixed --seqs 32 --frames 4 --precision fp8
    python -m paper_2605_20977_gb300.workloads serve --rate 200 --window 0.1 --precision fp8
    python -m paper_2605_20977_gb300.workloads encode --frames 4
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import build, psw, serve, synth

GRIDS = [(15, 26), (30, 52), (68, 120), (135, 240)]
PRECISIONS = {"bf16": psw.PSW_BF16, "fp8": psw.PSW_FP8}


class Pool:
    """Encoded P-frame sequences: per grid, `per_grid` sequences of `gop`
    frames (containers and hyperlatents on the device, latents kept for
    checking)."""

    def __init__(self, ctx, cfg, grids, per_grid, gop, dev, seed=1004):
        import torch
        self.items = {}
        for gi, (H, W) in enumerate(grids):
            c = cfg.with_grid(H, W)
            enc = ctx.seq_create(H, W)
            fd = psw.frame_desc(H, W, psw.PSW_SCHED_WAVEFRONT)
            seqs = []
            for k in range(per_grid):
                fr = synth.frames(c, gop, seed=seed + 1000 * gi + k)
                enc.reset()
                frames = []
                for f in range(gop):
                    bs = torch.zeros(ctx.bitstream_capacity(H, W), dtype=torch.uint8, device=dev)
                    z = torch.from_numpy(fr.z[f]).to(dev)
                    n = enc.encode_params(fd, torch.from_numpy(fr.y[f]).to(dev), z, bitstream=bs)
                    frames.append((bs, n, z, fr.y[f]))
                seqs.append(frames)
            enc.close()
            self.items[gi] = seqs


def _mixed_round(ctx, seqs, grids_of, pool_of, outs, f, grouping):
    """Decode frame f of every sequence: one call, or one call per grid."""
    groups = [list(range(len(seqs)))] if grouping == "mixed" else \
        [[i for i in range(len(seqs)) if grids_of[i] == g] for g in sorted(set(grids_of))]
    for idx in groups:
        if not idx:
            continue
        ctx.decode_batch([seqs[i] for i in idx],
                         [psw.frame_desc(*GRIDS[grids_of[i]], psw.PSW_SCHED_WAVEFRONT) for i in idx],
                         [pool_of[i][f][0] for i in idx], [pool_of[i][f][1] for i in idx],
                         [pool_of[i][f][2] for i in idx], [outs[i] for i in idx])


def run_mixed(nseq=32, nframes=4, tune_frames=1, seed=7, dev=None, precision="bf16"):
    import torch
    cfg = synth.config("p1080")
    ctx = psw.Context(cfg, synth.weights(cfg), precision=PRECISIONS[precision])
    per_grid = max(1, nseq // len(GRIDS))
    pool = Pool(ctx, cfg, GRIDS, per_grid, nframes, dev)
    rng = np.random.default_rng(seed)
    order = rng.permutation(per_grid * len(GRIDS))
    grids_of = [int(o) // per_grid for o in order]
    pool_of = [pool.items[int(o) // per_grid][int(o) % per_grid] for o in order]
    outs = [torch.zeros((*GRIDS[g], cfg.C), dtype=torch.int16, device=dev) for g in grids_of]

    def attempt(engine, grouping, frames):
        ctx.set_engine(engine)
        seqs = [ctx.seq_create(*GRIDS[g]) for g in grids_of]
        _mixed_round(ctx, seqs, grids_of, pool_of, outs, 0, grouping)     # records graphs, warms up
        for q in seqs:
            q.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for f in range(frames):
            _mixed_round(ctx, seqs, grids_of, pool_of, outs, f, grouping)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        ok = all(np.array_equal(outs[i].cpu().numpy(), pool_of[i][frames - 1][3]) for i in range(len(outs)))
        for q in seqs:
            q.close()
        return dt, ok

    plans = [(e, g) for e in (psw.ENGINE_GRAPH, psw.ENGINE_PERSISTENT) for g in ("mixed", "by_grid")]
    tune = {}
    for e, g in plans:
        dt, ok = attempt(e, g, tune_frames)
        if not ok:
            raise RuntimeError(f"mixed decode differs under plan {e}/{g}")
        tune[f"{'graph' if e == psw.ENGINE_GRAPH else 'persistent'}/{g}"] = len(outs) * tune_frames / dt
    best = max(tune, key=tune.get)
    e = psw.ENGINE_GRAPH if best.startswith("graph") else psw.ENGINE_PERSISTENT
    dt, ok = attempt(e, best.split("/")[1], nframes)
    if not ok:
        raise RuntimeError("mixed decode differs")
    gflop = {g: 2 * 57.3e6 * H * W / 1e9 for g, (H, W) in enumerate(GRIDS)}
    work = sum(gflop[g] for g in grids_of) * nframes
    ctx.close()
    return {"workload": f"{len(outs)} P-frame sequences ({per_grid} at each of "
            + ", ".join(f"{H}x{W}" for H, W in GRIDS) + f"), {nframes} frames each, {precision.upper()}",
            "plan": best, "autotune_frames_per_s": tune, "frames_per_s": len(outs) * nframes / dt,
            "tflops": work / dt / 1e3, "seconds": dt}


def tune_tiles(ctx, step, reps: int = 1, classes=(0, 1, 2, 3), widths=(0, 64, 128, 256)):
    """Autotuner of the wide projection kernel's tile widths (tokens per
    tile per launch class, psw_set_tile_policy): coordinate descent from the
    library's cost model, each candidate timed over `reps` calls of `step`
    after one untimed call (which records the new graphs).  Every width
    gives bit-identical results, so only time decides.  Leaves the best
    policy set; returns it with the timings."""
    import torch

    def timed():
        step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            step()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    names = {0: "qkv", 1: "residual", 2: "swiglu", 3: "other"}
    policy = [0, 0, 0, 0]
    for k in range(4):
        ctx.set_tile_policy(k, 0)
    best = timed()
    trials = {"auto": best}
    for k in classes:
        choice = policy[k]
        for wdt in widths:
            if wdt == policy[k]:
                continue
            ctx.set_tile_policy(k, wdt)
            t = timed()
            trials[f"{names[k]}={wdt}"] = t
            if t < best * 0.99:
                best, choice = t, wdt
        policy[k] = choice
        ctx.set_tile_policy(k, choice)
    return {"policy": {names[k]: policy[k] for k in range(4)}, "seconds_per_step": best,
            "trials_seconds_per_step": trials}


def run_serve(rate=200.0, window=0.1, per_grid=2, gop=16, budget_gb=120.0, max_batch=128, seed=1005, dev=None,
              unbatched=True, precision="fp8", engines=("graph",)):
    """Batched service in `precision` (once per decode engine in `engines`)
    against one frame per call in BF16, on the same arrival trace (each
    precision encodes its own streams)."""
    import torch
    cfg = synth.config("p1080")
    trace = serve.poisson_trace(rate, window, GRIDS, max_frames=gop, seed=seed)

    def requests(pool):
        reqs = []
        for rid, (t, gi, nf) in enumerate(trace):
            src = pool.items[gi][rid % per_grid]
            H, W = GRIDS[gi]
            r = serve.Request(rid=rid, arrival=t, H=H, W=W, frames=[(b, n, z) for b, n, z, _ in src[:nf]],
                              outputs=[torch.zeros((H, W, cfg.C), dtype=torch.int16, device=dev) for _ in range(nf)])
            r.truth = [y for *_, y in src[:nf]]
            reqs.append(r)
        return reqs

    out = {"workload": f"Poisson arrivals at {rate:g} requests/s over {window:g} s ({len(trace)} requests, "
           f"{sum(n for _, _, n in trace)} frames), 1..{gop} frames each, grids "
           + ", ".join(f"{H}x{W}" for H, W in GRIDS) + f"; HBM budget {budget_gb:g} GB; P-frame model"}
    eng = {"persistent": psw.ENGINE_PERSISTENT, "graph": psw.ENGINE_GRAPH}
    arms = [("batched" if len(engines) == 1 else f"batched_{e}", max_batch, precision, e) for e in engines]
    if unbatched:
        arms.append(("one_frame_per_call", 1, "bf16", engines[0]))
    ctxs = {}
    for name, mb, prec, e in arms:
        if prec not in ctxs:
            ctx = psw.Context(cfg, synth.weights(cfg), precision=PRECISIONS[prec])
            ctxs[prec] = (ctx, Pool(ctx, cfg, GRIDS, per_grid, gop, dev))
        ctx, pool = ctxs[prec]
        reqs = requests(pool)
        torch.cuda.synchronize()
        st = serve.Server(ctx, int(budget_gb * 2 ** 30), max_batch=mb, engine=eng[e]).run(reqs)
        for r in reqs:
            for f, y in enumerate(r.truth):
                if not np.array_equal(r.outputs[f].cpu().numpy(), y):
                    raise RuntimeError("served decode differs")
        st["precision"] = prec
        st["engine"] = e
        out[name] = st
        del reqs
    for ctx, pool in ctxs.values():
        del pool
        ctx.close()
    return out


def run_encode(nframes=4, dev=None, precision="bf16", rows=0):
    """Encode nframes 1080p I-frames one after another (masked pass plus
    rANS); the first is a warm-up.  Returns frames/s of the rest.  rows > 0:
    the top `rows` rows of the frame (rows x 120 tokens per launch, e.g. 34
    for the mean launch of a 128-frame wavefront decode)."""
    import torch
    base = synth.config("i1080")
    cfg = base.with_grid(rows, base.W) if rows else base
    ctx = psw.Context(base, synth.weights(base), precision=PRECISIONS[precision])
    seq = ctx.seq_create(cfg.H, cfg.W)
    fr = synth.frames(cfg, 1, seed=1002)
    fd = psw.frame_desc(cfg.H, cfg.W, psw.PSW_SCHED_WAVEFRONT)
    y = torch.from_numpy(fr.y[0]).to(dev)
    z = torch.from_numpy(fr.z[0]).to(dev)
    bs = torch.zeros(ctx.bitstream_capacity(cfg.H, cfg.W), dtype=torch.uint8, device=dev)
    seq.encode_params(fd, y, z, bitstream=bs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(max(0, nframes - 1)):
        seq.reset()
        seq.encode_params(fd, y, z, bitstream=bs)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    seq.close()
    ctx.close()
    n = max(0, nframes - 1)
    gflop = 505.0 * cfg.H / base.H
    return {"workload": f"encoder masked pass + rANS, 1080p I-frame model, {cfg.H}x{cfg.W}x{cfg.C} frames, "
            f"{precision.upper()}", "frames": n, "frames_per_s": n / dt if n else None,
            "tflops": n * gflop / dt / 1e3 if n else None}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["mixed", "serve", "encode"])
    ap.add_argument("--seqs", type=int, default=32)
    ap.add_argument("--frames", type=int, default=4)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--window", type=float, default=0.1)
    ap.add_argument("--no-unbatched", action="store_true")
    ap.add_argument("--rows", type=int, default=0, help="encode: rows of the 68-row frame (0: all)")
    ap.add_argument("--engines", default="graph",
                    help="serve: decode engines of the batched arm, comma separated (persistent, graph)")
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default=None,
                    help="mixed: bf16 (default); serve: the batched arm's precision, fp8 (default)")
    args = ap.parse_args()
    import torch
    build.build()
    dev = torch.device("cuda", 0)
    if args.what == "mixed":
        res = run_mixed(args.seqs, args.frames, dev=dev, precision=args.precision or "bf16")
    elif args.what == "encode":
        res = run_encode(args.frames, dev=dev, precision=args.precision or "bf16", rows=args.rows)
    else:
        res = run_serve(args.rate, args.window, dev=dev, unbatched=not args.no_unbatched,
                        precision=args.precision or "fp8", engines=tuple(args.engines.split(",")))
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
