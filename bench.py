#!/usr/bin/env python3
"""Benchmark: wavefront decode of 1080p latent frames on one GB300.

Workload: the 1080p I-frame configuration -- latents 68x120x192 (a
1088x1920 frame after the /16 feature transform), hyperlatents 17x30x128,
context model d=384, 6 heads, 7x7 windows, 8 blocks in each spatial module
plus the accumulator, BF16 projections with FP32 accumulation.  A step
decodes one batch of frames (default 512) from their rANS containers along the
254 wavefronts 2i+j = t: every position of a wavefront is predicted
together, its symbols decoded, and the next wavefront follows.  Inputs are
synthetic (seeded AR(1) latents, random weights); the containers are made by
the library's own encoder before timing.

Printed: one JSON line (rank 0) with the device-timed frames/s (`value`),
the same through the C ABI with host buffers (`e2e`), raster-order decode of
the same frame on the same GPU, the roofline of the dominant kernel class
from CUDA events, SM clocks sampled during the timed region, and the FP64
CPU oracle timed on a bounded crop (`cpu_baseline`).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun, one rank per GPU) runs independent replicas: each rank
decodes its own frames (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "1080p latent frames/s (wavefront vs raster SWA, same GB300) at ≤0.1% rate delta vs FP64"
WORKLOAD = ("1080p I-frame decode: latents 68x120x192, hyperlatents 17x30x128, d=384 nh=6 k=7, "
            "8+1+8 blocks, BF16 projections / FP32 accumulate, wavefront 2i+j (254 steps)")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--batch", type=int, default=512, help="frames decoded per step (1..512)")
    ap.add_argument("--raster-frames", type=int, default=1, help="timed raster steps (0: skip raster)")
    ap.add_argument("--no-raster-batch", dest="raster_batch", action="store_false")
    ap.add_argument("--raster-batch-size", type=int, default=16,
                    help="frames per step of the batched raster comparison (the wavefront is timed at the same size)")
    ap.add_argument("--cpu-rows", type=int, default=8, help="rows of the 1080p frame in the oracle's sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--pframe-seqs", type=int, default=48,
                    help="P-frame GOP measurement: sequences decoded together (0: skip)")
    ap.add_argument("--pframe-gop", type=int, default=16, help="frames per P-frame sequence")
    ap.add_argument("--precision", choices=["bf16", "fp8"], default="bf16",
                    help="projections of the main leg: bf16, or fp8 (E4M3 block projections; the fp8 leg is then skipped)")
    ap.add_argument("--fp8-steps", type=int, default=2,
                    help="timed steps of the same I-frame workload with E4M3 block projections (0: skip)")
    ap.add_argument("--cyclic-steps", type=int, default=2,
                    help="timed steps of the cyclic s = 4 schedule leg (0: skip)")
    ap.add_argument("--lrp-steps", type=int, default=3,
                    help="timed LRP Transformer passes over one decoded 1080p frame (0: skip)")
    ap.add_argument("--hyper-steps", type=int, default=3,
                    help="timed passes of the convolutional hyperprior leg (0: skip)")
    ap.add_argument("--mixed-frames", type=int, default=4,
                    help="batched-uneven leg: frames per sequence of 32 P-frame sequences over four grids (0: skip)")
    ap.add_argument("--serve-rates", default="2,8,24",
                    help="serving sweep: Poisson request rates per second, comma separated (empty: skip)")
    ap.add_argument("--serve-window", type=float, default=5.0, help="serving sweep: arrival window in seconds")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="skip the tile-width autotuner (keep the library's cost model)")
    ap.add_argument("--engine", choices=["auto", "graph", "persistent"], default="auto",
                    help="decode engine: one cooperative kernel over all steps, or per-phase kernels in CUDA graphs")
    return ap.parse_args(argv)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {k: float(d[k]) for k in FALLBACK_PEAKS}, "measured"
    return dict(FALLBACK_PEAKS), "fallback"


# ------------------------------------------------------------------ clocks

class Clocks:
    """nvidia-smi sampling every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None

    def start(self):
        if os.environ.get("CUDA_INJECTION64_PATH"):     # under a profiler: no sampler child process
            return
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.f.flush(); self.f.seek(0)
        text = self.f.read()
        os.unlink(self.f.name)
        return self.summarise(text)

    @staticmethod
    def summarise(text: str) -> dict:
        """Median SM clock, the maximum clock and the throttle reasons seen
        active in nvidia-smi's CSV rows (the query Q, no header, no units);
        rows that do not parse are skipped."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in text.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ oracle leg

class OracleSample:
    """The FP64 oracle's wavefront decode of the top `rows` rows of the
    1080p frame (their parameters depend only on rows above them, so the
    crop is an exact sub-problem).  The crop is encoded once by the oracle;
    `time_decode` times one decode of it, rANS included."""

    def __init__(self, rows: int):
        import torch
        import oracle
        from paper_2605_20977_gb300 import synth
        oracle.build()
        self.O = oracle
        cfg = synth.config("i1080")
        self.cfg, self.rows = cfg, rows
        self.crop = cfg.with_grid(rows, cfg.W)
        w = synth.weights(cfg)
        fr = synth.frames(cfg, 1, seed=1002)
        self.y = fr.y[:, :rows].copy()
        self.z = fr.z[:, :self.crop.Hh].copy()
        mask = synth.matrix_mask(cfg)
        w64 = w.astype(np.float64)
        w64[mask] = torch.from_numpy(w[mask]).to(torch.bfloat16).to(torch.float64).numpy()
        self.w64 = w64
        self.bs, mu, sg = oracle.encode_frames(self.crop, w64, self.y, self.z)
        self.mu, self.sg = mu[0], sg[0]
        self.npos = rows * cfg.W
        self.threads = oracle.num_threads()
        self.synth = synth

    def fp8_params(self):
        """The oracle's parameters of the crop with the weights of an FP8
        context: E4M3-stored projections quantised per tensor, the other
        projections rounded to bf16."""
        w64 = self.w64.copy()
        w = self.synth.weights(self.cfg)
        for off, n in self.synth.e4m3_ranges(self.cfg):
            w64[off:off + n] = self.O.e4m3_tensor(w[off:off + n].astype(np.float64))[0]
        mu, sg = self.O.run(self.crop, w64, self.y, self.z, driver=0)
        return mu[0], sg[0]

    def time_decode(self) -> float:
        t0 = time.perf_counter()
        yd, _, _ = self.O.decode_frames(self.crop, self.w64, self.bs, self.z)
        dt = time.perf_counter() - t0
        if not np.array_equal(yd, self.y):
            raise RuntimeError("oracle decode differs")
        return dt

    def describe(self, secs: float) -> str:
        return (f"FP64 oracle wavefront decode (rANS included) of the top {self.rows} rows "
                f"({self.npos} of {self.cfg.H * self.cfg.W} positions) of the 1080p frame: "
                f"{secs:.2f} s per crop, extrapolated to a frame by positions")


def oracle_single_thread(rows: int = 1):
    """The oracle's decode of the top `rows` rows timed on one host thread
    (a child process with OMP_NUM_THREADS=1, set before the OpenMP runtime
    starts).  Returns (frames/s extrapolated by positions, sample text) or
    None if the child fails."""
    code = ("import sys, json; sys.path.insert(0, %r); import bench; s = bench.OracleSample(%d); "
            "t = s.time_decode(); print(json.dumps([t, s.npos, s.cfg.H * s.cfg.W, s.threads]))" % (ROOT, rows))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        t, npos, hw, threads = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception:
        return None
    return (npos / hw) / t, (f"FP64 oracle wavefront decode (rANS included) of the top {rows} row(s) "
                                     f"({npos} positions) on {threads} thread: {t:.2f} s, extrapolated by positions")


# ------------------------------------------------------------------ reference arm

def arm_config(args, world: int, engine: int) -> dict:
    """The workload's config object, the same on both arms (the reference
    arm's sample of it is described in its cpu_baseline).  engine: 2 for the
    persistent decoder, else the graph engine."""
    return {"workload": WORKLOAD if args.precision == "bf16" else WORKLOAD.replace(
                "BF16 projections", "E4M3 block projections (BF16 embedding and heads)"),
            "frames_per_step": args.batch,
            "l2": "flushed between steps (256 MiB write)",
            "launch": ("persistent: per-frame prologue in a CUDA graph, then one cooperative kernel "
                       "(one CTA per SM, grid barrier between phases) over all wavefront steps"
                       if engine == 2 else "CUDA graph per batch shape (segments of 512 wavefront steps)"),
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def run_reference(args, rank: int):
    if rank != 0:
        return 0
    rows = args.cpu_rows
    smp = OracleSample(rows)
    # warmup steps, then timed steps, each one decode of the crop
    secs = []
    for s in range(args.warmup + args.steps):
        t = smp.time_decode()
        if s >= args.warmup:
            secs.append(t)
    npos, threads = smp.npos, smp.threads
    frac = npos / (smp.cfg.H * smp.cfg.W)
    value = frac / float(np.mean(secs))
    sample = smp.describe(float(np.mean(secs)))
    line = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": arm_config(args, args.gpus, 2 if args.engine == "persistent" else 1),
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm

def traffic_for(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if
    the kernel source is unchanged since it was taken (the summary names the
    launch size it was measured at)."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")     # JSON: per-kernel DRAM bytes from the ncu summaries
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(kernel)
    if not d:
        return None
    src = os.path.join(ROOT, d["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest() != d["sha256"]:
        return None
    return d["dram_bytes_per_launch"]


def pframe_run(args, dev, stream, flush, timed):
    """1080p P-frame GOPs (Context Transformer over the current and two
    previous frames, temporal cross-attention in every spatial block):
    S sequences of G frames; call f decodes frame f of all S together."""
    import torch
    from paper_2605_20977_gb300 import psw, synth
    cfg = synth.config("p1080")
    ctx = psw.Context(cfg, synth.weights(cfg), precision=psw.PSW_BF16)
    S, G = args.pframe_seqs, args.pframe_gop
    fd = psw.frame_desc(cfg.H, cfg.W, psw.PSW_SCHED_WAVEFRONT)
    cap = ctx.bitstream_capacity(cfg.H, cfg.W)
    enc = ctx.seq_create(cfg.H, cfg.W)
    data = []                                   # [seq][frame] -> (bitstream, len, z, y)
    for s_ in range(S):
        fr = synth.frames(cfg, G, seed=1003 + 100 * s_)
        enc.reset()
        row = []
        for f in range(G):
            y = torch.from_numpy(fr.y[f]).to(dev); z = torch.from_numpy(fr.z[f]).to(dev)
            bs = torch.zeros(cap, dtype=torch.uint8, device=dev)
            row.append((bs, enc.encode_params(fd, y, z, bitstream=bs), z, y))
        data.append(row)
    enc.close()
    decs = [ctx.seq_create(cfg.H, cfg.W) for _ in range(S)]
    outs = [torch.zeros_like(data[0][0][3]) for _ in range(S)]

    def gop():
        for q in decs:
            q.reset()
        for f in range(G):
            ctx.decode_batch(decs, [fd] * S, [data[s_][f][0] for s_ in range(S)], [data[s_][f][1] for s_ in range(S)],
                             [data[s_][f][2] for s_ in range(S)], outs)

    gop()                                       # records the graphs
    ms = timed(gop, 2)
    for s_ in range(S):
        if not torch.equal(outs[s_], data[s_][G - 1][3]):
            raise RuntimeError("P-frame decode differs")
    t = float(np.mean(ms))
    ctx.close()
    return {"value": S * G * 1e3 / t, "unit": "frames/s", "sequences_per_call": S, "gop": G,
            "ms_per_gop": t, "workload": "1080p P-frame GOPs: latents 68x120x192 with temporal AR(1) 0.9, "
            "Context Transformer 8 blocks over the current and 2 previous frames, temporal cross-attention, BF16"}


def fp8_run(args, dev, timed, cfg, w, ys, zs, B):
    """The headline I-frame workload again with E4M3 block projections
    (encoded by an FP8 context, decoded B frames per call): throughput, the
    projection class's tensor rate against the E4M3 peak, and frame 0's
    parameters for the rate comparison."""
    import torch
    from paper_2605_20977_gb300 import psw
    ctx = psw.Context(cfg, w, precision=psw.PSW_FP8)
    fd = psw.frame_desc(cfg.H, cfg.W, psw.PSW_SCHED_WAVEFRONT)
    cap = ctx.bitstream_capacity(cfg.H, cfg.W)
    enc = ctx.seq_create(cfg.H, cfg.W)
    bss, lens = [], []
    for b in range(B):
        enc.reset()
        bs = torch.zeros(cap, dtype=torch.uint8, device=dev)
        lens.append(enc.encode_params(fd, ys[b], zs[b], bitstream=bs))
        bss.append(bs)
    mu = torch.zeros(ys[0].shape, dtype=torch.float32, device=dev); sg = torch.zeros_like(mu)
    enc.reset()
    enc.encode_params(fd, ys[0], zs[0], mu, sg)
    enc.close()
    decs = [ctx.seq_create(cfg.H, cfg.W) for _ in range(B)]
    outs = [torch.zeros_like(y) for y in ys]

    def step():
        for q in decs:
            q.reset()
        ctx.decode_batch(decs, [fd] * B, bss, lens, zs, outs)

    step()                                      # records the graphs
    ms = timed(step, args.fp8_steps)
    for b in range(B):
        if not torch.equal(outs[b], ys[b]):
            raise RuntimeError("FP8 decode differs")
    ctx.profile_begin()
    step()
    stats = ctx.profile_end()
    g = next((s_ for s_ in stats if s_["name"] == "gemm_tc"), None)
    pk, pk_kind = peaks()
    out = {"value": B * 1e3 / float(np.mean(ms)), "unit": "frames/s", "frames_per_step": B,
           "ms_per_step": float(np.mean(ms)), "dtype": "e4m3 block projections (per-tensor power-of-two weight "
           "scales, per-token activation scales), bf16 embedding/heads/caches, f32 accumulation",
           "bits_per_symbol": ctx.rate(ys[0], mu, sg) / ys[0].numel(),
           "container_bits_per_symbol": 8.0 * lens[0] / ys[0].numel()}
    if g:
        ach = g["flops"] / (g["ms"] / 1e3) / 1e12
        peak8 = 2.0 * pk["bf16_tflops_sustained"]
        out["projections"] = {"achieved": ach, "unit": "TFLOP/s", "peak": peak8, "frac": ach / peak8,
                              "peak_source": ("2 x measured sustained bf16 (nominal E4M3:BF16 ratio)"
                                              if pk_kind == "measured" else "2 x fallback bf16"),
                              "share_of_kernel_time": g["ms"] / sum(s_["ms"] for s_ in stats)}
    for q in decs:
        q.close()
    ctx.close()
    return out, mu, sg


def lrp_run(args, dev, timed, ys, zs):
    """The LRP Transformer (Sec. 3.1 latent residual prediction; 4 blocks,
    unmasked 7 x 7 windows) over one coded 68x120 frame: frames/s of
    psw_lrp_residual, its kernel classes from one instrumented pass and the
    projections' tensor rate (8160 tokens per launch)."""
    import torch
    from paper_2605_20977_gb300 import psw, synth
    cfg = synth.config("i1080_lrp")
    ctx = psw.Context(cfg, synth.weights(cfg), precision=psw.PSW_BF16)
    fd = psw.frame_desc(cfg.H, cfg.W, psw.PSW_SCHED_WAVEFRONT)
    q = ctx.seq_create(cfg.H, cfg.W)
    q.encode_params(fd, ys[0], zs[0])
    eps = torch.zeros(ys[0].shape, dtype=torch.float32, device=dev)
    q.lrp_residual(fd, eps)
    ms = timed(lambda: q.lrp_residual(fd, eps), args.lrp_steps)
    ctx.profile_begin()
    q.lrp_residual(fd, eps)
    stats = ctx.profile_end()
    if not bool(torch.isfinite(eps).all()):
        raise RuntimeError("LRP residual not finite")
    pk, _ = peaks()
    g = next((s_ for s_ in stats if s_["name"] == "gemm_tc"), None)
    nrm = next((s_ for s_ in stats if s_["name"] == "rmsnorm"), None)
    out = {"value": 1e3 / float(np.mean(ms)), "unit": "frames/s", "ms_per_frame": float(np.mean(ms)),
           "workload": "LRP Transformer (4 blocks, d = 384, 7x7 unmasked windows) over one coded 1080p frame "
                       "68x120x192 after its encode, BF16",
           "classes": {s_["name"]: {"ms": round(s_["ms"], 3), "launches": s_["launches"],
                                    "gflop": round(s_["flops"] / 1e9, 2)} for s_ in stats}}
    if g:
        t = g["ms"] + (nrm["ms"] if nrm else 0.0)
        ach = g["flops"] / (t / 1e3) / 1e12
        out["projections"] = {"achieved": ach, "unit": "TFLOP/s", "peak": pk["bf16_tflops_sustained"],
                              "frac": ach / pk["bf16_tflops_sustained"],
                              "timing": "CUDA events, projection launches plus the row normalisations feeding them",
                              "tokens_per_launch": cfg.H * cfg.W}
    q.close()
    ctx.close()
    return out


def hyper_run(args, dev, timed, ys, B):
    """The convolutional hyperprior (Fig. 1 right) at 1080p: per frame the
    encoder's analysis and z-hat coding (psw_hyper_encode: Spatial Module 1,
    two RB-down blocks, rANS under the factorized prior), the decoder's
    z-hat decode (psw_hyper_decode), and a B-frame batched decode whose
    prologues synthesise the hyperprior tokens (two RB-up blocks per frame).
    Inputs resident in HBM; the z-hat of each frame comes from its own
    analysis."""
    import torch
    from paper_2605_20977_gb300 import psw, synth
    cfg = synth.config("i1080_hp")
    ctx = psw.Context(cfg, synth.weights(cfg), precision=psw.PSW_BF16)
    fd = psw.frame_desc(cfg.H, cfg.W, psw.PSW_SCHED_WAVEFRONT)
    cap_z = ctx.bitstream_capacity(cfg.Hh, cfg.Wh) + 16 * cfg.Ch
    cap_y = ctx.bitstream_capacity(cfg.H, cfg.W)
    enc = ctx.seq_create(cfg.H, cfg.W)
    zhs, bzs, nzs, bys, nys = [], [], [], [], []
    for b in range(B):
        enc.reset()
        zh = torch.zeros((cfg.Hh, cfg.Wh, cfg.Ch), dtype=torch.int16, device=dev)
        bz = torch.zeros(cap_z, dtype=torch.uint8, device=dev)
        nzs.append(enc.hyper_encode(fd, ys[b], zh, None, bz))
        by = torch.zeros(cap_y, dtype=torch.uint8, device=dev)
        nys.append(enc.encode_params(fd, ys[b], zh, None, None, by))
        zhs.append(zh); bzs.append(bz); bys.append(by)
    zt = torch.zeros_like(zhs[0])
    ms_enc = timed(lambda: (enc.reset(), enc.hyper_encode(fd, ys[0], zt, None, bzs[0])), args.hyper_steps)
    ms_dec = timed(lambda: ctx.hyper_decode(fd, bzs[0], nzs[0], zt), args.hyper_steps)
    if not torch.equal(zt, zhs[0]):
        raise RuntimeError("z-hat decode differs")
    ctx.profile_begin()
    enc.reset()
    enc.hyper_encode(fd, ys[0], zt, None, bzs[0])
    st_enc = ctx.profile_end()
    enc.close()
    decs = [ctx.seq_create(cfg.H, cfg.W) for _ in range(B)]
    outs = [torch.zeros_like(y) for y in ys[:B]]

    def step():
        for q in decs:
            q.reset()
        ctx.decode_batch(decs, [fd] * B, bys, nys, zhs, outs)

    step()
    ms = timed(step, max(2, args.hyper_steps - 1))
    for b in range(B):
        if not torch.equal(outs[b], ys[b]):
            raise RuntimeError("hyperprior-model decode differs")
    for q in decs:
        q.close()
    ctx.close()
    g = next((s_ for s_ in st_enc if s_["name"] == "gemm_tc"), None)
    out = {"analysis_and_zhat_coding_ms_per_frame": float(np.mean(ms_enc)),
           "zhat_decode_ms_per_frame": float(np.mean(ms_dec)),
           "decode": {"value": B * 1e3 / float(np.mean(ms)), "unit": "frames/s", "frames_per_step": B},
           "zhat_bytes_per_frame": float(np.mean(nzs)),
           "workload": "1080p I-frames 68x120x192 with the convolutional hyperprior (2 RB-down / 2 RB-up "
                       "blocks, Ch = 128, factorized prior), BF16",
           "encode_classes": {s_["name"]: {"ms": round(s_["ms"], 3), "launches": s_["launches"],
                                           "gflop": round(s_["flops"] / 1e9, 2)} for s_ in st_enc}}
    if g:
        out["encode_projections_tflops"] = g["flops"] / (g["ms"] / 1e3) / 1e12
    return out


def cyclic_run(args, dev, timed, w, ys, zs, B, name="i1080_cyc"):
    """The paper's own schedule (cyclic s = 4 mask, Fig. 2a): the same model
    sizes and frames, 4 steps per frame of 2040 positions each.  Frames/s at
    B frames per call, single-frame latency, and the projections' tensor
    rate from one instrumented step (2040 tokens per frame in every launch).  name = "i1080_cyc_ct" adds the Channel Transformer (4 channel
    groups after each spatial step: s x N = 16 steps per frame, the paper's
    configuration), with its own weights."""
    import torch
    from paper_2605_20977_gb300 import psw, synth
    cfg = synth.config(name)
    if cfg.Nc:
        w = synth.weights(cfg)
    ctx = psw.Context(cfg, w, precision=psw.PSW_BF16)
    fd = psw.frame_desc(cfg.H, cfg.W, psw.PSW_SCHED_WAVEFRONT)
    cap = ctx.bitstream_capacity(cfg.H, cfg.W)
    enc = ctx.seq_create(cfg.H, cfg.W)
    bss, lens = [], []
    for b in range(B):
        enc.reset()
        bs = torch.zeros(cap, dtype=torch.uint8, device=dev)
        lens.append(enc.encode_params(fd, ys[b], zs[b], bitstream=bs))
        bss.append(bs)
    enc.close()
    decs = [ctx.seq_create(cfg.H, cfg.W) for _ in range(B)]
    outs = [torch.zeros_like(y) for y in ys]

    def step(n):
        for q in decs[:n]:
            q.reset()
        ctx.decode_batch(decs[:n], [fd] * n, bss[:n], lens[:n], zs[:n], outs[:n])

    step(B)                                     # records the graphs
    ms = timed(lambda: step(B), args.cyclic_steps)
    for b in range(B):
        if not torch.equal(outs[b], ys[b]):
            raise RuntimeError("cyclic decode differs")
    step(1)
    lat = timed(lambda: step(1), max(2, args.cyclic_steps))
    ctx.profile_begin()
    step(B)
    stats = ctx.profile_end()
    pk, pk_kind = peaks()
    g = next((s_ for s_ in stats if s_["name"] == "gemm_tc"), None)
    nrm = next((s_ for s_ in stats if s_["name"] == "rmsnorm"), None)
    out = {"value": B * 1e3 / float(np.mean(ms)), "unit": "frames/s", "frames_per_step": B,
           "ms_per_step": float(np.mean(ms)), "steps_per_frame": 4 * max(cfg.Nc, 1),
           "latency_one_frame": {"ms_per_frame": float(np.mean(lat)), "frames_per_s": 1e3 / float(np.mean(lat))},
           "workload": ("1080p I-frames 68x120x192 with the cyclic s = 4 mask (Fig. 2a), same model sizes and "
                        "frames as the headline, BF16") + (
                           f"; Channel Transformer with N = {cfg.Nc} groups, width {cfg.dc}, {cfg.Lct} blocks "
                           f"(16 autoregressive steps per frame)" if cfg.Nc else ""),
           "classes": {s_["name"]: {"ms": round(s_["ms"], 3), "launches": s_["launches"],
                                    "gflop": round(s_["flops"] / 1e9, 2)} for s_ in stats}}
    if g:
        t = g["ms"] + (nrm["ms"] if nrm else 0.0)
        ach = g["flops"] / (t / 1e3) / 1e12
        out["projections"] = {"achieved": ach, "unit": "TFLOP/s", "peak": pk["bf16_tflops_sustained"],
                              "frac": ach / pk["bf16_tflops_sustained"],
                              "timing": "CUDA events, projection launches plus the row normalisations feeding them",
                              "tokens_per_launch": B * 2040}
    for q in decs:
        q.close()
    ctx.close()
    return out


def job_rate(units_per_rank, local_seconds, world, device):
    """Whole-job throughput of `world` replicas: every rank's units over the
    slowest rank's time (all-reduce MAX).  Returns (units / s, max seconds)."""
    import torch
    t = torch.tensor([float(local_seconds)], device=device, dtype=torch.float64)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return world * units_per_rank / float(t.item()), float(t.item())


def replica_seed(rank: int, frames_per_rank: int, b: int) -> int:
    """Seed of frame b of a rank's batch: replicas decode distinct frames."""
    return 1002 + rank * frames_per_rank + b


def run_ours(args, rank: int, world: int, local: int):
    import torch
    import torch.distributed as dist
    from paper_2605_20977_gb300 import build, psw, synth

    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    cfg = synth.config("i1080")
    w = synth.weights(cfg)
    ctx = psw.Context(cfg, w, precision=psw.PSW_FP8 if args.precision == "fp8" else psw.PSW_BF16)
    ctx.set_engine({"auto": psw.ENGINE_AUTO, "graph": psw.ENGINE_GRAPH,
                    "persistent": psw.ENGINE_PERSISTENT}[args.engine])
    B = args.batch
    fdw = psw.frame_desc(cfg.H, cfg.W, psw.PSW_SCHED_WAVEFRONT)
    fdr = psw.frame_desc(cfg.H, cfg.W, psw.PSW_SCHED_RASTER)
    frames = [synth.frames(cfg, 1, seed=replica_seed(rank, B, b)) for b in range(B)]
    ys = [torch.from_numpy(f.y[0]).to(dev) for f in frames]
    zs = [torch.from_numpy(f.z[0]).to(dev) for f in frames]
    cap = ctx.bitstream_capacity(cfg.H, cfg.W)
    enc = ctx.seq_create(cfg.H, cfg.W)

    def encode(fd, n=B):
        bss, lens = [], []
        for b in range(n):
            enc.reset()
            bs = torch.zeros(cap, dtype=torch.uint8, device=dev)
            lens.append(enc.encode_params(fd, ys[b], zs[b], bitstream=bs))
            bss.append(bs)
        return bss, lens

    bss, lens = encode(fdw)
    mu0 = torch.zeros(ys[0].shape, dtype=torch.float32, device=dev); sg0 = torch.zeros_like(mu0)
    enc.reset()
    enc.encode_params(fdw, ys[0], zs[0], mu0, sg0)
    decs = [ctx.seq_create(cfg.H, cfg.W) for _ in range(B)]
    outs = [torch.zeros_like(y) for y in ys]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def batch_step(seqs, fd, bs_, ln_, n):
        for q in seqs[:n]:
            q.reset()
        ctx.decode_batch(seqs[:n], [fd] * n, bs_[:n], ln_[:n], zs[:n], outs[:n])

    def timed(fn, reps):
        ms = []
        for k in range(reps):
            flush.fill_(k & 0xFF)                   # evict L2 between steps
            a = torch.cuda.Event(enable_timing=True); b_ = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b_.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b_))
        return ms

    for _ in range(args.warmup):
        batch_step(decs, fdw, bss, lens, B)
    torch.cuda.synchronize()
    # the autotuner picks the projection tile widths on this very step
    tuned = None
    if args.tune:
        from paper_2605_20977_gb300 import workloads
        tuned = workloads.tune_tiles(ctx, lambda: batch_step(decs, fdw, bss, lens, B))
        batch_step(decs, fdw, bss, lens, B)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    l0 = ctx.launch_count()
    step_ms = timed(lambda: batch_step(decs, fdw, bss, lens, B), args.steps)
    launches = (ctx.launch_count() - l0) / args.steps
    engine = ctx.last_engine()
    clk = clocks.stop()
    for b in range(B):
        if not torch.equal(outs[b], ys[b]):
            raise RuntimeError("decoded latents differ from the encoded ones")
    value, total_max = job_rate(B * args.steps, sum(step_ms) / 1e3, world, dev)

    # single-frame latency (one frame per call)
    lat = None
    if B > 1:
        batch_step(decs, fdw, bss, lens, 1)
        lat_ms = timed(lambda: batch_step(decs, fdw, bss, lens, 1), max(2, args.steps))
        lat = {"ms_per_frame": float(np.mean(lat_ms)), "frames_per_s": 1e3 / float(np.mean(lat_ms))}

    # end to end through the C ABI with pinned host buffers: every step copies
    # its containers and hyperlatents in and its latents out; the copies run
    # on a second stream, double-buffered, so step k+1's inputs go in and step
    # k's latents come out while a decode runs (the host waits for each
    # decode).  The frames' containers, hyperlatents and latents each sit in
    # one contiguous buffer per side, so a step's copies are three transfers
    # (the library takes a pointer per frame into them)
    boff = [0]
    for b in range(B):
        boff.append(boff[-1] + (int(lens[b]) + 255) // 256 * 256)
    h_bs_all = torch.zeros(boff[-1], dtype=torch.uint8).pin_memory()
    for b in range(B):
        h_bs_all[boff[b]:boff[b] + lens[b]].copy_(bss[b][:lens[b]].cpu())
    h_z_all = torch.stack([z.cpu() for z in zs]).pin_memory()
    h_y_all = torch.empty((B,) + tuple(ys[0].shape), dtype=torch.int16).pin_memory()
    h_y = [h_y_all[b] for b in range(B)]
    d_bs_all = [torch.zeros(boff[-1], dtype=torch.uint8, device=dev) for _ in range(2)]
    d_z_all = [torch.zeros_like(h_z_all, device=dev) for _ in range(2)]
    d_y_all = [torch.zeros((B,) + tuple(ys[0].shape), dtype=torch.int16, device=dev) for _ in range(2)]
    d_bs = [[d_bs_all[k][boff[b]:boff[b] + lens[b]] for b in range(B)] for k in range(2)]
    d_z = [[d_z_all[k][b] for b in range(B)] for k in range(2)]
    d_y = [[d_y_all[k][b] for b in range(B)] for k in range(2)]
    cstream = torch.cuda.Stream(device=dev)
    in_ready = [torch.cuda.Event(), torch.cuda.Event()]
    dec_done = [torch.cuda.Event(), torch.cuda.Event()]

    def copy_in(k):
        with torch.cuda.stream(cstream):
            d_bs_all[k].copy_(h_bs_all, non_blocking=True)
            d_z_all[k].copy_(h_z_all, non_blocking=True)
            in_ready[k].record(cstream)

    def e2e_run(n):
        copy_in(0)
        for k in range(n):
            cur = k & 1
            if k + 1 < n:
                copy_in(cur ^ 1)                    # the previous decode that read this set has finished
            stream.wait_event(in_ready[cur])
            for q in decs:
                q.reset()
            ctx.decode_batch(decs, [fdw] * B, d_bs[cur], lens, d_z[cur], d_y[cur], stream=stream)
            dec_done[cur].record(stream)
            with torch.cuda.stream(cstream):
                cstream.wait_event(dec_done[cur])
                h_y_all.copy_(d_y_all[cur], non_blocking=True)
        stream.wait_stream(cstream)

    e2e_run(2)
    flush.fill_(1)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    for b in range(B):
        if not torch.equal(h_y[b], ys[b].cpu()):
            raise RuntimeError("end-to-end decode differs")
    e2e_value, _ = job_rate(B * args.steps, e0.elapsed_time(e1) / 1e3, world, dev)
    h2d = h_bs_all.numel() + h_z_all.numel() * 2
    d2h = h_y_all.numel() * 2

    # roofline of the dominant kernel class from CUDA events (one
    # instrumented step with direct launches, after the timed region)
    flush.fill_(2)
    ctx.profile_begin()
    batch_step(decs, fdw, bss, lens, B)
    stats = ctx.profile_end()
    pk, pk_kind = peaks()
    dom = max(stats, key=lambda s: s["ms"])
    tot_ms = sum(s["ms"] for s in stats)
    nrm = next((s for s in stats if s["name"] == "rmsnorm"), None)
    if dom["name"].startswith("gemm"):
        # the projections' time includes the row normalisations that feed
        # their wide launches (the operand a tile would otherwise build)
        dom_ms = dom["ms"] + (nrm["ms"] if nrm and dom["name"] == "gemm_tc" else 0.0)
        achieved = dom["flops"] / (dom_ms / 1e3) / 1e12
        peak, unit, bound = pk["bf16_tflops_sustained"], "TFLOP/s", "tensor"
    else:
        achieved = dom["bytes"] / (dom["ms"] / 1e3) / 1e9
        peak, unit, bound = pk["hbm_gbs"], "GB/s", "hbm"
    if dom["name"] == "persistent":
        # the whole wavefront walk is one kernel: its algorithmic FLOPs
        # (projections and attention of every position) over its duration
        achieved = dom["flops"] / (dom["ms"] / 1e3) / 1e12
        peak, unit, bound = pk["bf16_tflops_sustained"], "TFLOP/s", "tensor"
    kname = {"gemm_tc": "k_gemm_ws", "attention": "k_attention", "heads": "k_heads", "rmsnorm": "k_rmsnorm",
             "rans": "k_rans_dec_step", "embed": "k_embed_latent", "gemm_simt": "k_gemm_simt",
             "persistent": "k_persist"}.get(dom["name"])
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
            "traffic": traffic_for(kname), "kernel": dom["name"], "launches_per_step": dom["launches"],
            "avg_launch_us": 1e3 * dom["ms"] / max(dom["launches"], 1),
            "share_of_kernel_time": dom["ms"] / tot_ms,
            "peak_source": ("measured, MEASURED_PEAKS.json (sustained bf16 for a kernel inside a long step)"
                            if pk_kind == "measured" else "fallback"),
            "timing": ("CUDA events around each launch of one instrumented step (direct launches, same engine); "
                       "projection time includes the row normalisations feeding the wide launches"),
            "classes": {s["name"]: {"ms": round(s["ms"], 3), "launches": s["launches"],
                                    "gflop": round(s["flops"] / 1e9, 2)} for s in stats}}

    # raster order, same model and masks, same GPU, same launch mechanism
    raster = None
    if rank == 0 and args.raster_frames > 0:
        RB = min(B, args.raster_batch_size)
        rbss, rlens = encode(fdr, RB)
        rdecs = [ctx.seq_create(cfg.H, cfg.W) for _ in range(RB)]
        raster = {}
        sizes = [1] + ([RB] if RB > 1 and args.raster_batch else [])
        for n in sizes:
            batch_step(rdecs, fdr, rbss, rlens, n)          # captures the graph segments
            r_ms = timed(lambda: batch_step(rdecs, fdr, rbss, rlens, n), args.raster_frames)
            for b in range(n):
                if not torch.equal(outs[b], ys[b]):
                    raise RuntimeError("raster decode differs")
            raster[f"frames_per_step_{n}"] = {"value": n * 1e3 / float(np.mean(r_ms)), "unit": "frames/s",
                                              "ms_per_step": float(np.mean(r_ms)), "steps_per_frame": cfg.H * cfg.W}
    speedup = None
    if raster:
        speedup = {}
        if lat is not None or B == 1:
            w1 = lat["frames_per_s"] if lat else value / world
            speedup["frames_per_step_1"] = w1 / raster["frames_per_step_1"]["value"]
        RB = min(B, args.raster_batch_size)
        if f"frames_per_step_{RB}" in raster and RB > 1:
            if RB == B:
                wv = value / world
            else:
                # the wavefront at the raster comparison's batch size
                batch_step(decs, fdw, bss, lens, RB)
                w_ms = timed(lambda: batch_step(decs, fdw, bss, lens, RB), max(2, args.steps))
                wv = RB * 1e3 / float(np.mean(w_ms))
                raster[f"wavefront_frames_per_step_{RB}"] = {"value": wv, "unit": "frames/s"}
            speedup[f"frames_per_step_{RB}"] = wv / raster[f"frames_per_step_{RB}"]["value"]
        for q in rdecs:
            q.close()
    # the legs below hold their own contexts and sequences: the main leg's
    # decoder caches (about 270 MB per 1080p frame) go first
    for q in decs:
        q.close()
    torch.cuda.empty_cache()

    # P-frame GOPs (temporal model, 1080p): frame f of every sequence per
    # call; every sequence's frames in order
    pframe = None
    if rank == 0 and args.pframe_seqs > 0:
        pframe = pframe_run(args, dev, stream, flush, timed)

    fp8 = mu8 = sg8 = None
    if rank == 0 and args.fp8_steps > 0 and args.precision == "bf16":
        fp8, mu8, sg8 = fp8_run(args, dev, timed, cfg, w, ys, zs, B)

    # the paper's own cyclic s = 4 schedule on the same frames
    cyclic = None
    if rank == 0 and args.cyclic_steps > 0 and args.precision == "bf16":
        cyclic = cyclic_run(args, dev, timed, w, ys, zs, B)

    # the paper's configuration: cyclic s = 4 plus the Channel Transformer
    cyclic_ct = None
    if rank == 0 and args.cyclic_steps > 0 and args.precision == "bf16":
        cyclic_ct = cyclic_run(args, dev, timed, w, ys, zs, B, name="i1080_cyc_ct")

    # the convolutional hyperprior
    hyper = None
    if rank == 0 and args.hyper_steps > 0 and args.precision == "bf16":
        hyper = hyper_run(args, dev, timed, ys, min(B, 16))

    # batched uneven: four grids of P-frame sequences per call, autotuned plan
    mixed = None
    if rank == 0 and args.mixed_frames > 0 and args.precision == "bf16":
        from paper_2605_20977_gb300 import workloads
        mixed = workloads.run_mixed(32, args.mixed_frames, dev=dev, precision="bf16")

    # serving: continuous batching under Poisson arrivals, a sweep of rates
    serving = None
    if rank == 0 and args.serve_rates.strip() and args.precision == "bf16":
        from paper_2605_20977_gb300 import workloads
        sweep = []
        for lam in [float(x) for x in args.serve_rates.split(",") if x.strip()]:
            st = workloads.run_serve(rate=lam, window=args.serve_window, dev=dev, unbatched=False, precision="bf16")
            b = st["batched"]
            offered = b["frames"] / args.serve_window
            sweep.append({"rate_per_s": lam, "offered_frames_per_s": offered, "served_frames_per_s": b["frames_per_s"],
                          "latency_p50_s": b["latency_p50_s"], "latency_p99_s": b["latency_p99_s"],
                          "requests": b["requests"], "frames": b["frames"], "mean_batch": b["mean_batch"]})
        # the knee: the highest rate whose p99 latency stays within 1.5 x that
        # of the lowest rate (requests of up to 16 frames of a 135 x 240 grid
        # set the latency floor)
        p0 = sweep[0]["latency_p99_s"] if sweep else 0.0
        ok = [x["rate_per_s"] for x in sweep if x["latency_p99_s"] <= 1.5 * p0]
        serving = {"workload": f"P-frame requests of 1..16 frames at the grids 15x26, 30x52, 68x120, 135x240, "
                               f"Poisson arrivals over {args.serve_window:g} s, continuous batching, BF16, graph engine",
                   "sweep": sweep, "knee_rate_per_s": max(ok) if ok else None}

    # the LRP Transformer over one coded frame
    lrp = None
    if rank == 0 and args.lrp_steps > 0 and args.precision == "bf16":
        lrp = lrp_run(args, dev, timed, ys, zs)

    # rate: GPU parameters vs the FP64 oracle on the sample rows
    rate = {"bits_per_symbol": ctx.rate(ys[0], mu0, sg0) / ys[0].numel(),
            "container_bits_per_symbol": 8.0 * lens[0] / ys[0].numel()}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        smp = OracleSample(args.cpu_rows)
        secs = smp.time_decode()
        frac = smp.npos / (cfg.H * cfg.W)
        cpu = {"value": frac / secs, "unit": "frames/s", "cores": smp.threads, "kind": "oracle",
               "sample": smp.describe(secs)}
        one = oracle_single_thread(1)
        if one:
            cpu["single_thread"] = {"value": one[0], "unit": "frames/s", "cores": 1, "sample": one[1]}
        R = args.cpu_rows
        r_gpu = smp.O.rate_bits(smp.y[0], mu0[:R].double().cpu().numpy(), sg0[:R].double().cpu().numpy())
        r_64 = smp.O.rate_bits(smp.y[0], smp.mu, smp.sg)
        rate["delta_vs_fp64_on_sample"] = abs(r_gpu - r_64) / r_64
        if fp8 is not None:
            # FP8 against the FP64 oracle with the weights the FP8 context
            # holds (E4M3 block projections, bf16 embedding and heads)
            mu_q, sg_q = smp.fp8_params()
            r8 = smp.O.rate_bits(smp.y[0], mu8[:R].double().cpu().numpy(), sg8[:R].double().cpu().numpy())
            r8_64 = smp.O.rate_bits(smp.y[0], mu_q, sg_q)
            fp8["rate_delta_vs_fp64_on_sample"] = abs(r8 - r8_64) / r8_64

    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if args.precision == "bf16" else "e4m3+bf16",
            "data": "synthetic",
            "config": arm_config(args, world, engine),
            "e2e": {"value": e2e_value, "unit": "frames/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(round(launches)),
            "latency_one_frame": lat,
            "roofline": roof, "raster": raster, "speedup_vs_raster": speedup,
            "rate": rate, "clocks": clk, "cpu_baseline": cpu, "pframe": pframe, "fp8": fp8, "cyclic": cyclic,
            "cyclic_channel_groups": cyclic_ct, "lrp": lrp, "hyperprior": hyper,
            "batched_uneven": mixed, "serving": serving, "tile_autotune": tuned}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    try:
        return run_ours(args, rank, world, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
