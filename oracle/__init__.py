"""FP64 CPU oracle for the P-SWA context model -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never does; it shares no code with this package.

The arithmetic lives in ``psw_oracle.c`` (plain loops, double precision,
``-ffp-contract=off``); this module builds it with gcc and wraps it with
ctypes.  Functions take and return numpy arrays.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "psw_oracle.c")
_LIB = os.path.join(_HERE, "libpsw_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                        "-shared", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Cfg(ct.Structure):
    _fields_ = [(n, ct.c_int) for n in
                ("H", "W", "C", "Hh", "Wh", "Ch", "r", "d", "nh", "F", "L", "k",
                 "temporal", "Lc", "Tf", "mask", "Llrp", "Nc", "dc", "Lct", "Fc", "hp")]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ct.CDLL(build())
            P = ct.c_void_p
            lib.or_weights_count.argtypes = [ct.POINTER(_Cfg)]
            lib.or_weights_count.restype = ct.c_long
            lib.or_rmsnorm.argtypes = [P, P, ct.c_int, P]
            lib.or_matvec.argtypes = [P, P, ct.c_int, ct.c_int, P]
            lib.or_silu.argtypes = [ct.c_double]
            lib.or_silu.restype = ct.c_double
            lib.or_swiglu.argtypes = [P, P, P, P, ct.c_int, ct.c_int, P]
            lib.or_attend.argtypes = [P, ct.c_int, P, P, P, ct.c_int, ct.c_int, P]
            lib.or_label.argtypes = [ct.c_int, ct.c_int, ct.c_int]
            lib.or_visible.argtypes = [ct.c_int] * 7
            lib.or_window_keys.argtypes = [ct.POINTER(_Cfg), ct.c_int, ct.c_int, P, P]
            lib.or_schedule.argtypes = [ct.POINTER(_Cfg), ct.c_int, P, P]
            lib.or_e4m3.argtypes = [ct.c_double]
            lib.or_e4m3.restype = ct.c_double
            lib.or_e4m3_tensor.argtypes = [ct.c_long, P, P]
            lib.or_e4m3_tensor.restype = ct.c_double
            lib.or_scale_table.argtypes = [P]
            lib.or_quantize.argtypes = [ct.c_long, P, P, P, P]
            lib.or_cdf_T.argtypes = [ct.c_int]
            lib.or_cdf_freq.argtypes = [ct.c_int, P]
            lib.or_likelihood.argtypes = [ct.c_double] * 3
            lib.or_likelihood.restype = ct.c_double
            lib.or_rate_bits.argtypes = [ct.c_long, P, P, P]
            lib.or_rate_bits.restype = ct.c_double
            lib.or_rans_encode.argtypes = [ct.c_int] * 4 + [P, P, P, P, P, ct.c_long]
            lib.or_rans_encode.restype = ct.c_long
            lib.or_rans_decode.argtypes = [ct.c_int] * 4 + [P, P, ct.c_int, P, P, P, ct.c_long, P]
            lib.or_run.argtypes = [ct.POINTER(_Cfg), P, ct.c_int, P, P, ct.c_int, ct.c_int, P, P, P, P]
            lib.or_run_lrp.argtypes = [ct.POINTER(_Cfg), P, ct.c_int, P, P, ct.c_int, ct.c_int, P, P, P, P, P]
            lib.or_num_threads.restype = ct.c_int
            lib.or_hyper_analysis.argtypes = [ct.POINTER(_Cfg), P, ct.c_int, P, P, P]
            lib.or_hyper_encode.argtypes = [ct.POINTER(_Cfg), P, P, P, ct.c_long]
            lib.or_hyper_encode.restype = ct.c_long
            lib.or_hyper_decode.argtypes = [ct.POINTER(_Cfg), P, P, ct.c_long, P]
            lib.or_prior_freq.argtypes = [ct.POINTER(_Cfg), P, ct.c_int, P]
            lib.or_hyper_rate.argtypes = [ct.POINTER(_Cfg), P, P]
            lib.or_hyper_rate.restype = ct.c_double
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ct.c_void_p)


def _cfg(c) -> _Cfg:
    d = c if isinstance(c, dict) else c.as_dict()
    return _Cfg(**{k: int(d.get(k, 0)) for k, _ in _Cfg._fields_})


def num_threads() -> int:
    return int(_load().or_num_threads())


# ---------------------------------------------------------------- elementary

def weights_count(c) -> int:
    return int(_load().or_weights_count(ct.byref(_cfg(c))))


def rmsnorm(x, g):
    x = np.ascontiguousarray(x, np.float64); g = np.ascontiguousarray(g, np.float64)
    y = np.zeros_like(x)
    _load().or_rmsnorm(_p(x), _p(g), x.size, _p(y))
    return y


def matvec(x, W):
    x = np.ascontiguousarray(x, np.float64); W = np.ascontiguousarray(W, np.float64)
    y = np.zeros(W.shape[1])
    _load().or_matvec(_p(x), _p(W), W.shape[0], W.shape[1], _p(y))
    return y


def silu(v: float) -> float:
    return float(_load().or_silu(float(v)))


def swiglu(x, Wg, Wu, Wd):
    x, Wg, Wu, Wd = (np.ascontiguousarray(a, np.float64) for a in (x, Wg, Wu, Wd))
    out = np.zeros(Wd.shape[1])
    _load().or_swiglu(_p(x), _p(Wg), _p(Wu), _p(Wd), Wg.shape[0], Wg.shape[1], _p(out))
    return out


def attend(q, K, V, bias, nh):
    """q: [d]; K, V: [n][d]; bias: [n][nh]."""
    q = np.ascontiguousarray(q, np.float64)
    K = np.ascontiguousarray(K, np.float64).reshape(-1, q.size)
    V = np.ascontiguousarray(V, np.float64).reshape(-1, q.size)
    bias = np.ascontiguousarray(bias, np.float64).reshape(-1, nh)
    n = K.shape[0]
    kp = (ct.c_void_p * max(n, 1))(*[K[j].ctypes.data for j in range(n)])
    vp = (ct.c_void_p * max(n, 1))(*[V[j].ctypes.data for j in range(n)])
    out = np.zeros(q.size)
    _load().or_attend(_p(q), n, kp, vp, _p(bias), nh, q.size, _p(out))
    return out


def label(mask: int, i: int, j: int) -> int:
    return int(_load().or_label(mask, i, j))


def visible(mask: int, kind: int, W: int, pi: int, pj: int, qi: int, qj: int) -> bool:
    return bool(_load().or_visible(mask, kind, W, pi, pj, qi, qj))


def window_keys(c, kind: int, p: int):
    idx = np.zeros(c.k * c.k, np.int32); off = np.zeros(c.k * c.k, np.int32)
    n = _load().or_window_keys(ct.byref(_cfg(c)), kind, p, _p(idx), _p(off))
    return idx[:n].copy(), off[:n].copy()


def schedule(c, kind: int):
    """(order, start): positions in schedule order and step boundaries."""
    HW = c.H * c.W
    order = np.zeros(HW, np.int32); start = np.zeros(HW + 1, np.int32)
    T = _load().or_schedule(ct.byref(_cfg(c)), kind, _p(order), _p(start))
    return order, start[:T + 1].copy()


# ---------------------------------------------------------------- E4M3

def e4m3(x: float) -> float:
    """Nearest E4M3 value of x (ties to even, saturating at 448)."""
    return float(_load().or_e4m3(float(x)))


def e4m3_tensor(x):
    """(dequantised values, scale) of one tensor quantised as the FP8
    weights: a power-of-two scale s putting max |x| / s in [128, 256)."""
    x = np.ascontiguousarray(x, np.float64)
    out = np.zeros_like(x)
    s = _load().or_e4m3_tensor(x.size, _p(x), _p(out))
    return out, float(s)


# ---------------------------------------------------------------- coding

def scale_table() -> np.ndarray:
    t = np.zeros(64, np.float32)
    _load().or_scale_table(_p(t))
    return t


def quantize(mu, sigma):
    """FP32 (mu, sigma) -> (scale index uint8, rounded mean int32)."""
    mu = np.ascontiguousarray(mu, np.float32); sigma = np.ascontiguousarray(sigma, np.float32)
    idx = np.zeros(mu.shape, np.uint8); m = np.zeros(mu.shape, np.int32)
    _load().or_quantize(mu.size, _p(mu), _p(sigma), _p(idx), _p(m))
    return idx, m


def cdf_T(l: int) -> int:
    return int(_load().or_cdf_T(l))


def cdf_freq(l: int) -> np.ndarray:
    f = np.zeros(4096, np.uint32)
    n = _load().or_cdf_freq(l, _p(f))
    return f[:n].copy()


def likelihood(y: float, mu: float, sigma: float) -> float:
    return float(_load().or_likelihood(float(y), float(mu), float(sigma)))


def rate_bits(y, mu, sigma) -> float:
    y = np.ascontiguousarray(y, np.int16)
    mu = np.ascontiguousarray(mu, np.float64); sigma = np.ascontiguousarray(sigma, np.float64)
    return float(_load().or_rate_bits(y.size, _p(y), _p(mu), _p(sigma)))


def rans_encode(c, sched: int, y, idx, m, cap: int | None = None) -> bytes:
    """Container for one frame; y, idx, m: [H][W][C]."""
    order, _ = schedule(c, sched)
    y = np.ascontiguousarray(y, np.int16); idx = np.ascontiguousarray(idx, np.uint8)
    m = np.ascontiguousarray(m, np.int32)
    cap = cap or (16 + 4 * (c.C + 1) + c.C * (132 + 6 * c.H * c.W))
    out = np.zeros(cap, np.uint8)
    n = _load().or_rans_encode(c.H, c.W, c.C, sched, _p(order), _p(y), _p(idx), _p(m), _p(out), cap)
    if n < 0:
        raise ValueError(f"rans_encode failed ({n})")
    return out[:n].tobytes()


def rans_decode(c, sched: int, idx, m, bs: bytes):
    """Coder-only decode with known (idx, m); returns (ok, y)."""
    order, start = schedule(c, sched)
    idx = np.ascontiguousarray(idx, np.uint8); m = np.ascontiguousarray(m, np.int32)
    buf = np.frombuffer(bs, np.uint8).copy()
    y = np.zeros((c.H, c.W, c.C), np.int16)
    rc = _load().or_rans_decode(c.H, c.W, c.C, sched, _p(order), _p(start), len(start) - 1,
                                _p(idx), _p(m), _p(buf), len(buf), _p(y))
    return rc == 0, y


# ---------------------------------------------------------------- hyperprior

def hyper_analysis(c, w, y):
    """(z-hat int16, z float64) [nf][Hh][Wh][Ch] of a convolutional
    hyperprior model from the frames' latents y [nf][H][W][C]."""
    w = np.ascontiguousarray(w, np.float64)
    y = np.ascontiguousarray(y, np.int16)
    nf = y.shape[0]
    zh = np.zeros((nf, c.Hh, c.Wh, c.Ch), np.int16)
    z = np.zeros(zh.shape, np.float64)
    if _load().or_hyper_analysis(ct.byref(_cfg(c)), _p(w), nf, _p(y), _p(zh), _p(z)) != 0:
        raise ValueError("hyper_analysis failed")
    return zh, z


def hyper_encode(c, w, zhat, cap: int | None = None) -> bytes:
    """z-hat container of one frame ([Hh][Wh][Ch]) under the factorized prior."""
    w = np.ascontiguousarray(w, np.float64)
    zhat = np.ascontiguousarray(zhat, np.int16)
    cap = cap or (16 + 4 * (c.Ch + 1) + c.Ch * (132 + 6 * c.Hh * c.Wh))
    out = np.zeros(cap, np.uint8)
    n = _load().or_hyper_encode(ct.byref(_cfg(c)), _p(w), _p(zhat), _p(out), cap)
    if n < 0:
        raise ValueError(f"hyper_encode failed ({n})")
    return out[:n].tobytes()


def hyper_decode(c, w, bs: bytes):
    """(ok, z-hat [Hh][Wh][Ch]) from a z-hat container."""
    w = np.ascontiguousarray(w, np.float64)
    buf = np.frombuffer(bs, np.uint8).copy()
    zh = np.zeros((c.Hh, c.Wh, c.Ch), np.int16)
    rc = _load().or_hyper_decode(ct.byref(_cfg(c)), _p(w), _p(buf), len(buf), _p(zh))
    return rc == 0, zh


def prior_freq(c, w, ch: int) -> np.ndarray:
    """Integer frequency table of channel ch of the factorized prior."""
    w = np.ascontiguousarray(w, np.float64)
    f = np.zeros(4096, np.uint32)
    n = _load().or_prior_freq(ct.byref(_cfg(c)), _p(w), ch, _p(f))
    return f[:n].copy()


def hyper_rate(c, w, zhat) -> float:
    w = np.ascontiguousarray(w, np.float64)
    zhat = np.ascontiguousarray(zhat, np.int16)
    return float(_load().or_hyper_rate(ct.byref(_cfg(c)), _p(w), _p(zhat)))


# ---------------------------------------------------------------- model

def run(c, w, y, z, driver: int = 0, sched: int = 0, bitstreams=None, with_eps: bool = False):
    """Run the context model over a sequence (see or_run in psw_oracle.c).

    w: flat weights (float64 copy made); y: [nf][H][W][C] int16 (for driver 2
    it receives the decoded latents); z: [nf][Hh][Wh][Ch] int16.
    Returns (mu, sigma) float64 [nf][H][W][C], and with with_eps (a model
    with an LRP Transformer) also each frame's residual eps (or_run_lrp)."""
    w = np.ascontiguousarray(w, np.float64)
    if w.size != weights_count(c):
        raise ValueError(f"weights: {w.size} != {weights_count(c)}")
    y = np.ascontiguousarray(y, np.int16); z = np.ascontiguousarray(z, np.int16)
    nf = y.shape[0]
    mu = np.zeros(y.shape, np.float64); sg = np.zeros(y.shape, np.float64)
    bsp, lens, keep = None, None, []
    if driver == 2:
        bufs = [np.frombuffer(b, np.uint8).copy() for b in bitstreams]
        keep = bufs
        bsp = (ct.c_void_p * nf)(*[b.ctypes.data for b in bufs])
        lens = np.array([len(b) for b in bufs], np.int64)
    eps = np.zeros(y.shape, np.float64) if with_eps else None
    rc = _load().or_run_lrp(ct.byref(_cfg(c)), _p(w), nf, _p(y), _p(z), driver, sched,
                            bsp, _p(lens) if lens is not None else None, _p(mu), _p(sg),
                            _p(eps) if with_eps else None)
    del keep
    if rc == -2:
        raise ValueError("corrupt bitstream")
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return (mu, sg, eps) if with_eps else (mu, sg)


def encode_frames(c, w, y, z, sched: int = 0):
    """Oracle encoder: masked parallel pass, float rounding, quantisation,
    rANS.  Returns (bitstreams, mu, sigma)."""
    mu, sg = run(c, w, y, z, driver=0)
    out = []
    for f in range(y.shape[0]):
        idx, m = quantize(mu[f].astype(np.float32), sg[f].astype(np.float32))
        out.append(rans_encode(c, sched, y[f], idx, m))
    return out, mu, sg


def decode_frames(c, w, bitstreams, z, sched: int = 0):
    """Oracle decoder: schedule-driven decode of the bitstreams.
    Returns (y, mu, sigma)."""
    nf = len(bitstreams)
    y = np.zeros((nf, c.H, c.W, c.C), np.int16)
    mu, sg = run(c, w, y, z, driver=2, sched=sched, bitstreams=bitstreams)
    return y, mu, sg
