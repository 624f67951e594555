"""Python binding of the C ABI in include/psw.h (ctypes; marshalling only).

Every function here forwards to the CUDA library libpsw.so under the same
name; all computation runs in its kernels.  PyTorch supplies device memory
and streams.  There is no fallback: if the library cannot be loaded, or no
CUDA device is present, calls raise.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpsw.so")

PSW_OK, PSW_ERR_INVALID, PSW_ERR_OOM, PSW_ERR_CUDA, PSW_ERR_CORRUPT, PSW_ERR_TIMEOUT, PSW_ERR_CAPACITY = range(7)
PSW_FP32, PSW_BF16, PSW_FP8 = 0, 1, 2
PSW_SCHED_WAVEFRONT, PSW_SCHED_RASTER = 0, 1
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "OOM", 3: "CUDA", 4: "CORRUPT", 5: "TIMEOUT", 6: "CAPACITY"}

EXPORTS = ["psw_weights_count", "psw_create", "psw_destroy", "psw_last_error", "psw_ctx_bytes", "psw_seq_bytes",
           "psw_seq_create", "psw_seq_reset", "psw_seq_destroy", "psw_bitstream_capacity", "psw_encode_params",
           "psw_decode_frame", "psw_decode_batch", "psw_rate", "psw_quantize", "psw_scale_table", "psw_cdf_table",
           "psw_rans_encode", "psw_rans_decode", "psw_launch_count", "psw_profile_begin", "psw_profile_end",
           "psw_rans_encode_noalloc", "psw_set_engine", "psw_last_engine", "psw_quantize_e4m3",
           "psw_check_wait_timeout", "psw_lrp_residual", "psw_hyper_encode", "psw_hyper_decode",
           "psw_prior_table", "psw_set_tile_policy", "psw_tile_policy"]
TILE_QKV, TILE_RESIDUAL, TILE_SWIGLU, TILE_OTHER = 0, 1, 2, 3

ENGINE_AUTO, ENGINE_GRAPH, ENGINE_PERSISTENT = 0, 1, 2


class ModelDesc(ct.Structure):
    _fields_ = [(n, ct.c_int) for n in ("C", "Ch", "r", "d", "nh", "F", "L", "k", "temporal", "Lc", "Tf", "mask",
                                         "Llrp", "Nc", "dc", "Lct", "Fc", "hp")]


class FrameDesc(ct.Structure):
    _fields_ = [("H", ct.c_int), ("W", ct.c_int), ("schedule", ct.c_int)]


class KernelStat(ct.Structure):
    _fields_ = [("name", ct.c_char * 32), ("launches", ct.c_long), ("ms", ct.c_double), ("flops", ct.c_double),
                ("bytes", ct.c_double)]


class PswError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libpsw.so (built by paper_2605_20977_gb300.build) and declare
    its signatures.  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with paper_2605_20977_gb300.build.build()")
        lib = ct.CDLL(path)
        P, S, I = ct.c_void_p, ct.c_size_t, ct.c_int
        MD, FD = ct.POINTER(ModelDesc), ct.POINTER(FrameDesc)
        sig = {
            "psw_weights_count": (S, [MD]),
            "psw_create": (I, [MD, P, S, I, S, ct.POINTER(P)]),
            "psw_destroy": (None, [P]),
            "psw_last_error": (ct.c_char_p, [P]),
            "psw_ctx_bytes": (S, [P]),
            "psw_seq_bytes": (S, [P, I, I]),
            "psw_seq_create": (I, [P, I, I, ct.POINTER(P)]),
            "psw_seq_reset": (I, [P]),
            "psw_seq_destroy": (None, [P]),
            "psw_bitstream_capacity": (S, [P, FD]),
            "psw_encode_params": (I, [P, P, FD, P, P, P, P, P, S, ct.POINTER(S), P]),
            "psw_decode_frame": (I, [P, P, FD, P, S, P, P, P, P, P]),
            "psw_decode_batch": (I, [P, I, P, FD, P, P, P, P, P, P, P, P]),
            "psw_rate": (I, [P, S, P, P, P, ct.POINTER(ct.c_double), P]),
            "psw_lrp_residual": (I, [P, P, FD, P, P]),
            "psw_hyper_encode": (I, [P, P, FD, P, P, P, P, S, ct.POINTER(S), P]),
            "psw_hyper_decode": (I, [P, FD, P, S, P, P]),
            "psw_prior_table": (I, [P, I, P, I, ct.POINTER(I)]),
            "psw_set_tile_policy": (I, [P, I, I]),
            "psw_tile_policy": (I, [P, I]),
            "psw_quantize": (I, [P, S, P, P, P, P, P]),
            "psw_scale_table": (I, [P, P]),
            "psw_cdf_table": (I, [P, I, P, I, ct.POINTER(I), ct.POINTER(I)]),
            "psw_rans_encode": (I, [P, P, FD, P, P, P, P, S, ct.POINTER(S), P]),
            "psw_rans_decode": (I, [P, P, FD, P, S, P, P, P, P]),
            "psw_launch_count": (ct.c_long, [P]),
            "psw_set_engine": (ct.c_int, [P, ct.c_int]),
            "psw_last_engine": (ct.c_int, [P]),
            "psw_profile_begin": (I, [P]),
            "psw_profile_end": (I, [P, ct.POINTER(KernelStat), I, ct.POINTER(I)]),
            "psw_rans_encode_noalloc": (I, [P, FD, P, P, P, P, S, ct.POINTER(S), P]),
            "psw_quantize_e4m3": (I, [S, P, P, ct.POINTER(ct.c_float)]),
            "psw_check_wait_timeout": (I, [P, ct.c_double]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _ptr(t) -> int | None:
    if t is None:
        return None
    return int(t.data_ptr())


def _stream(stream=None) -> int | None:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) or None


def model_desc(cfg) -> ModelDesc:
    d = cfg if isinstance(cfg, dict) else cfg.as_dict()
    return ModelDesc(**{k: int(d[k]) for k, _ in ModelDesc._fields_})


def frame_desc(H: int, W: int, schedule: int = PSW_SCHED_WAVEFRONT) -> FrameDesc:
    return FrameDesc(H, W, schedule)


def psw_weights_count(cfg) -> int:
    return int(load().psw_weights_count(ct.byref(model_desc(cfg))))


def quantize_e4m3(src, dst) -> float:
    """psw_quantize_e4m3: src float32 device tensor -> dst uint8 device
    tensor of the same element count (E4M3 bytes); returns the scale."""
    s = ct.c_float(0.0)
    st = load().psw_quantize_e4m3(src.numel(), _ptr(src), _ptr(dst), ct.byref(s))
    if st != 0:
        raise PswError(st, (load().psw_last_error(None) or b"").decode())
    return float(s.value)


class Context:
    """Owns a psw_ctx.  Methods map 1:1 onto the C ABI."""

    def __init__(self, cfg, weights: np.ndarray, precision: int = PSW_BF16, hbm_budget: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the P-SWA library runs on the GPU only")
        lib = load()
        self.cfg = cfg
        self.lib = lib
        self.precision = precision
        w = np.ascontiguousarray(weights, np.float32)
        out = ct.c_void_p()
        st = lib.psw_create(ct.byref(model_desc(cfg)), w.ctypes.data, w.size, precision, hbm_budget, ct.byref(out))
        if st != PSW_OK:
            raise PswError(st, lib.psw_last_error(None).decode())
        self.h = out
        self._seqs = []

    def close(self):
        if getattr(self, "h", None):
            self.lib.psw_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != PSW_OK:
            raise PswError(st, self.lib.psw_last_error(self.h).decode())

    def last_error(self) -> str:
        return self.lib.psw_last_error(self.h).decode()

    def ctx_bytes(self) -> int:
        return int(self.lib.psw_ctx_bytes(self.h))

    def seq_bytes(self, H: int, W: int) -> int:
        return int(self.lib.psw_seq_bytes(self.h, H, W))

    def seq_create(self, max_H: int, max_W: int) -> "Sequence":
        out = ct.c_void_p()
        self._check(self.lib.psw_seq_create(self.h, max_H, max_W, ct.byref(out)))
        return Sequence(self, out)

    def bitstream_capacity(self, H: int, W: int, schedule: int = 0) -> int:
        fd = frame_desc(H, W, schedule)
        return int(self.lib.psw_bitstream_capacity(self.h, ct.byref(fd)))

    def rate(self, y, mu, sigma, stream=None) -> float:
        out = ct.c_double()
        self._check(self.lib.psw_rate(self.h, y.numel(), _ptr(y), _ptr(mu), _ptr(sigma), ct.byref(out),
                                      _stream(stream)))
        return float(out.value)

    def quantize(self, mu, sigma, idx, m, stream=None):
        self._check(self.lib.psw_quantize(self.h, mu.numel(), _ptr(mu), _ptr(sigma), _ptr(idx), _ptr(m),
                                          _stream(stream)))

    def scale_table(self) -> np.ndarray:
        t = np.zeros(64, np.float32)
        self._check(self.lib.psw_scale_table(self.h, t.ctypes.data))
        return t

    def cdf_table(self, l: int):
        n, T = ct.c_int(), ct.c_int()
        f = np.zeros(4096, np.uint32)
        self._check(self.lib.psw_cdf_table(self.h, l, f.ctypes.data, 4096, ct.byref(n), ct.byref(T)))
        return f[:n.value].copy(), T.value

    def hyper_decode(self, fd: FrameDesc, bitstream, length: int, zhat, stream=None, check: bool = True) -> int:
        st = self.lib.psw_hyper_decode(self.h, ct.byref(fd), _ptr(bitstream), length, _ptr(zhat), _stream(stream))
        if check:
            self._check(st)
        return st

    def prior_table(self, ch: int) -> np.ndarray:
        f = (ct.c_uint32 * 64)()
        n = ct.c_int(0)
        self._check(self.lib.psw_prior_table(self.h, ch, f, 64, ct.byref(n)))
        return np.array(f[:n.value], np.uint32)

    def rans_encode_noalloc(self, fd: FrameDesc, y, idx, m, bitstream, stream=None, check: bool = True):
        """Coder-only encode without device allocation; returns (status, length)."""
        n = ct.c_size_t(0)
        st = self.lib.psw_rans_encode_noalloc(self.h, ct.byref(fd), _ptr(y), _ptr(idx), _ptr(m), _ptr(bitstream),
                                              bitstream.numel(), ct.byref(n), _stream(stream))
        if check:
            self._check(st)
        return st, int(n.value)

    def check_wait_timeout(self, seconds: float) -> int:
        """psw_check_wait_timeout: the status (PSW_ERR_TIMEOUT expected)."""
        return int(self.lib.psw_check_wait_timeout(self.h, float(seconds)))

    def launch_count(self) -> int:
        return int(self.lib.psw_launch_count(self.h))

    def set_engine(self, engine: int):
        """Decode engine: ENGINE_AUTO, ENGINE_GRAPH or ENGINE_PERSISTENT."""
        self._check(self.lib.psw_set_engine(self.h, int(engine)))

    def set_tile_policy(self, cls: int, tokens: int):
        self._check(self.lib.psw_set_tile_policy(self.h, cls, tokens))

    def tile_policy(self) -> list:
        return [int(self.lib.psw_tile_policy(self.h, k)) for k in range(4)]

    def last_engine(self) -> int:
        """Engine of the last decode (0: individual launches)."""
        return int(self.lib.psw_last_engine(self.h))

    def profile_begin(self):
        self._check(self.lib.psw_profile_begin(self.h))

    def profile_end(self) -> list:
        arr = (KernelStat * 16)()
        n = ct.c_int()
        self._check(self.lib.psw_profile_end(self.h, arr, 16, ct.byref(n)))
        return [dict(name=a.name.decode(), launches=int(a.launches), ms=float(a.ms), flops=float(a.flops),
                     bytes=float(a.bytes)) for a in arr[:n.value]]

    def decode_batch(self, seqs, fds, bitstreams, lens, zhats, outs, mus=None, sigmas=None, stream=None,
                     check: bool = True):
        """Decode one frame of each sequence together; returns per-frame statuses."""
        n = len(seqs)
        sp = (ct.c_void_p * n)(*[s.h for s in seqs])
        fa = (FrameDesc * n)(*fds)
        bp = (ct.c_void_p * n)(*[_ptr(b) for b in bitstreams])
        ln = (ct.c_size_t * n)(*lens)
        zp = (ct.c_void_p * n)(*[_ptr(z) for z in zhats])
        op = (ct.c_void_p * n)(*[_ptr(o) for o in outs])
        mp = (ct.c_void_p * n)(*[_ptr(x) for x in mus]) if mus is not None else None
        gp = (ct.c_void_p * n)(*[_ptr(x) for x in sigmas]) if sigmas is not None else None
        stv = (ct.c_int * n)()
        st = self.lib.psw_decode_batch(self.h, n, sp, fa, bp, ln, zp, op, mp, gp, stv, _stream(stream))
        if check:
            self._check(st)
        return list(stv)


class Sequence:
    """Owns a psw_seq (per-sequence device caches)."""

    def __init__(self, ctx: Context, h):
        self.ctx = ctx
        self.h = h
        ctx._seqs.append(self)

    def close(self):
        if getattr(self, "h", None) and self.ctx.h:
            self.ctx.lib.psw_seq_destroy(self.h)
        self.h = None

    def reset(self):
        self.ctx._check(self.ctx.lib.psw_seq_reset(self.h))

    def encode_params(self, fd: FrameDesc, y, z, mu=None, sigma=None, bitstream=None, stream=None) -> int:
        """Returns the container length (0 if no bitstream buffer)."""
        n = ct.c_size_t(0)
        cap = bitstream.numel() if bitstream is not None else 0
        self.ctx._check(self.ctx.lib.psw_encode_params(
            self.ctx.h, self.h, ct.byref(fd), _ptr(y), _ptr(z), _ptr(mu), _ptr(sigma), _ptr(bitstream), cap,
            ct.byref(n), _stream(stream)))
        return int(n.value)

    def decode_frame(self, fd: FrameDesc, bitstream, length: int, z, y_out, mu=None, sigma=None, stream=None,
                     check: bool = True) -> int:
        st = self.ctx.lib.psw_decode_frame(self.ctx.h, self.h, ct.byref(fd), _ptr(bitstream), length, _ptr(z),
                                           _ptr(y_out), _ptr(mu), _ptr(sigma), _stream(stream))
        if check:
            self.ctx._check(st)
        return st

    def hyper_encode(self, fd: FrameDesc, y, zhat, z=None, bitstream=None, stream=None) -> int:
        """Convolutional hyperprior: z-hat of the next frame (and z), and
        its container if a bitstream buffer is given; returns its length."""
        n = ct.c_size_t(0)
        cap = bitstream.numel() if bitstream is not None else 0
        self.ctx._check(self.ctx.lib.psw_hyper_encode(self.ctx.h, self.h, ct.byref(fd), _ptr(y), _ptr(zhat), _ptr(z),
                                                      _ptr(bitstream), cap, ct.byref(n), _stream(stream)))
        return int(n.value)

    def lrp_residual(self, fd: FrameDesc, eps=None, stream=None):
        """The LRP Transformer's residual eps [H][W][C] float32 of the last
        coded frame (eps may be None for the temporal model: the ring of
        per-block keys and values advances only)."""
        self.ctx._check(self.ctx.lib.psw_lrp_residual(self.ctx.h, self.h, ct.byref(fd), _ptr(eps), _stream(stream)))

    def rans_encode(self, fd: FrameDesc, y, idx, m, bitstream, stream=None) -> int:
        n = ct.c_size_t(0)
        self.ctx._check(self.ctx.lib.psw_rans_encode(self.ctx.h, self.h, ct.byref(fd), _ptr(y), _ptr(idx), _ptr(m),
                                                     _ptr(bitstream), bitstream.numel(), ct.byref(n),
                                                     _stream(stream)))
        return int(n.value)

    def rans_decode(self, fd: FrameDesc, bitstream, length: int, idx, m, y_out, stream=None, check=True) -> int:
        st = self.ctx.lib.psw_rans_decode(self.ctx.h, self.h, ct.byref(fd), _ptr(bitstream), length, _ptr(idx),
                                          _ptr(m), _ptr(y_out), _stream(stream))
        if check:
            self.ctx._check(st)
        return st
