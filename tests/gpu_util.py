"""Helpers for the GPU tests: contexts, oracle weights, tolerances."""
import numpy as np
import pytest

from paper_2605_20977_gb300 import synth

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def oracle_weights(cfg, w, precision):
    """The weights the GPU computes with, upcast to FP64: block projections
    rounded to bf16 (round-to-nearest-even, by torch on the CPU) in BF16
    mode; in FP8 mode the E4M3-stored projections quantised per tensor by
    the oracle's E4M3 rounding, the other projections rounded to bf16;
    everything else as stored."""
    from paper_2605_20977_gb300 import psw
    import oracle as O
    w64 = np.asarray(w, np.float64).copy()
    if precision == psw.PSW_BF16 or precision == psw.PSW_FP8:
        mask = synth.matrix_mask(cfg)
        t = torch.from_numpy(np.asarray(w, np.float32)[mask]).to(torch.bfloat16).to(torch.float64)
        w64[mask] = t.numpy()
    if precision == psw.PSW_FP8:
        for off, n in synth.e4m3_ranges(cfg):
            w64[off:off + n] = O.e4m3_tensor(np.asarray(w[off:off + n], np.float64))[0]
    return w64


def param_errors(mu, sg, mu_ref, sg_ref):
    """|dmu| / sigma_ref and |d ln sigma| arrays."""
    return np.abs(mu - mu_ref) / sg_ref, np.abs(np.log(sg) - np.log(sg_ref))


def dev():
    return torch.device("cuda:0")
