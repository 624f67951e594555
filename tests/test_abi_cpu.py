"""The C-ABI library builds, loads without a GPU and exports every entry
point include/psw.h declares; host-only entry points agree with the weight
layout of the synthetic-input module and the oracle."""
import ctypes as ct
import os
import re

import pytest

from paper_2605_20977_gb300 import psw, synth
import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "psw.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(psw_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_20977_gb300 import build
    build.build()
    return psw.load()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(psw.EXPORTS) == names


@pytest.mark.parametrize("name", ["tiny", "tiny_p", "tiny_cyc", "i1080", "p1080", "tiny_lrp", "tiny_p_lrp",
                                  "i1080_lrp", "p1080_lrp", "tiny_ct", "tiny_cyc_ct", "tiny_p_ct", "tiny_ct_lrp",
                                  "i1080_ct", "i1080_cyc_ct", "tiny_hp", "tiny_p_hp", "i1080_hp", "p1080_hp"])
def test_weights_count_matches_layouts(lib, name):
    c = synth.config(name)
    assert psw.psw_weights_count(c) == synth.weights_count(c) == O.weights_count(c)


def test_invalid_descriptors_rejected(lib):
    c = synth.config("tiny").as_dict()
    for bad in (dict(d=100), dict(nh=3), dict(k=4), dict(C=0), dict(mask=2), dict(F=0),
                dict(temporal=1, Lc=0), dict(temporal=1, Lc=1, Tf=5), dict(Llrp=-1), dict(Llrp=65),
                dict(dc=256), dict(Nc=4, dc=256, Lct=0, Fc=192), dict(Nc=3, dc=192, Lct=2, Fc=192),
                dict(Nc=4, dc=128, Lct=2, Fc=192), dict(Nc=4, dc=256, Lct=2, Fc=100),
                dict(Nc=2, dc=2048, Lct=2, Fc=192), dict(hp=2), dict(hp=1, r=3), dict(hp=1, Ch=30)):
        d = dict(c); d.update(bad)
        assert psw.psw_weights_count(d) == 0, bad


def test_create_errors_without_crashing(lib):
    # argument checks happen before any device call
    out = ct.c_void_p()
    md = psw.model_desc(synth.config("tiny"))
    st = lib.psw_create(ct.byref(md), None, 0, psw.PSW_FP32, 0, ct.byref(out))
    assert st == psw.PSW_ERR_INVALID and not out.value
    assert b"weights" in lib.psw_last_error(None)
    st = lib.psw_create(ct.byref(md), None, 0, 7, 0, ct.byref(out))
    assert st == psw.PSW_ERR_INVALID
