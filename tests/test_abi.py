"""Host-side checks of the C ABI library (no GPU needed).

The library must load, export every entry point that include/blowchoc.h
declares, and reject bad parameters before touching the device.
"""
import os
import re
import subprocess

import pytest

import paper_2501_18977_gb300 as bc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "blowchoc.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^[a-z0-9_ ]+\**\s*\**(blowchoc_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2501_18977_gb300 import build as pkg_build
    pkg_build.build()
    return bc.load_library()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["blowchoc_create", "blowchoc_insert", "blowchoc_query", "blowchoc_stats",
                 "blowchoc_destroy"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", bc.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (blowchoc_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    # and the binding wraps exactly the declared names
    assert sorted(bc.exported_symbols()) == _declared()


def _params(**kw):
    p = dict(nblocks=64, k=8, choices=2, cost=bc.COST_MIX, bitsel=0, cost_param=50.0,
             hash_seed=1, batch=1)
    p.update(kw)
    return bc.blowchoc_params(**p)


@pytest.mark.parametrize("kw", [dict(nblocks=0), dict(nblocks=(1 << 32) + 1), dict(k=0),
                                dict(k=33), dict(choices=0), dict(choices=4), dict(cost=3),
                                dict(cost=-1), dict(cost_param=-1.0),
                                dict(cost=bc.COST_EXP, cost_param=0.0),
                                dict(cost_param=float("nan")), dict(bitsel=2), dict(batch=0)])
def test_create_rejects_bad_params(lib, kw):
    with pytest.raises(bc.BlowChocError) as ei:
        bc.blowchoc_create(_params(**kw), 0)
    assert ei.value.code == bc.BLOWCHOC_EINVAL
    assert bc.blowchoc_last_error()


def test_null_handles_rejected(lib):
    import ctypes
    assert lib.blowchoc_insert(None, None, 5, None) == bc.BLOWCHOC_EINVAL
    assert lib.blowchoc_query(None, None, 5, None, None) == bc.BLOWCHOC_EINVAL
    assert lib.blowchoc_stats(None, None) == bc.BLOWCHOC_EINVAL
    assert lib.blowchoc_destroy(None) == bc.BLOWCHOC_OK
    assert lib.blowchoc_create(None, None, None) == bc.BLOWCHOC_EINVAL
    h = ctypes.c_void_p()
    assert lib.blowchoc_create(None, None, ctypes.byref(h)) == bc.BLOWCHOC_EINVAL
    assert h.value is None


def test_no_cpu_fallback_without_device(lib):
    """On a machine without a usable GPU, creation fails loudly (ECUDA)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(bc.BlowChocError) as ei:
        bc.blowchoc_create(_params(), 0)
    assert ei.value.code == bc.BLOWCHOC_ECUDA
