"""The C-ABI library loads and exports every entry point include/psfd.h declares.

CPU-only: only host-side calls (string tables, length support, workspace sizing)
are made; nothing touches a device.
"""
import ctypes
import os
import re

import pytest

from paper_2606_25541_b300 import build as build_mod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(psfd_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return ctypes.CDLL(build_mod.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_host_side_entry_points():
    from paper_2606_25541_b300 import psfd
    build_mod.build()
    lib = psfd.load()
    assert psfd.strerror(psfd.E_ANOMALY).startswith("Rayleigh")
    for n in (4, 8, 64, 96, 128, 160, 384, 512, 640, 768, 1024):
        assert psfd.supported_length(n)
    for n in (0, 2, 7, 100, 1000, 2048):
        assert not psfd.supported_length(n)
    g = psfd.make_grid(128, 128, 60, 128, 1.0, 1.0, 1.0, 13.5)
    b32 = psfd.workspace_bytes(g, psfd.FP32_REFINED, 18)
    b64 = psfd.workspace_bytes(g, psfd.FP64, 18)
    U = 3 * 60 * 128 * 128
    assert b32 > 18 * U * (4 * 16 + 8 * 8)
    assert b64 > 18 * U * 9 * 16
    bad = psfd.make_grid(128, 128, 64, 128, 1.0, 1.0, 1.0, 13.5)  # nf < 2 nslab + 2
    with pytest.raises(psfd.PsfdError):
        psfd.workspace_bytes(bad, psfd.FP64, 1)
    assert lib.psfd_last_error(None) == b"null context"


def test_tune_set_rejects_shapes_the_kernels_cannot_take():
    from paper_2606_25541_b300 import psfd
    build_mod.build()
    psfd.load()
    g = psfd.make_grid(128, 128, 60, 128, 1.0, 1.0, 1.0, 13.5)
    for bad in ((3, 0, 0), (2, 0, 0), (32, 0, 0), (0, 0, 0)):
        if bad == (0, 0, 0):
            psfd.tune_set(g, psfd.FP32_REFINED, *bad)  # all built-in: accepted
            continue
        with pytest.raises(psfd.PsfdError):  # lane-group z transform: 4, 8 or 16 x-modes only
            psfd.tune_set(g, psfd.FP32_REFINED, *bad)
    psfd.tune_set(g, psfd.FP32_REFINED, 16, 0, 0)
    g2 = psfd.make_grid(256, 256, 12, 96, 1.0, 1.0, 1.0, 13.5)
    psfd.tune_set(g2, psfd.FP64, 2, 4, 8)
    with pytest.raises(psfd.PsfdError):
        psfd.tune_set(g2, psfd.FP64, 0, 3, 0)  # rows per CTA must divide ny
    psfd.tune_reset()
