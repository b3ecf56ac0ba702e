"""The C-ABI library builds, loads and exports every symbol include/*.h declares.

CPU-only: no kernel is launched.  lsp_grid is host arithmetic and is checked
against the oracle's Eq. 10-11; lsp_create must refuse cleanly when no GPU is
present.
"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w \*]*?\b(lsp_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1007_1658_gb300 import build, lsp
    build.build()
    return lsp.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("lsp_create", "lsp_periodogram", "lsp_batch", "lsp_fap_predict", "lsp_destroy", "lsp_sync",
                 "lsp_grid", "lsp_last_error", "lsp_noise", "lsp_fap_train_step", "lsp_periodogram_noalloc",
                 "lsp_periodogram_gls", "lsp_press_rybicki", "lsp_batch_gls"):
        assert must in names, must


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_grid_matches_oracle(lib):
    import oracle
    from paper_1007_1658_gb300 import lsp
    for args in [(0.0, 100.0, 1000, 4.0, 1.0), (3.5, 1303.5, 65536, 10.0, 1.88), (0.0, 999.5, 100000, 4.0, 4.0)]:
        assert lsp.grid(*args) == oracle.grid(*args)
    with pytest.raises(lsp.LspError):
        lsp.grid(1.0, 1.0, 10, 4.0, 1.0)


def test_default_options_and_bad_create(lib):
    import torch
    from paper_1007_1658_gb300 import lsp
    o = lsp.options()
    assert o.sincos_mode == lsp.SINCOS_AUTO and o.phase_mode == lsp.PHASE_FIXED64
    if torch.cuda.is_available():
        pytest.skip("GPU present: refusal path not reachable")
    h = ctypes.c_void_p()
    assert lib.lsp_create(ctypes.byref(h), 0, None, None) == lsp.ERR_INVALID_ARG
    assert not h.value


def test_pointer_kind_decision(lib):
    # cudaMemoryType: 0 unregistered host, 1 host (pinned/registered), 2 device, 3 managed
    from paper_1007_1658_gb300 import lsp
    HOST, IN_PLACE, OTHER_GPU = 0, 1, 2
    for dev in (0, 1, 5):
        assert lsp.pointer_kind(0, -2, dev) == HOST
        assert lsp.pointer_kind(1, dev, dev) == HOST
        assert lsp.pointer_kind(1, dev + 1, dev) == HOST  # pinned memory is reachable from every GPU
        assert lsp.pointer_kind(2, dev, dev) == IN_PLACE
        assert lsp.pointer_kind(3, dev, dev) == IN_PLACE
        assert lsp.pointer_kind(3, dev + 1, dev) == IN_PLACE  # managed memory migrates on demand
        for other in (dev + 1, dev + 2, 7 if dev != 7 else 6):
            assert lsp.pointer_kind(2, other, dev) == OTHER_GPU
