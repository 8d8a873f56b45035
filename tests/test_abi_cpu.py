"""CPU-only checks of the C ABI: the library loads and exports every symbol
include/lsnif.h declares, and the binding's signature table matches them.
No compute call is made (no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lsnif.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lsnif_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_21627_gb300 import build as B
    try:
        path = B.build()
    except RuntimeError as e:  # pragma: no cover - nvcc is part of the image
        pytest.skip(f"cannot build: {e}")
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("lsnif_create", "lsnif_destroy", "lsnif_load_object", "lsnif_save_object", "lsnif_query_rays",
                 "lsnif_query_rays_host", "lsnif_train_step", "lsnif_submit", "lsnif_poll", "lsnif_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_every_declared_symbol(lib):
    from paper_2504_21627_gb300 import lsnif
    assert sorted(lsnif.SIGNATURES) == _declared()
    assert lsnif.load_library().lsnif_version() == 2


def test_library_exports_nothing_else(lib):
    # the shared object's dynamic symbols: only the C ABI is visible
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = sorted({l.split()[-1] for l in out.splitlines() if " T " in l and l.split()[-1].startswith("lsnif")})
    assert exported == _declared()


def test_context_creation_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2504_21627_gb300 import lsnif
    with pytest.raises(lsnif.LsnifError):
        lsnif.Context(0)
    assert "device" in lsnif.last_error().lower() or "cuda" in lsnif.last_error().lower()
