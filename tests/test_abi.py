"""The C ABI library builds, loads without a GPU, and exports every entry
point that include/hfp.h declares (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(hfp_[a-z0-9_]+)\s*\(", text))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("hfp_build_flow_network", "hfp_max_flow", "hfp_min_cut_source_side",
                     "hfp_pierce_and_augment", "hfp_flowcutter", "hfp_ctx_create",
                     "hfp_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2201_01556_gb300 import _build
    lib_path = _build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_loads_and_reports_no_device_cleanly():
    """Without a GPU the binding still loads; creating a context fails with a
    status (no fallback path), never silently."""
    torch = pytest.importorskip("torch")
    from paper_2201_01556_gb300 import hfp
    hfp.load()
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(hfp.HfpError):
        hfp.ctx_create(0)
