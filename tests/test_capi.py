"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/cqr.h declares.  No compute calls (runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cqr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cqr_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cqr_factor", "cqr_backward", "cqr_factor_batched", "cqr_workspace_size", "cqr_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2405_04237_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (cqr_\w+)", out))
    assert set(declared_functions()) <= exported


def test_library_targets_sm_103a():
    from paper_2405_04237_gb300 import build

    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_host_only_entry_points():
    import paper_2405_04237_gb300 as P

    assert P.default_panel(1024) == 256
    assert P.default_panel(64) == 16
    assert P.default_panel(16) == 4
    assert P.default_panel(7) == 1
    assert "breakdown" in P.status_string(3)
    assert "invalid" in P.status_string(-4)


def test_no_cpu_fallback():
    torch = pytest.importorskip("torch")
    import paper_2405_04237_gb300 as P

    with pytest.raises(ValueError):
        P.factor(torch.zeros(10, 2, dtype=torch.float64))
    # every entry point refuses host tensors before anything reaches the library
    Q, R = torch.zeros(10, 2, dtype=torch.float64), torch.eye(2, dtype=torch.float64)
    with pytest.raises(ValueError):
        P.backward(Q, R, Q, R)
    with pytest.raises(ValueError):
        P.factor_batched([Q])
    with pytest.raises(ValueError):
        P.qr_batched([Q], 1)
    assert P.factor_batched([]) == [] and P.qr_batched([]) == []


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2405_04237_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "cqr_oracle" not in text, f
