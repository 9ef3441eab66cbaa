"""The C-ABI libraries build for sm_103a, load, and export every symbol that
include/*.h declares; argument validation needs no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libs():
    from paper_1212_0262_gb300 import build

    return build.build()


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b(md[a-z_]*)\s*\(", txt)
    return sorted(set(names))


@pytest.mark.parametrize("header,lib", [("md.h", "libmd.so"), ("md_peaks.h", "libmdpeaks.so")])
def test_every_declared_symbol_is_exported(libs, header, lib):
    so = ctypes.CDLL(libs[lib])
    names = _declared(header)
    assert len(names) >= (30 if header == "md.h" else 1)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_binding_covers_the_header(libs):
    from paper_1212_0262_gb300 import binding

    assert set(_declared("md.h")) == set(binding._SIGS)


def test_invalid_arguments_fail_before_touching_the_device(libs):
    from paper_1212_0262_gb300 import binding as B

    lib = B.load()
    for args in [(7, 10, 0.0, 0.1, 1), (B.MD_RING, 0, 0.01, 0.1, 1), (B.MD_RING, 10, 0.0, 0.1, 1),
                 (B.MD_GRAV2D, 10, -1.0, 0.1, 1), (B.MD_HMF, 10, float("nan"), 0.1, 1),
                 (B.MD_HMF, 10, 0.0, float("inf"), 1)]:
        assert not lib.md_init(*args)
        assert lib.md_last_error(None)
        assert lib.md_last_status() == B.MD_EINVAL
    assert lib.md_set_allocator(ctypes.c_void_p(1), None, None) == B.MD_EINVAL
    assert lib.md_set_precision(None, 0) == B.MD_EINVAL
    assert lib.md_step(None, 1) == B.MD_EINVAL
    assert lib.md_launch_count(None) == 0
    lib.md_free(None)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1212_0262_gb300 import binding as B

    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "LIB_PATH", str(tmp_path / "libmd.so"))
    with pytest.raises(RuntimeError, match="missing"):
        B.load()
