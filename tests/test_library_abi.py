"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/modal.h
declares (CPU only: no compute calls)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "modal.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(modal_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1105_2791_gb300 import build
    return build.build()


def test_library_loads_and_exports_every_declared_symbol(libpath):
    import paper_1105_2791_gb300 as M
    lib = M.load_library()
    declared = _declared_symbols()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(M.binding.EXPORTS) == declared


def test_library_is_built_for_sm103a_only(libpath):
    """Every translation unit is compiled and linked with the one sm_103a target and no
    other architecture flag (checked on the build's own command lines)."""
    from paper_1105_2791_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    for flag in build.FLAGS:
        assert "arch" not in flag and "sm_" not in flag and "compute_" not in flag, flag
    assert os.path.getsize(libpath) > 0


def test_no_cpu_fallback_without_library(monkeypatch, tmp_path):
    import paper_1105_2791_gb300.binding as B
    monkeypatch.setattr(B, "_LIB", None)
    monkeypatch.setattr(B, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        B.load_library()


def test_status_and_precision_codes_match_header():
    import paper_1105_2791_gb300 as M
    src = open(os.path.join(ROOT, "include", "modal.h")).read()
    for name in ["MODAL_OK", "MODAL_EINVAL", "MODAL_ENOMEM", "MODAL_ECUDA", "MODAL_ENOTPD",
                 "MODAL_ETIMEOUT", "MODAL_ESTATE", "MODAL_FP32", "MODAL_3XTF32", "MODAL_BF16X3",
                 "MODAL_BF16", "MODAL_FP16X3"]:
        val = int(re.search(r"\b%s\s*=\s*(\d+)" % name, src).group(1))
        assert getattr(M.binding, name) == val, name
