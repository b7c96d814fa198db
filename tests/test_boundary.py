"""The C-ABI library builds for sm_103a, loads, and exports exactly what include/rwmi.h declares
(no compute calls: this runs on machines without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rwmi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"RWMI_API[^;{(]*?\b(rwmi_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2308_05007_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("rwmi_create", "rwmi_set_metaballs", "rwmi_step", "rwmi_concentration",
                     "rwmi_walker_moments", "rwmi_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(rwmi_\w+)\b", out))
    assert set(_declared()) <= exported, set(_declared()) - exported
    # nothing else leaks out of the C ABI
    assert exported == set(_declared())


def test_library_targets_sm_103a(lib_path):
    out = subprocess.run(["cuobjdump", "--list-elf", lib_path], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_binding_loads_and_matches_header(lib_path):
    from paper_2308_05007_gb300 import rwmi
    L = rwmi.load()
    assert set(rwmi.EXPORTED) == set(_declared())
    for name in rwmi.EXPORTED:
        assert hasattr(L, name)


def test_binding_refuses_without_library(monkeypatch, tmp_path):
    """The product path has no fallback: a missing library is an error."""
    from paper_2308_05007_gb300 import build, rwmi
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(rwmi, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        rwmi.load()


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2308_05007_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"(#|//).*", "", text).lower() or f == "inputs.py", f
