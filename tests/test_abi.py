"""The C-ABI library loads and exports every symbol include/pwqt.h declares
(no compute calls: this runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pwqt.h")).read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(pwqt_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1903_00548_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("pwqt_create", "pwqt_assemble_intrinsic", "pwqt_set_extrinsic", "pwqt_solve", "pwqt_bands"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(pwqt_\w+)$", out, flags=re.M))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing


def test_binding_loads_and_names_match(lib_path):
    from paper_1903_00548_gb300 import pwqt
    lib = pwqt.load(lib_path)
    for s in declared_symbols():
        assert hasattr(lib, s)
    assert set(pwqt.EXPORTS) == set(declared_symbols())


def test_missing_library_fails_loudly(tmp_path):
    from paper_1903_00548_gb300 import pwqt
    with pytest.raises(RuntimeError):
        pwqt._lib = None
        pwqt.load(str(tmp_path / "nope.so"))
    pwqt._lib = None
