"""CPU checks of the boundary: the library builds for sm_103a, loads, and exports every declared entry point."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dp_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    import paper_2005_00223_gb300 as pkg
    return pkg.build()


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (dp_[a-z0-9_]+)$", out, flags=re.M))
    declared = _declared()
    assert declared, "no declarations found"
    missing = [d for d in declared if d not in exported]
    assert not missing, missing


def test_binding_names_match_header(libpath):
    from paper_2005_00223_gb300 import _lib
    assert sorted(_lib.EXPORTS) == _declared()
    lib = _lib.load(libpath)
    for name in _lib.EXPORTS:
        assert hasattr(lib, name)


def test_status_strings_without_gpu(libpath):
    from paper_2005_00223_gb300 import _lib
    lib = _lib.load(libpath)
    for code, name in _lib.STATUS.items():
        assert lib.dp_status_string(code).decode() == name


def test_missing_library_fails_loudly(tmp_path):
    from paper_2005_00223_gb300 import _lib
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            _lib.load(str(tmp_path / "nope.so"))
    finally:
        _lib._lib = saved


def test_bounds_checked_build_compiles_and_reports_itself():
    """The debug build with every index check compiled in builds for sm_103a and exports the same
    entry points; dp_bounds_checked() tells the two builds apart without a GPU."""
    import paper_2005_00223_gb300 as pkg
    path = pkg.build(bounds_check=True)
    assert path.endswith(os.path.join("_build_bounds", "libdp.so"))
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (dp_[a-z0-9_]+)$", out, flags=re.M))
    assert not [d for d in _declared() if d not in exported]
    code = ("import ctypes, sys; a = ctypes.CDLL(sys.argv[1]); b = ctypes.CDLL(sys.argv[2]); "
            "print(a.dp_bounds_checked(), b.dp_bounds_checked())")
    r = subprocess.run([sys.executable, "-c", code, path, pkg.build()], capture_output=True, text=True, check=True)
    assert r.stdout.split() == ["1", "0"]
