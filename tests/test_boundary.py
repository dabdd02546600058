"""The C-ABI library builds, loads on a machine without a GPU and exports
every entry point declared in include/isc.h; the binding fails loudly when
the library is missing (no CPU fallback)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "isc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(isc_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1811_11992_gb300 import build, isc
    lib_path = build.build()
    lib = isc.load_library(lib_path)
    names = _declared()
    assert len(names) >= 30
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(isc._SIGS), set(names) ^ set(isc._SIGS)


def test_status_strings_without_gpu():
    from paper_1811_11992_gb300 import isc
    lib = isc.load_library()
    assert lib.isc_status_string(0) == b"ok"
    assert lib.isc_status_string(-4) == b"singular diagonal block"
    o = isc.default_options()
    assert o.restart == 30 and o.prec == 2 and o.decouple == 1


def test_missing_library_fails_loudly(tmp_path):
    from paper_1811_11992_gb300 import isc
    saved = isc._lib
    isc._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            isc.load_library(str(tmp_path / "nope.so"))
    finally:
        isc._lib = saved
