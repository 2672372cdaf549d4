"""The C-ABI library loads without a GPU and exports every symbol include/dj.h declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "dj.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(dj_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2504_03667_gb300 import build, dj
    build.build()
    return dj.load_library()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("dj_load_edges", "dj_sssp", "dj_sssp_batch", "dj_serve", "dj_graph_free", "dj_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2504_03667_gb300 import dj
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert missing == []
    # the binding marshals every declared entry point under the same name
    assert sorted(dj.SIGNATURES) == _declared()


def test_exports_with_nm(lib):
    from paper_2504_03667_gb300 import dj
    out = subprocess.run(["nm", "-D", "--defined-only", dj.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (dj_[a-z0-9_]+)", out))
    assert set(_declared()) <= exported


def test_host_only_calls(lib):
    from paper_2504_03667_gb300 import dj
    assert dj.dj_version() >= 10000
    assert lib.dj_status_string(dj.DJ_ETIMEOUT) == b"in-kernel wait timed out"
    o = dj.make_solve_opts()
    assert o.debug_skip_cta == -1 and o.mode == 0


def test_missing_library_fails_loudly(tmp_path):
    from paper_2504_03667_gb300 import dj
    with pytest.raises(OSError):
        dj.load_library(str(tmp_path / "libdj.so"))
