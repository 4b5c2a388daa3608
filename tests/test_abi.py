"""The C-ABI library loads and exports every function include/*.h declares.

No compute call is made here (no GPU in this environment)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def _declared():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        for m in re.finditer(r"\b(dbscan_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1912_06255_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_entry_points():
    names = _declared()
    assert {"dbscan_create", "dbscan_run", "dbscan_border_ids", "dbscan_destroy"} <= names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    from paper_1912_06255_gb300 import _lib
    assert _declared() <= set(_lib.SIGNATURES)


def test_status_strings_and_version(lib):
    from paper_1912_06255_gb300 import _lib
    for code in _lib.STATUS:
        assert lib.dbscan_status_string(code)
    assert lib.dbscan_status_string(99) == b"unknown status"
    assert lib.dbscan_version() >= 100


def test_stats_struct_layout_matches_header():
    """The ctypes mirror of dbscan_stats lists the header's fields in order."""
    from paper_1912_06255_gb300 import _lib
    text = (ROOT / "include" / "dbscan_gb300.h").read_text()
    body = text[text.index("typedef struct {"): text.index("} dbscan_stats;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(\w+)\s*(?:\[\d+\])?\s*[,;]", body.split("{", 1)[1])
    assert fields == [f for f, _ in _lib.Stats._fields_]


def test_null_context_calls_fail_cleanly(lib):
    """Argument checks happen on the host before any device call."""
    assert lib.dbscan_set_option(None, 0, 1) == 1
    assert lib.dbscan_get_stats(None, None) == 1
    assert lib.dbscan_border_ids(None, None, 0, None) == 1
    assert lib.dbscan_set_approx(None, 0.1) == 1
    n = ctypes.c_int64(-5)
    assert lib.dbscan_link_witnesses(None, None, None, 0, ctypes.byref(n), None) == 1
    n = ctypes.c_int64(-5)
    assert lib.dbscan_run_slabs(None, None, 10, 3, 0, 1.0, 5, 0, None, None, None, ctypes.byref(n), None, None) == 1
    assert n.value == -5  # nothing is written through a call that has no context
    assert lib.dbscan_slab_border_ids(None, None, 0, None) == 1
    out = ctypes.c_void_p()
    assert lib.dbscan_create(ctypes.byref(out), -1, 3) == 1
    assert lib.dbscan_create(ctypes.byref(out), 10, 9) == 2
    assert not out.value


def _c_layout(struct: str, fields: list, tmp_path) -> dict:
    """sizeof and offsetof of a header struct, as the C compiler lays it out."""
    import subprocess
    src = tmp_path / "layout.c"
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "dbscan_gb300.h"', "int main(void) {",
             f'  printf("size %zu\\n", sizeof({struct}));']
    lines += [f'  printf("{f} %zu\\n", offsetof({struct}, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", f"-I{ROOT / 'include'}", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


@pytest.mark.parametrize("struct,cls", [("dbscan_stats", "Stats"), ("dbscan_instance", "Instance"),
                                        ("dbscan_tuning", "Tuning"), ("dbscan_slab_stats", "SlabStats")])
def test_struct_layouts_match_the_c_compiler(struct, cls, tmp_path):
    """The ctypes mirrors have the C compiler's size and field offsets."""
    import shutil
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_1912_06255_gb300 import _lib
    mirror = getattr(_lib, cls)
    fields = [f for f, _ in mirror._fields_]
    c = _c_layout(struct, fields, tmp_path)
    assert c["size"] == ctypes.sizeof(mirror), struct
    for f in fields:
        assert c[f] == getattr(mirror, f).offset, (struct, f)


def test_injected_create_failure_needs_no_device(lib, monkeypatch):
    """DBSCAN_FAULT=create makes dbscan_create report OOM before any CUDA call."""
    monkeypatch.setenv("DBSCAN_FAULT", "create")
    out = ctypes.c_void_p()
    assert lib.dbscan_create(ctypes.byref(out), 10, 3) == 3
    assert not out.value
