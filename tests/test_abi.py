"""Host-side checks of the C ABI (no GPU needed): the library builds for sm_103a, loads, and
exports every entry point that include/negf.h declares; the binding refuses to run without it."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "negf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:[\w\s\*]+?)\b(negf_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1805_10164_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("negf_build_tables", "negf_walk", "negf_current", "negf_create",
                     "negf_export_tables", "negf_walk_trace", "negf_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert lib.negf_abi_version() == 6


def test_binding_signatures_cover_header(lib_path):
    from paper_1805_10164_gb300 import negf
    lib = negf.load()
    for n in declared_functions():
        assert getattr(lib, n).restype is not None or n in (
            "negf_destroy", "negf_tables_free", "negf_tally_free", "negf_plan_destroy"), n


def test_status_codes_match_header():
    from paper_1805_10164_gb300 import negf
    src = open(os.path.join(ROOT, "include", "negf.h")).read()
    for name, val in (("NEGF_OK", 0), ("NEGF_E_INVALID", 1), ("NEGF_E_NOMEM", 2),
                      ("NEGF_E_CUDA", 3), ("NEGF_E_NUMERIC", 4), ("NEGF_E_STEPCAP", 5),
                      ("NEGF_E_TIMEOUT", 6)):
        assert re.search(rf"{name}\s*=\s*{val}\b", src)
        assert getattr(negf, name) == val


def test_struct_layouts_match_header(lib_path):
    """Field sizes of the ctypes mirrors against a C compile of the header."""
    import subprocess
    import tempfile
    from paper_1805_10164_gb300 import negf
    code = r'''
    #include <stdio.h>
    #include <stddef.h>
    #include "negf.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(negf_wire),
             offsetof(negf_wire, gamma_lead), sizeof(negf_build_opts), sizeof(negf_task_info),
             sizeof(negf_run_opts), offsetof(negf_run_opts, walk_blocks_per_sm),
             sizeof(negf_plan_tuning), sizeof(negf_thermal_result),
             offsetof(negf_thermal_result, truncated));
      return 0;
    }'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(code)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(x) for x in out]
    assert sizes == [ctypes.sizeof(negf.negf_wire), negf.negf_wire.gamma_lead.offset,
                     ctypes.sizeof(negf.negf_build_opts), ctypes.sizeof(negf.negf_task_info),
                     ctypes.sizeof(negf.negf_run_opts), negf.negf_run_opts.walk_blocks_per_sm.offset,
                     ctypes.sizeof(negf.negf_plan_tuning), ctypes.sizeof(negf.negf_thermal_result),
                     negf.negf_thermal_result.truncated.offset]


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1805_10164_gb300 import negf
    monkeypatch.setattr(negf, "_lib", None)
    monkeypatch.setattr(negf, "library_path", lambda: str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="not built"):
        negf.load()


def test_device_error_words_map_to_statuses(lib_path):
    """The bits kernels set in a device error word surface as the documented statuses; a
    bounded device wait that gave up (bit 16, the tensor-core kernels' mbarrier waits) is
    NEGF_E_TIMEOUT unless an input error is also recorded."""
    from paper_1805_10164_gb300 import negf
    assert negf.negf_device_error_status(0) == (negf.NEGF_OK, "")
    st, msg = negf.negf_device_error_status(16)
    assert st == negf.NEGF_E_TIMEOUT and "bounded device wait" in msg
    assert negf.negf_device_error_status(16 | 1)[0] == negf.NEGF_E_TIMEOUT
    assert negf.negf_device_error_status(16 | 4)[0] == negf.NEGF_E_INVALID
    for word in (1, 2, 8, 1 | 2 | 8):
        assert negf.negf_device_error_status(word)[0] == negf.NEGF_E_NUMERIC
    assert negf.negf_device_error_status(4)[0] == negf.NEGF_E_INVALID
    lib = negf.load()
    small = ctypes.create_string_buffer(8)
    assert lib.negf_device_error_status(16, small, 8) == negf.NEGF_E_TIMEOUT
    assert len(small.value) == 7
