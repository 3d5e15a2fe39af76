"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/dfpr.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(pr_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2401_15870_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for need in ("pr_graph_create", "pr_apply_batch", "pr_update", "pr_ranks", "pr_set_ranks", "pr_graph_destroy",
                 "pr_last_error"):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_entry_points() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_need_no_gpu(lib):
    lib.pr_status_string.restype = ctypes.c_char_p
    lib.pr_status_string.argtypes = [ctypes.c_int]
    assert lib.pr_status_string(0) == b"PR_OK"
    assert lib.pr_status_string(4) == b"PR_ENORANKS"


def test_argument_errors_are_reported_before_any_device_work(lib):
    """Invalid arguments are rejected on the host without touching the GPU."""
    P = ctypes.c_void_p
    lib.pr_graph_create_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, P, P, ctypes.c_int32, ctypes.c_int32, P,
                                          ctypes.POINTER(P)]
    h = P()
    assert lib.pr_graph_create_edges(0, 0, None, None, 0, 0, None, ctypes.byref(h)) == 1      # n < 1
    assert lib.pr_graph_create_edges(4, -1, None, None, 0, 0, None, ctypes.byref(h)) == 1     # m < 0
    src = (ctypes.c_int32 * 2)(0, 7)
    dst = (ctypes.c_int32 * 2)(1, 2)
    assert lib.pr_graph_create_edges(4, 2, src, dst, 0, 0, None, ctypes.byref(h)) == 2        # id out of range
    lib.pr_update.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_double, P, P]
    assert lib.pr_update(None, 0, 0.85, 1e-10, None, None) == 1
    lib.pr_autotune.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int32, P]
    assert lib.pr_autotune(None, 1, 0.85, 1e-10, 3, None) == 1
    lib.pr_set_tuning.argtypes = [P, P]
    assert lib.pr_set_tuning(None, None) == 1
    for name in ("pr_apply_batches", "pr_apply_batches_device"):
        fn = getattr(lib, name)
        fn.argtypes = [ctypes.c_int32, P, P, P, P, P, P, P]
        counts = (ctypes.c_int64 * 1)(0)
        nulls = (P * 1)()
        assert fn(0, None, None, None, None, None, None, None) == 0                   # nothing to apply
        assert fn(-1, None, None, None, None, None, None, None) == 1                  # count < 0
        assert fn(1, None, nulls, nulls, counts, nulls, nulls, counts) == 1           # no graph array
        assert fn(1, nulls, nulls, nulls, counts, nulls, nulls, counts) == 1          # a null graph


def test_product_path_has_no_oracle_or_cpu_fallback():
    """The package never imports the oracle, and fails loudly without its library."""
    pkg = os.path.join(ROOT, "paper_2401_15870_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text
                assert "dfpr_oracle" not in text and "liboracle" not in text


def test_binding_structs_match_the_header(tmp_path):
    """Sizes and field offsets of the ctypes mirrors equal those gcc computes
    from include/dfpr.h."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("gcc not found")
    import paper_2401_15870_gb300 as pr
    structs = {"pr_options": pr.pr_options, "pr_stats": pr.pr_stats, "pr_server_options": pr.pr_server_options,
               "pr_request_info": pr.pr_request_info, "pr_tuning": pr.pr_tuning,
               "pr_group_tuning": pr.pr_group_tuning, "pr_sweep_record": pr.pr_sweep_record}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dfpr.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)]).decode().splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got[name + "." + field]) == getattr(cls, field).offset, (name, field)


def test_binding_constants_match_the_header():
    """Every PR_OPT_* flag and size limit the Python binding passes through has
    the header's value."""
    import paper_2401_15870_gb300 as pr
    text = open(os.path.join(ROOT, "include", "dfpr.h")).read()
    defs = {}
    for name, val in re.findall(r"#define\s+(PR_[A-Z_0-9]+)\s+\(?([0-9]+(?:ll)?(?:\s*<<\s*[0-9]+)?)\)?", text):
        defs[name] = eval(val.replace("ll", ""))
    checked = 0
    for name in dir(pr):
        if name.startswith(("PR_OPT_", "PR_ONE_", "PR_DEVICE_")) and name in defs:
            assert getattr(pr, name) == defs[name], name
            checked += 1
    assert checked >= 8
    assert pr.LOOPS["one"] == defs["PR_OPT_ONE_KERNEL"] and pr.LOOPS["device"] == defs["PR_OPT_DEVICE_LOOP"]
