"""The C-ABI library builds, loads without a GPU and exports every function that
include/*.h declares; the ctypes structures match the header's layout."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*([a-z_][a-z0-9_]*)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1504_05022_gb300 import _build, _lib
    _build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["spgemm_symbolic", "spgemm_numeric", "spgemm_free", "spgemm_status_string",
                     "spgemm_opts_init", "spgemm_plan_stats"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1504_05022_gb300 import _lib
    so = _lib.lib_path()
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in _declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    for n in _declared_functions():
        assert hasattr(lib, n)
    # the ctypes signature table covers every declared function
    assert set(_lib.SIGNATURES) == _declared_functions()


def test_status_strings_and_defaults(lib):
    from paper_1504_05022_gb300 import _lib
    for code in range(8):
        s = lib.spgemm_status_string(code)
        assert isinstance(s, bytes) and len(s) > 3
    o = _lib.Opts()
    assert lib.spgemm_opts_init(ctypes.byref(o)) == 0
    assert o.alloc_policy == 0 and o.initial_cap == 256 and o.check_inputs == 0
    assert lib.spgemm_opts_init(None) == 1


def test_struct_layout_matches_header():
    from paper_1504_05022_gb300 import _lib
    assert ctypes.sizeof(_lib.CsrIn) == 56
    assert ctypes.sizeof(_lib.CsrOut) == 48
    assert _lib.Opts.predictor.offset == 64 and ctypes.sizeof(_lib.Opts) == 96
    assert _lib.Opts.dense_pred_min.offset == 80 and _lib.Opts.dense_keep.offset == 84
    assert _lib.Opts.max_bytes.offset == 88
    assert _lib.Stats.launches.offset == 38 * 8 + 10 * 8
    assert _lib.Opts.long_rows.offset == 7 * 4


def test_argument_errors_without_gpu(lib):
    """Invalid arguments are rejected before any CUDA call, so this runs on CPU."""
    from paper_1504_05022_gb300 import _lib
    plan = ctypes.c_void_p()
    A = _lib.CsrIn(4, 5, 0, ctypes.c_void_p(1), 32, None, None)
    B = _lib.CsrIn(6, 3, 0, ctypes.c_void_p(1), 32, None, None)
    assert lib.spgemm_symbolic(ctypes.byref(A), ctypes.byref(B), None, None, ctypes.byref(plan), None) == 2
    B.nrows = 5
    B.rowptr_bits = 16
    assert lib.spgemm_symbolic(ctypes.byref(A), ctypes.byref(B), None, None, ctypes.byref(plan), None) == 1
    assert lib.spgemm_symbolic(ctypes.byref(A), ctypes.byref(B), None, None, None, None) == 1
    assert lib.spgemm_numeric(None, None) == 1
    assert lib.spgemm_free(None) == 0
    assert lib.spgemm_pool_trim(-1, 0) == 1 and lib.spgemm_pool_trim(0, -1) == 1
    assert lib.spgemm_pool_trim(0, 0) == 0  # no pool yet: nothing to return
    code = ctypes.c_int64(0)
    assert lib.spgemm_check_status(None, 0) == 1
    assert lib.spgemm_check_status(ctypes.byref(code), 0) == 0 and code.value == -1  # not the checked build


def test_every_field_offset_matches_the_c_compiler(tmp_path):
    """Compiles a C program against include/spgemm.h that prints sizeof and offsetof of every
    field of the public structs, and compares them with the ctypes mirror."""
    import shutil
    from paper_1504_05022_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirror = {"spgemm_csr_in": _lib.CsrIn, "spgemm_csr_out": _lib.CsrOut, "spgemm_opts": _lib.Opts,
              "spgemm_stats": _lib.Stats, "spgemm_plan_arrays": _lib.PlanArrays}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "spgemm.h"', "int main(void) {"]
    for cname, cls in mirror.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in out:
        if not line:
            continue
        cname, what, value = line.split()
        cls = mirror[cname]
        if what == "size":
            assert ctypes.sizeof(cls) == int(value), cname
        else:
            assert getattr(cls, what).offset == int(value), (cname, what)
        seen += 1
    assert seen == sum(len(c._fields_) + 1 for c in mirror.values())


def test_single_precision_library_exports_the_same_boundary():
    from paper_1504_05022_gb300 import _build, _lib
    _build.build()
    L32 = _lib.load(dtype="f32")
    assert L32 is not _lib.load()
    for name in _declared_functions():
        assert hasattr(L32, name), name
    o = _lib.Opts()
    assert L32.spgemm_opts_init(ctypes.byref(o)) == 0 and o.initial_cap == 256
