"""The C-ABI library loads and exports what include/slrcount.h declares (CPU only, no compute)."""
import ctypes
import os
import re
import subprocess

import pytest

from .conftest import ROOT

HEADER = os.path.join(ROOT, "include", "slrcount.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_05890_gb300 as pkg
    return pkg.load_library()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char)\s*\*?\s*(slr_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_binding_names():
    import paper_2312_05890_gb300 as pkg
    assert declared_functions() == sorted(pkg.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    so = os.path.join(ROOT, "paper_2312_05890_gb300", "libslrcount.so")
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(\w+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert getattr(lib, n) is not None


def test_default_options(lib):
    import paper_2312_05890_gb300 as pkg
    o = pkg.slr_default_options()
    assert o.precision == pkg.PREC_FP32 and o.relax_mode == pkg.RELAX_NEURIFY
    assert o.fp64_recheck == 1 and o.record_leaves == 0
    assert o.frontier_cap == 1 << 24


def test_null_context_is_rejected_without_a_gpu(lib):
    import paper_2312_05890_gb300 as pkg
    assert lib.slr_load_network(None, 1, None, None, None) == -1
    assert lib.slr_set_box(None, 1, None, None) == -1
    assert lib.slr_count(None, 3, None) == -1
    used = ctypes.c_size_t(7)
    assert lib.slr_count_checkpoint(None, 3, 1, None, 0, ctypes.byref(used)) == -1
    assert lib.slr_count_resume(None, b"", 0, None) == -1
    assert lib.slr_destroy(None) == 0
    assert b"null context" in lib.slr_last_error(None)
    out = ctypes.c_void_p()
    rc = lib.slr_create(ctypes.byref(out), -1, None)
    assert rc in (-1, -3) and not out.value   # no device here, or device -1 out of range
    _ = pkg


def test_result_struct_matches_header_size(lib):
    import paper_2312_05890_gb300 as pkg
    src = (
        '#include <stdio.h>\n#include <stddef.h>\n#include "slrcount.h"\n'
        'int main(void){printf("%zu %zu %zu %zu", sizeof(slr_result), sizeof(slr_options),'
        ' offsetof(slr_result, device_ms), offsetof(slr_options, frontier_cap)); return 0;}\n')
    import tempfile
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "t.c")
        exe = os.path.join(td, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        sizes = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert sizes[0] == ctypes.sizeof(pkg.slr_result)
    assert sizes[1] == ctypes.sizeof(pkg.slr_options)
    assert sizes[2] == pkg.slr_result.device_ms.offset
    assert sizes[3] == pkg.slr_options.frontier_cap.offset


def test_every_struct_field_matches_the_header(lib):
    """Every field of every ctypes mirror sits at the header's offset, and each
    struct has the header's size (the binding and include/slrcount.h agree)."""
    import tempfile
    import paper_2312_05890_gb300 as pkg
    structs = [pkg.slr_options, pkg.slr_result, pkg.slr_approx_options, pkg.slr_approx_result, pkg.slr_problem]
    lines = []
    for st in structs:
        name = st.__name__
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f in st._fields_:
            lines.append(f'printf("{name}.{f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    src = ('#include <stdio.h>\n#include <stddef.h>\n#include "slrcount.h"\nint main(void){\n' +
           "\n".join(lines) + "\nreturn 0;}\n")
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "t.c")
        exe = os.path.join(td, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.split() for line in out if line.strip())
    for st in structs:
        name = st.__name__
        assert int(got[name]) == ctypes.sizeof(st), name
        for f in st._fields_:
            assert int(got[f"{name}.{f[0]}"]) == getattr(st, f[0]).offset, (name, f[0])
