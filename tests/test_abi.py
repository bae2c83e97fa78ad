"""The C-ABI library loads and exports every entry point that include/mstep.h
declares (CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mstep.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ms_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2406_18356_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("ms_plan_create", "ms_grid", "ms_degrid", "ms_minor_cycle",
                 "ms_reconstruct_two_step", "ms_reconstruct_single_step"):
        assert want in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib_path):
    import paper_2406_18356_gb300 as ms
    assert set(_declared()) == set(ms.exported_symbols())
    ms.load_library()


def test_struct_layouts_match_the_header(lib_path):
    """ctypes mirrors of the ABI structs have the C sizes (checked against a
    tiny C program compiled from the header)."""
    import subprocess
    import tempfile
    import paper_2406_18356_gb300 as ms
    code = ('#include "mstep.h"\n#include <stdio.h>\nint main(void){printf("%zu %zu %zu",'
            'sizeof(ms_plan_desc),sizeof(ms_stats),sizeof(ms_recon_opts));return 0;}\n')
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(code)
        exe = os.path.join(d, "s")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        sizes = [int(x) for x in subprocess.run([exe], capture_output=True, text=True,
                                                check=True).stdout.split()]
    assert sizes == [ctypes.sizeof(ms.ms_plan_desc), ctypes.sizeof(ms.ms_stats),
                     ctypes.sizeof(ms.ms_recon_opts)]


def test_plan_create_rejects_bad_arguments_without_gpu(lib_path):
    """Argument checks run before any device work: a NULL descriptor is an
    argument error, not a crash."""
    import paper_2406_18356_gb300 as ms
    lib = ms.load_library()
    h = ctypes.c_void_p()
    assert lib.ms_plan_create(None, ctypes.byref(h)) == ms.MS_ERR_ARG
    assert lib.ms_plan_destroy(None) == ms.MS_ERR_ARG
