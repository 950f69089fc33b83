"""The C-ABI library builds for sm_103a, loads, and exports every symbol of include/epw.h.

No compute call is made here (no GPU needed).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(epw_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1604_03525_gb300 import _lib
    return _lib.load()


def test_library_exports_every_declared_symbol(lib):
    declared = _declared_functions()
    assert "epw_linewidth" in declared and "epw_load_wannier" in declared
    for name in declared:
        assert hasattr(lib, name), name
    from paper_1604_03525_gb300 import _lib
    assert set(declared) <= set(_lib.SIGNATURES)


def test_abi_version_and_error_string(lib):
    assert lib.epw_abi_version() == 1
    assert isinstance(lib.epw_last_error(), bytes)


def test_null_arguments_rejected_without_gpu_work(lib):
    from paper_1604_03525_gb300 import _lib
    # null descriptor / null model are rejected before any CUDA call
    assert lib.epw_load_wannier(None, None) == 1
    assert lib.epw_model_info(None, None, None, None, None, None) == 1
    assert lib.epw_sync(None, None) == 1
    assert b"null" in lib.epw_last_error()
    lib.epw_free_model(None)  # no-op


def test_struct_layouts_match_header(tmp_path):
    from paper_1604_03525_gb300 import _lib
    # epw_wannier_desc: ints and pointers in declaration order (LP64)
    assert ctypes.sizeof(_lib.WannierDesc) == 120
    assert ctypes.sizeof(_lib.Params) == 4 * 8 + 2 * 4
    # the C compiler's view of the header (plain C, no CUDA headers needed)
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include "epw.h"\nint main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n",'
                   ' sizeof(epw_wannier_desc), sizeof(epw_params), sizeof(epw_linewidth_job),'
                   ' offsetof(epw_linewidth_job, params), offsetof(epw_linewidth_job, imsigma),'
                   ' sizeof(epw_polar_desc), offsetof(epw_polar_desc, gmax));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run([cc, "-include", "stddef.h", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    sizes = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    J = _lib.LinewidthJob
    assert sizes == [ctypes.sizeof(_lib.WannierDesc), ctypes.sizeof(_lib.Params), ctypes.sizeof(J),
                     J.params.offset, J.imsigma.offset, ctypes.sizeof(_lib.PolarDesc), _lib.PolarDesc.gmax.offset]


def test_selftest_arguments_rejected_without_gpu_work(lib):
    assert lib.epw_selftest_wait_timeout(0, None) == 1
    assert lib.epw_selftest_wait_timeout(5000000000, None) == 1


def test_batch_arguments_rejected_without_gpu_work(lib):
    h = ctypes.c_void_p()
    assert lib.epw_batch_create(-1, None, ctypes.byref(h)) == 1
    assert lib.epw_batch_create(2, None, ctypes.byref(h)) == 1
    assert lib.epw_batch_create(0, None, None) == 1
    assert lib.epw_batch_run(None, None) == 1
    assert lib.epw_batch_info(None, None, None, None) == 1
    lib.epw_batch_free(None)  # no-op
