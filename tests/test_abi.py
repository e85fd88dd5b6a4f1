"""The C-ABI library builds for sm_103a, loads without a GPU and exports every entry point
that include/rtg.h declares; host-only entry points behave as documented."""
import os
import re

import numpy as np
import pytest

from paper_1409_8112_gb300 import gen, rtg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(rtg_\w+)\s*\(", text, flags=re.M))
    return names


def test_library_exports_every_declared_function():
    L = rtg.lib()
    declared = header_functions()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(L, name), f"{name} declared in include/ but not exported"
    assert set(rtg.exported_symbols()) <= declared | {"rtg_zz_unused"}


def test_status_strings():
    assert rtg.status_name(rtg.RTG_OK) == "RTG_OK"
    assert rtg.status_name(rtg.RTG_E_KEY_OVERFLOW) == "RTG_E_KEY_OVERFLOW"
    assert rtg.status_name(99) == "RTG_E_UNKNOWN_STATUS"


def test_transforms_generate_matches_generator_module():
    for flags in (0, rtg.RTG_FLAG_SHIFT_ONLY):
        a = rtg.rtg_transforms_generate(5, 6, 8, 0.2, flags)
        b = gen.transforms(5, 6, 8, 0.2, flags=gen.SHIFT_ONLY if flags else 0)
        assert np.array_equal(a, b)


def test_transforms_generate_rejects_bad_arguments():
    for args in ((1, 0, 3, 0.1), (1, 17, 3, 0.1), (1, 3, 0, 0.1), (1, 3, 3, 0.0),
                 (1, 3, 3, float("nan"))):
        with pytest.raises(rtg.RTGError) as e:
            rtg.rtg_transforms_generate(*args)
        assert e.value.status == rtg.RTG_E_INVALID


def test_all_pairs_rejects_null_context():
    L = rtg.lib()
    out = rtg.rtg_csr()
    T = np.zeros(12)
    st = L.rtg_all_pairs(None, None, 0, 0, 0, 3, 0.1, T.ctypes.data, 1, 0.1, 0, out)
    assert st == rtg.RTG_E_INVALID


def test_create_without_gpu_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(rtg.RTGError) as e:
        rtg.rtg_create(0)
    assert e.value.status == rtg.RTG_E_CUDA


def test_header_is_plain_c(tmp_path):
    """The boundary is a C ABI: the public header compiles as strict C99 (no C++ in it)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    src = tmp_path / "use_header.c"
    src.write_text('#include "rtg.h"\n'
                   'int main(void) { return rtg_status_string(RTG_OK) ? 0 : 1; }\n')
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-fsyntax-only", "-I", os.path.join(ROOT, "include"), str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
