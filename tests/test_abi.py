"""The C-ABI library loads and exports every entry point that include/geomatch.h declares (CPU only: no compute
call is made without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

import __graft_entry__
from paper_1512_06235_gb300 import geomatch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "geomatch.h")).read()
    return sorted(set(re.findall(r"^GM_API\s+[\w\s\*]*?\b(gm_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return geomatch.load_library()


def test_header_declares_entry_points():
    names = _declared()
    assert "gm_match_pairs" in names and "gm_image_put" in names and len(names) >= 13


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    assert set(_declared()) <= set(geomatch.EXPORTED)


def test_struct_layouts_match_header():
    """Compile a tiny C program against the header and compare sizeof/offsetof with the ctypes mirrors."""
    src = os.path.join(ROOT, "_build", "abi_layout.c")
    exe = os.path.join(ROOT, "_build", "abi_layout")
    os.makedirs(os.path.dirname(src), exist_ok=True)
    with open(src, "w") as fh:
        fh.write('#include <stdio.h>\n#include <stddef.h>\n#include "geomatch.h"\nint main(void){\n'
                 'printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(gm_config), sizeof(gm_pair), '
                 'sizeof(gm_stats), sizeof(gm_serving_stats), offsetof(gm_pair, band_px), offsetof(gm_pair, ratio_den), '
                 'offsetof(gm_config, cuda_stream), sizeof(gm_tune_result), offsetof(gm_tune_result, ms), '
                 'sizeof(gm_image), offsetof(gm_image, desc));\nreturn 0;}\n')
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
    vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert vals == [ctypes.sizeof(geomatch.GmConfig), ctypes.sizeof(geomatch.GmPair), ctypes.sizeof(geomatch.GmStats),
                    ctypes.sizeof(geomatch.GmServingStats), geomatch.GmPair.band_px.offset,
                    geomatch.GmPair.ratio_den.offset, geomatch.GmConfig.cuda_stream.offset,
                    ctypes.sizeof(geomatch.GmTuneResult), geomatch.GmTuneResult.ms.offset,
                    ctypes.sizeof(geomatch.GmImage), geomatch.GmImage.desc.offset]


def test_no_cpu_fallback_when_library_missing(tmp_path):
    with pytest.raises(ImportError):
        geomatch._lib_backup = geomatch._lib
        try:
            geomatch._lib = None
            geomatch.load_library(str(tmp_path / "missing.so"))
        finally:
            geomatch._lib = geomatch._lib_backup
