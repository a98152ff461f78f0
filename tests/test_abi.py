"""The C ABI: the library builds for sm_103a, loads, exports every entry point
include/msstab.h declares, and the ctypes structures match the C layout.
No GPU is needed (no compute call is made)."""

import ctypes
import os
import re
import shutil
import subprocess
import tempfile

import pytest

from paper_1604_06043_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "msstab.h")

needs_nvcc = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(msstab_[a-z0-9_]+)\s*\(", text)))


@needs_nvcc
def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


@needs_nvcc
def test_binding_declares_the_header():
    from paper_1604_06043_gb300 import msstab
    B.build()
    assert set(msstab.exported_symbols()) == set(declared_functions())


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_struct_layout_matches_ctypes():
    from paper_1604_06043_gb300 import msstab
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "msstab.h"
int main(void) {
  printf("%zu %zu\n", sizeof(msstab_options), sizeof(msstab_stats));
  printf("%zu %zu %zu\n", offsetof(msstab_options, stream), offsetof(msstab_options, max_mvs),
         offsetof(msstab_options, inner_tol));
  printf("%zu %zu %zu\n", offsetof(msstab_stats, t_ms), offsetof(msstab_stats, n_launch),
         offsetof(msstab_stats, status));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    vals = list(map(int, out))
    O, S = msstab.Options, msstab.Stats
    assert vals[0] == ctypes.sizeof(O) and vals[1] == ctypes.sizeof(S)
    assert vals[2] == O.stream.offset and vals[3] == O.max_mvs.offset and vals[4] == O.inner_tol.offset
    assert vals[5] == S.t_ms.offset and vals[6] == S.n_launch.offset and vals[7] == S.status.offset


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1604_06043_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", text, flags=re.M), f


@needs_nvcc
def test_row_bound_is_checked_before_any_device_work():
    # n above 2^31 - 2^22 would let a signed 32-bit grid-stride row index
    # overflow; both entry points reject it on the host, before any CUDA call
    from paper_1604_06043_gb300 import msstab
    B.build()
    lib = msstab.load()
    big = (1 << 31) - (1 << 22) + 1
    dummy = ctypes.c_void_p(256)             # never dereferenced: the size check comes first
    h = ctypes.c_void_p()
    rc = lib.msstab_create(big, 0, dummy, None, None, 4, 2, dummy, None, ctypes.byref(h))
    assert rc == msstab.ERR_INVALID_ARG and not h.value
    assert b"n must be" in lib.msstab_last_error(None)
    rc = lib.msstab_spmv_dot_noalloc(big, 0, dummy, None, None, dummy, dummy, dummy, big, 4, dummy, None)
    assert rc == msstab.ERR_INVALID_ARG
    assert b"n must be" in lib.msstab_last_error(None)
