"""CPU checks of the C ABI boundary: the shared library loads, exports every
function include/swpic.h declares, the Python binding names exactly those
functions, and the ctypes structures have the C layout.  No compute calls
(there is no GPU here)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "swpic.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(swpic_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_21794_gb300 import build, swpic
    build.build()
    return swpic.load_library()


def test_header_declares_the_paper_boundary():
    names = declared_functions()
    for required in ("swpic_init_particles", "swpic_deposit", "swpic_solve_field",
                     "swpic_gather_push", "swpic_step", "swpic_diagnostics"):
        assert required in names


def test_library_exports_every_declared_function(lib):
    out = subprocess.run(["nm", "-D", "--defined-only",
                          os.path.join(ROOT, "paper_2605_21794_gb300", "_build", "libswpic.so")],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(swpic_[a-z_0-9]+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_binding_covers_exactly_the_header():
    from paper_2605_21794_gb300 import swpic
    assert sorted(swpic.SIGNATURES) == declared_functions()


def test_struct_layouts_match_c(tmp_path):
    from paper_2605_21794_gb300 import swpic
    src = tmp_path / "layout.c"
    src.write_text('''
#include <stdio.h>
#include <stddef.h>
#include "swpic.h"
int main(void) {
  printf("%zu %zu %zu\\n", sizeof(swpic_config), sizeof(swpic_diag), sizeof(swpic_lattice));
  printf("%zu %zu %zu\\n", offsetof(swpic_config, diag_capacity), offsetof(swpic_diag, step),
         offsetof(swpic_lattice, decorate));
  printf("%d %d\\n", SWPIC_ABI_VERSION, SWPIC_NX_MAX);
  return 0;
}''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    sizes = [int(x) for x in lines[0].split()]
    offs = [int(x) for x in lines[1].split()]
    assert sizes == [C.sizeof(swpic.swpic_config), C.sizeof(swpic.swpic_diag),
                     C.sizeof(swpic.swpic_lattice)]
    assert offs == [swpic.swpic_config.diag_capacity.offset, swpic.swpic_diag.step.offset,
                    swpic.swpic_lattice.decorate.offset]
    assert [int(x) for x in lines[2].split()] == [1, swpic.SWPIC_NX_MAX]


def test_status_strings_and_version_without_gpu(lib):
    assert lib.swpic_abi_version() == 1
    assert lib.swpic_status_string(0) == b"ok"
    assert lib.swpic_status_string(5).startswith(b"numeric")


def test_create_rejects_bad_configs_before_touching_the_device(lib):
    from paper_2605_21794_gb300 import swpic
    ctx = swpic._CTX()
    bad = [swpic.make_config(-1.0, 0.1, 64), swpic.make_config(1.0, 0.0, 64),
           swpic.make_config(1.0, 0.1, 1), swpic.make_config(1.0, 0.1, swpic.SWPIC_NX_MAX + 1),
           swpic.make_config(1.0, 0.1, 64, precision=16),
           swpic.make_config(1.0, 0.1, 64, threads_per_block=100)]
    for cfg in bad:
        assert lib.swpic_create(C.byref(cfg), 10, C.byref(ctx)) == swpic.SWPIC_EINVAL
    cfg = swpic.make_config(1.0, 0.1, 64)
    assert lib.swpic_create(C.byref(cfg), -1, C.byref(ctx)) == swpic.SWPIC_EINVAL
    off = (C.c_int64 * 3)(0, 5, 3)          # decreasing offsets
    cfgs = (swpic.swpic_config * 2)(cfg, cfg)
    assert lib.swpic_create_batch(cfgs, 2, off, C.byref(ctx)) == swpic.SWPIC_EINVAL


def test_null_context_is_rejected(lib):
    from paper_2605_21794_gb300 import swpic
    assert lib.swpic_step(None, 1, 0) == swpic.SWPIC_EINVAL
    assert lib.swpic_deposit(None) == swpic.SWPIC_EINVAL
    lib.swpic_destroy(None)
