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
HEADERS = [os.path.join(ROOT, "include", h) for h in ("swpic.h", "swpic2d.h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(swpic(?:2d)?_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


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
    exported = set(re.findall(r"\sT\s(swpic(?:2d)?_[a-z_0-9]+)$", out, flags=re.M))
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
  printf("%d %d %d\\n", SWPIC_ABI_VERSION, SWPIC_NX_MAX, SWPIC_STATIC_NX_MAX);
  printf("%d %d %d\\n", SWPIC_FIELD_SOLVE_AUTO, SWPIC_FIELD_SOLVE_LAST_CTA, SWPIC_FIELD_SOLVE_AT_START);
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
    assert [int(x) for x in lines[2].split()] == [1, swpic.SWPIC_NX_MAX, swpic.SWPIC_STATIC_NX_MAX]
    assert [int(x) for x in lines[3].split()] == [swpic.SWPIC_FIELD_SOLVE_AUTO, swpic.SWPIC_FIELD_SOLVE_LAST_CTA,
                                                  swpic.SWPIC_FIELD_SOLVE_AT_START]


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
    assert lib.swpic_set_field_solve(None, 0) == swpic.SWPIC_EINVAL
    assert lib.swpic_deposit(None) == swpic.SWPIC_EINVAL
    lib.swpic_destroy(None)


def test_2d_struct_layouts_match_c(tmp_path):
    from paper_2605_21794_gb300 import swpic
    src = tmp_path / "layout2d.c"
    src.write_text('''
#include <stdio.h>
#include <stddef.h>
#include "swpic2d.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(swpic2d_config), sizeof(swpic2d_diag),
         offsetof(swpic2d_config, diag_capacity), offsetof(swpic2d_diag, step));
  return 0;
}''')
    exe = tmp_path / "layout2d"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got == [C.sizeof(swpic.swpic2d_config), C.sizeof(swpic.swpic2d_diag),
                   swpic.swpic2d_config.diag_capacity.offset, swpic.swpic2d_diag.step.offset]


def test_2d_create_rejects_bad_configs_before_touching_the_device(lib):
    from paper_2605_21794_gb300 import swpic
    ctx = swpic._CTX()

    def cfg(**kw):
        base = dict(Lx=1.0, Ly=1.0, dt=0.1, nx=16, ny=16, precision=32, decorated=1,
                    threads_per_block=0, blocks_per_sm=0, diag_capacity=0, reserved=0)
        base.update(kw)
        return swpic.swpic2d_config(*base.values())
    bad = [cfg(Lx=-1.0), cfg(Ly=0.0), cfg(dt=0.0), cfg(nx=12), cfg(ny=2), cfg(nx=2048),
           cfg(nx=128, ny=128), cfg(precision=64, nx=128, ny=64), cfg(precision=16),
           cfg(threads_per_block=100), cfg(threads_per_block=1024), cfg(diag_capacity=-1)]
    for c in bad:
        assert lib.swpic2d_create(C.byref(c), 10, C.byref(ctx)) == swpic.SWPIC_EINVAL
    assert lib.swpic2d_create(C.byref(cfg()), -1, C.byref(ctx)) == swpic.SWPIC_EINVAL
    assert lib.swpic2d_step(None, 1, 0) == swpic.SWPIC_EINVAL
    assert lib.swpic2d_save(None, b"x") == swpic.SWPIC_EINVAL
    assert lib.swpic2d_load(None, b"x") == swpic.SWPIC_EINVAL
    assert lib.swpic2d_refresh(None) == swpic.SWPIC_EINVAL
    lib.swpic2d_destroy(None)


def test_2d_lattice_struct_layout_matches_c(tmp_path):
    from paper_2605_21794_gb300 import swpic
    src = tmp_path / "lat2d.c"
    src.write_text('''
#include <stdio.h>
#include <stddef.h>
#include "swpic2d.h"
int main(void) {
  printf("%zu %zu %zu\\n", sizeof(swpic2d_lattice), offsetof(swpic2d_lattice, vmin),
         offsetof(swpic2d_lattice, decorate));
  return 0;
}''')
    exe = tmp_path / "lat2d"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == [C.sizeof(swpic.swpic2d_lattice), swpic.swpic2d_lattice.vmin.offset,
                   swpic.swpic2d_lattice.decorate.offset]
