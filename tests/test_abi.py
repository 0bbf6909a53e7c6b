"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/lbfluct.h declares; host-side argument checks work without a GPU
(no compute call is made here)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbfluct.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_0803_2826_gb300 import build, lbfluct
    build.build()
    return lbfluct


def test_header_declares_binding_exports(lib):
    assert _declared() == sorted(lib.EXPORTS)


def test_header_constants_match_binding(lib):
    """Every numeric #define of the header has the same value in the binding."""
    defs = dict(re.findall(r"#define\s+(LB_\w+)\s+(0x[0-9a-fA-F]+|\d+)u?\b", open(HEADER).read()))
    assert {"LB_DERR_FENE_BROKEN", "LB_NSUMS", "LB_COUPLE_PER_SUBSTEP"} <= set(defs)
    for name, val in defs.items():
        assert getattr(lib, name) == int(val, 0), name


def test_library_exports_every_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    have = set(re.findall(r"\bT (lb_\w+)", out))
    missing = [s for s in _declared() if s not in have]
    assert not missing, missing
    raw = lib.load()
    for s in _declared():
        assert hasattr(raw, s)


def test_version_and_sizes(lib):
    assert "sm_103a" in lib.lb_version()
    p = lib.make_params((5, 6, 7))
    assert lib.lb_plane_pitch(p) == 256  # 210 rounded up to a multiple of 64
    assert lib.lb_population_bytes(p) == 19 * 256 * 4
    p16 = lib.make_params((5, 6, 7), dtype=lib.LB_F16)
    assert lib.lb_population_bytes(p16) == 19 * 256 * 2


@pytest.mark.parametrize("kw,msg", [
    (dict(gamma_shear=1.0), "gamma"),
    (dict(rho0=0.0), "rho0"),
    (dict(kT=-1.0), "kT"),
    (dict(dtype=7), "dtype"),
])
def test_params_rejected(lib, kw, msg):
    p = lib.make_params((4, 4, 4), **kw)
    assert lib.lb_population_bytes(p) == 0
    assert msg in lib.lb_last_error()
    h = C.c_void_p()
    st = lib.load().lb_create(C.byref(p), 256, 512, None, None, C.byref(h))
    assert st == lib.LB_EINVAL and not h.value


def test_bad_geometry_rejected(lib):
    raw = lib.load()
    h = C.c_void_p()
    p = lib.make_params((4, 4, 2), walls=True)
    assert raw.lb_create(C.byref(p), 256, 512, None, None, C.byref(h)) == lib.LB_EINVAL
    assert "nz >= 3" in lib.lb_last_error()
    p = lib.make_params((0, 4, 4))
    assert raw.lb_create(C.byref(p), 256, 512, None, None, C.byref(h)) == lib.LB_EINVAL
    p = lib.make_params((4, 4, 4))
    assert raw.lb_create(C.byref(p), 256, 256, None, None, C.byref(h)) == lib.LB_EINVAL
    assert raw.lb_create(C.byref(p), 256, 300, None, None, C.byref(h)) == lib.LB_EINVAL
    assert "aligned" in lib.lb_last_error()


def test_null_handles_rejected(lib):
    raw = lib.load()
    assert raw.lb_step(None, 1) == lib.LB_EINVAL
    assert raw.lb_moments(None, None, None, None, None) == lib.LB_EINVAL
    assert raw.lb_destroy(None) == lib.LB_OK
    assert raw.lb_noise_words(0, 0, 0, 0, 0, 4, 5, None, None, None) == lib.LB_EINVAL


def test_struct_layouts_match_header(lib, tmp_path):
    """Size and every field offset of the ABI structs, from the C compiler
    (gcc on include/lbfluct.h) against the ctypes binding."""
    import shutil
    if not shutil.which("gcc"):
        pytest.skip("gcc not found")
    structs = [lib.lb_params, lib.lb_particles, lib.lb_couple_params, lib.lb_spheres, lib.lb_batch_config]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lbfluct.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append('printf("%%zu\\n", sizeof(%s));' % name)
        for field in st._fields_:
            lines.append('printf("%%zu\\n", offsetof(%s, %s));' % (name, field[0]))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = []
    for st in structs:
        want.append(C.sizeof(st))
        want += [getattr(st, f[0]).offset for f in st._fields_]
    assert got == want


def test_index_checking_variant_compiles(tmp_path):
    """The LB_DEBUG_BOUNDS variant (index checks before every population pull
    and store) compiles for sm_103a: the fused stream-collide unit."""
    from paper_0803_2826_gb300 import build as B
    src = os.path.join(B.CSRC, "sc_f32.cu")
    cmd = [B.nvcc(), *B.ARCH, *B.NVCC_FLAGS, "-DLB_DEBUG_BOUNDS", "-c", src, "-o", str(tmp_path / "sc.o")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
