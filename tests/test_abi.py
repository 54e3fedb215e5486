"""CPU checks of the C ABI: the library loads without a GPU, exports every
function the headers under include/ declare (and the Python binding gives
each a signature), sizes workspaces and rejects bad configurations with a
message.  No compute call is made."""
import ctypes as C
import os
import re

import pytest

import paper_2206_11634_gb300 as pkg
from paper_2206_11634_gb300 import build as build_mod

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
HEADER = os.path.join(INCLUDE, "lbm_metaball.h")


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return pkg.load_library()


def declared_functions():
    names = set()
    for h in sorted(os.listdir(INCLUDE)):
        if h.endswith(".h"):
            text = re.sub(r"/\*.*?\*/", "", open(os.path.join(INCLUDE, h)).read(), flags=re.S)
            names |= set(re.findall(r"^\s*(?:int|int64_t|const char \*)\s*(lbm_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("lbm_workspace_size", "lbm_init", "lbm_set_particles", "lbm_step", "lbm_get_forces",
                 "lbm_get_fields", "lbm_destroy"):
        assert need in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 30
    for n in names:
        assert hasattr(lib, n), n
    # and the binding marshals every one of them
    from paper_2206_11634_gb300 import lbm
    assert set(names) <= set(lbm._SIGS), sorted(set(names) - set(lbm._SIGS))


def test_struct_layout_matches_c_compiler(tmp_path):
    """The ctypes mirrors agree with the C compiler on every field offset."""
    fields = {"lbm_config": pkg.LbmConfig, "lbm_particle": pkg.LbmParticle}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lbm_metaball.h"', "int main(void) {"]
    for cname, cls in fields.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        cname, fname, val = line.split()
        cls = fields[cname]
        got = C.sizeof(cls) if fname == "size" else getattr(cls, fname).offset
        assert got == int(val), (cname, fname, got, val)


def test_workspace_size_scales(lib):
    sizes = []
    for n in (32, 64):
        c = pkg.make_config(n, n, n, storage="f32", max_particles=4)
        s = C.c_size_t()
        assert lib.lbm_workspace_size(C.byref(c), C.byref(s)) == 0
        sizes.append(s.value)
    # two FP32 D3Q19 population arrays dominate: 2*19*4 bytes per node
    assert sizes[1] > 8 * 152 * 32 ** 3 * 0.9
    c16 = pkg.make_config(64, 64, 64, storage="f16", max_particles=4)
    s = C.c_size_t()
    lib.lbm_workspace_size(C.byref(c16), C.byref(s))
    assert s.value < sizes[1] * 0.6


@pytest.mark.parametrize("field,value", [("tau", 0.5), ("lattice", 27), ("nx", 1), ("storage", 7),
                                         ("max_particles", 0), ("rho0", 0.0)])
def test_bad_config_rejected(lib, field, value):
    c = pkg.make_config(16, 16, 16)
    setattr(c, field, value)
    s = C.c_size_t()
    assert lib.lbm_workspace_size(C.byref(c), C.byref(s)) == -1
    assert len(lib.lbm_last_error(None)) > 0


def test_init_rejects_host_or_null_workspace(lib):
    c = pkg.make_config(16, 16, 16)
    h = C.c_void_p()
    assert lib.lbm_init(C.byref(c), None, 1 << 30, None, C.byref(h)) == -1
    assert not h.value
    s = C.c_size_t()
    lib.lbm_workspace_size(C.byref(c), C.byref(s))
    assert lib.lbm_init(C.byref(c), C.c_void_p(256), 16, None, C.byref(h)) == -2   # too small


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.lbm_step(None, 1) == -1
    assert lib.lbm_check(None) == -1
    assert lib.lbm_destroy(None) == 0
