"""The C-ABI library builds, loads and exports every entry point the header
declares (no GPU needed; no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                             src, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names) - {"if", "while", "for", "return"})


@pytest.fixture(scope="module")
def lib():
    from paper_1906_08125_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("mesh_load", "inject", "push_relocate", "deposit", "poisson_solve", "pic_step",
                 "pic_adjoint", "pic_create", "pic_destroy", "pic_get_particles",
                 "pic_set_particles"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), f"libpicfem does not export {name}"


def test_binding_covers_the_exports(lib):
    from paper_1906_08125_gb300 import picfem
    assert set(picfem.EXPORTED) == set(_declared_functions())


def test_version_string(lib):
    lib.pic_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.pic_version()


def test_null_arguments_are_rejected(lib):
    """Argument checks run on the host before any CUDA call."""
    lib.pic_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.pic_create(None, None, None) == -1
    lib.pic_last_error.restype = ctypes.c_char_p
    lib.pic_last_error.argtypes = [ctypes.c_void_p]
    assert b"null" in lib.pic_last_error(None)
    lib.pic_adjoint.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p]
    assert lib.pic_adjoint(None, 1, 20, None, None, None) == -1
    lib.pic_set_applied_field.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.pic_set_applied_field(None, None) == -1


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1906_08125_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "picfem_oracle" not in src, f


STRUCTS = {"pic_params": "Params", "pic_step_stats": "StepStats", "pic_info": "MeshInfo",
           "pic_tuning": "Tuning"}


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    the C compiler gives the header's struct, and the default parameters
    marshal into it."""
    import shutil
    import subprocess
    from paper_1906_08125_gb300 import configs, picfem
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "picfem.h"', "int main(void) {"]
    for cname, pyname in STRUCTS.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in getattr(picfem, pyname)._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, pyname in STRUCTS.items():
        cls = getattr(picfem, pyname)
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)
    picfem._params(configs.params())
