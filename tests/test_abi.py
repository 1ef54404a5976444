"""The C-ABI library builds for sm_103a and exports every entry point that
include/ddm.h declares (no GPU needed: loading runs no kernel)."""
import os
import re

import paper_1812_05087_gb300.ddm as ddm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "ddm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:ddm_status|void|const char \*)\s*\*?\s*(ddm_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("ddm_build_tree", "ddm_matvec", "ddm_history_apply", "ddm_gmres_solve", "ddm_sif"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ddm.load()
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(header_functions()) <= set(ddm.EXPORTS) | {"ddm_submit", "ddm_poll"}


def test_header_compiles_standalone_as_c_and_cpp(tmp_path):
    """A C or C++ caller includes ddm.h on its own: it must bring every type
    it uses (size_t, int64_t) and declare the functions with C linkage."""
    import shutil
    import subprocess
    hdr = os.path.join(ROOT, "include", "ddm.h")
    for comp, args in (("gcc", ["-x", "c", "-std=c99"]), ("g++", ["-x", "c++"])):
        if shutil.which(comp) is None:
            continue
        r = subprocess.run([comp, "-fsyntax-only", "-Wall", "-Werror", *args, hdr], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes mirror in the binding has the size and field offsets of
    the C struct it stands for (a field added on one side only would shift
    every later field silently)."""
    import shutil
    import subprocess
    import ctypes
    if shutil.which("gcc") is None:
        return
    structs = [n for n in dir(ddm) if n.startswith("ddm_") and isinstance(getattr(ddm, n), type)
               and issubclass(getattr(ddm, n), ctypes.Structure)]
    assert {"ddm_fmm_params", "ddm_tree_info", "ddm_material", "ddm_request"} <= set(structs)
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{os.path.join(ROOT, "include", "ddm.h")}"',
             "int main(void) {"]
    for s in structs:
        lines.append(f'    printf("{s} size %zu\\n", sizeof({s}));')
        for f, _ in getattr(ddm, s)._fields_:
            lines.append(f'    printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    r = subprocess.run(["gcc", "-std=c99", "-o", str(exe), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = [ln for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
           if ln]
    assert len(out) == sum(1 + len(getattr(ddm, s)._fields_) for s in structs)
    for line in out:
        s, f, v = line.split()
        cls = getattr(ddm, s)
        got = ctypes.sizeof(cls) if f == "size" else getattr(cls, f).offset
        assert got == int(v), (s, f, got, v)


def test_tree_kind_values():
    """The binding maps the tree kind onto ddm_fmm_params.adaptive and
    rejects anything else before it reaches the library."""
    import pytest
    assert [ddm._tree_kind(v) for v in (False, True, "auto", 0, 1, 2)] == [0, 1, 2, 0, 1, 2]
    for bad in ("yes", 3, -1, None):
        with pytest.raises(ValueError):
            ddm._tree_kind(bad)
