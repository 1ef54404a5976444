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
