"""CPU checks of the C ABI: the library builds, loads and exports exactly
the entry points that include/nmodl_b300.h declares (no compute calls)."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"NMODL_API[^;(]*?\b(nmodl_\w+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    from paper_1905_02241_b300 import build
    lib = build.build()
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib], text=True)
    exported = set(re.findall(r"\bT (nmodl_\w+)", out))
    decl = declared()
    assert decl, "no declarations found"
    assert decl <= exported, decl - exported
    assert exported <= decl, exported - decl
    L = ctypes.CDLL(lib)
    for n in decl:
        assert getattr(L, n) is not None


def test_binding_covers_declarations_and_host_calls():
    from paper_1905_02241_b300 import _lib
    assert set(_lib.EXPORTED) == declared()
    assert _lib.nmodl_version() == 100
    assert _lib.nmodl_strerror(-2).startswith("node_index")
    o = _lib.nmodl_options_default()
    assert o.window == 40 and o.newton_max_iter == 8 and o.newton_tol == 1e-14


def test_header_compiles_as_c():
    src = '#include "nmodl_b300.h"\nint main(void){nmodl_options o; return nmodl_options_default(&o);}\n'
    p = subprocess.run(["gcc", "-x", "c", "-std=c99", "-Wall", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), "-"], input=src, text=True,
                       capture_output=True)
    assert p.returncode == 0, p.stderr


def test_product_package_has_no_route_to_the_oracle():
    """The shipped package (library, binding, workloads) imports, loads and
    names nothing under oracle/: parity claims rest on the two sharing no
    code.  Only tests, the smoke check and the bench's CPU legs use it."""
    pkg = os.path.join(ROOT, "paper_1905_02241_b300")
    pat = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b)|liboracle|nmodl_oracle",
                     re.M)
    hits = []
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                p = os.path.join(dirpath, fn)
                if pat.search(open(p, errors="replace").read()):
                    hits.append(os.path.relpath(p, ROOT))
    assert not hits, hits
