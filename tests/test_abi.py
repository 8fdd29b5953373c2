"""The C-ABI library builds, loads and exports every function that
include/piko_raster.h declares (no GPU needed; nothing is computed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(piko_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_core_entry_points():
    names = declared_functions()
    for n in ("piko_raster_create", "piko_raster_forward", "piko_raster_backward", "piko_raster_destroy"):
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1404_6293_gb300 import build
    path = build.build_library()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_header_compiles_as_plain_c():
    src = "#include <piko_raster.h>\nint main(void){ piko_scene s; piko_framebuffer f; (void)s; (void)f; return 0; }\n"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-I", os.path.join(ROOT, "include"),
                        "-x", "c", "-"], input=src, text=True, capture_output=True)
    assert r.returncode == 0, r.stderr


def test_struct_layout_matches_binding():
    from paper_1404_6293_gb300 import _lib as L
    assert ctypes.sizeof(L.PikoScene) == 4 * 4 + 6 * 8 + 2 * 4
    assert ctypes.sizeof(L.PikoFramebuffer) == 4 * 8


def test_binding_constants_match_the_header():
    """Every integer #define of the header that the binding names has the
    header's value, and the binding names every option and error code."""
    from paper_1404_6293_gb300 import _lib as L
    text = open(os.path.join(ROOT, "include", "piko_raster.h")).read()
    defines = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(PIKO_\w+)\s+(-?\d+)\b", text)}
    assert defines, "no integer defines found"
    for name, value in defines.items():
        if hasattr(L, name):
            assert getattr(L, name) == value, name
    for name in defines:
        if name.startswith(("PIKO_OPT_", "PIKO_ERR_", "PIKO_SCHED_", "PIKO_SHADE_")):
            assert hasattr(L, name), f"binding lacks {name}"
