"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and exports
every entry point that include/amnerf.h declares (no GPU calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "amnerf.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"AMNERF_API\s+[\w\s\*]*?\b(amnerf_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("amnerf_create", "amnerf_build_tree", "amnerf_load_mlps", "amnerf_render", "amnerf_destroy"):
        assert must in names


def test_library_loads_and_exports_every_declared_symbol():
    from paper_2310_01881_gb300 import build
    lib = ctypes.CDLL(build.build())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_uses_the_same_names():
    from paper_2310_01881_gb300 import amnerf
    for n in _declared():
        if n in ("amnerf_status_string", "amnerf_last_error"):
            continue
        assert hasattr(amnerf, n), n


def test_status_strings_without_a_gpu():
    from paper_2310_01881_gb300 import amnerf
    lib = amnerf.load()
    assert lib.amnerf_status_string(0) == b"ok"
    assert lib.amnerf_status_string(6) == b"device wait timed out"
    ctx = ctypes.c_void_p()
    # no GPU in this container: creation must fail cleanly, not crash
    st = lib.amnerf_create(ctypes.byref(ctx), 0, None)
    assert st in (0, amnerf.E_DEVICE)
    if st == 0:
        lib.amnerf_destroy(ctx)


def test_struct_layouts_match_the_binding(tmp_path):
    """Every struct of include/amnerf.h has the size and field offsets that the ctypes
    binding assumes (gcc compiles a probe that prints sizeof and offsetof)."""
    import json
    import shutil
    import subprocess

    import pytest
    from paper_2310_01881_gb300 import amnerf
    if not shutil.which("gcc"):
        pytest.skip("gcc not found")
    structs = ["amnerf_tree_params", "amnerf_node", "amnerf_mlp_desc", "amnerf_render_params", "amnerf_tuning",
               "amnerf_stats", "amnerf_debug"]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "amnerf.h"', "int main(void) {",
             '    printf("{");']
    for i, name in enumerate(structs):
        cls = getattr(amnerf, name)
        parts = [f'\\"size\\": %zu'] + [f'\\"{f}\\": %zu' for f, _ in cls._fields_]
        args = [f"sizeof({name})"] + [f"offsetof({name}, {f})" for f, _ in cls._fields_]
        sep = "," if i + 1 < len(structs) else ""
        lines.append(f'    printf("\\"{name}\\": {{{", ".join(parts)}}}{sep}", {", ".join(args)});')
    lines += ['    printf("}\\n");', "    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = json.loads(subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout)
    for name in structs:
        cls = getattr(amnerf, name)
        assert got[name]["size"] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[name][f] == getattr(cls, f).offset, (name, f)
