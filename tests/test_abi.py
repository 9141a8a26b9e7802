"""The C ABI without a GPU: the library builds, loads, exports every function
include/nam.h declares, and the binding's ctypes structures have the C
layout (checked against sizeof/offsetof from a C compiler)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nam.h")


@pytest.fixture(scope="module")
def libnam():
    from paper_2305_02678_gb300 import _build
    _build.build()
    from paper_2305_02678_gb300 import binding
    return binding


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w[\w\s\*]*?\b(nam_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("nam_init", "nam_create_material", "nam_eval", "nam_train_step", "nam_submit", "nam_poll"):
        assert required in names


def test_every_declared_symbol_is_exported(libnam):
    lib = libnam.lib()
    names = _declared_functions()
    assert names, "no declarations parsed"
    for n in names:
        assert hasattr(lib, n), f"{n} declared in nam.h but not exported"
    assert set(names) == set(libnam.EXPORTS)


def test_exported_symbols_via_nm(libnam):
    from paper_2305_02678_gb300._build import LIB
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(nam_\w+)", out))
    assert set(_declared_functions()) <= exported


def test_status_strings_without_gpu(libnam):
    assert libnam.nam_status_string(0) == "ok"
    assert libnam.nam_status_string(libnam.NAM_ERR_BUDGET) == "HBM budget exceeded"
    assert libnam.nam_status_string(12345) == "unknown status"


def test_struct_layouts_match_c(libnam, tmp_path):
    structs = {
        "nam_config": libnam.nam_config,
        "nam_material_desc": libnam.nam_material_desc,
        "nam_material_info": libnam.nam_material_info,
        "nam_queries": libnam.nam_queries,
        "nam_work_item": libnam.nam_work_item,
        "nam_adam": libnam.nam_adam,
        "nam_frame": libnam.nam_frame,
        "nam_frame_stats": libnam.nam_frame_stats,
        "nam_stats": libnam.nam_stats,
        "nam_sphere": libnam.nam_sphere,
        "nam_scene": libnam.nam_scene,
        "nam_gbuffer": libnam.nam_gbuffer,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            k, v = line.rsplit(" ", 1)
            got[k] = int(v)
    for name, cls in structs.items():
        assert got[f"{name} size"] == C.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert got[f"{name}.{fname}"] == getattr(cls, fname).offset, f"{name}.{fname}"


def _header_constants():
    """Names of the #define and enum constants of nam.h (NAM_*)."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    names = set(re.findall(r"^#define\s+(NAM_[A-Z0-9_]+)\s+\S", src, flags=re.M))
    for body in re.findall(r"enum\s*\{(.*?)\}", src, flags=re.S):
        names |= set(re.findall(r"\b(NAM_[A-Z0-9_]+)\s*=", body))
    return sorted(names)


def test_binding_constants_match_header(libnam, tmp_path):
    """Every NAM_* constant the binding defines has the header's value (the
    values printed by a C compiler, so that the header is read as C reads it)."""
    names = [n for n in _header_constants() if hasattr(libnam, n)]
    assert len(names) >= 30, names
    lines = ["#include <stdio.h>", f'#include "{HEADER}"', "int main(void) {"]
    for n in names:
        lines.append(f'  printf("{n} %lld\\n", (long long)({n}));')
    lines.append("  return 0; }")
    src = tmp_path / "consts.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-std=c11", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in out:
        if line.strip():
            k, v = line.rsplit(" ", 1)
            assert getattr(libnam, k) == int(v), (k, getattr(libnam, k), v)


def test_init_without_gpu_fails_cleanly(libnam):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(libnam.NamError) as e:
        libnam.nam_init(0)
    assert e.value.status in (libnam.NAM_ERR_CUDA, libnam.NAM_ERR_INVALID_ARG)


def test_every_entry_point_refuses_null_arguments(libnam):
    """Each entry point checks its context (and other pointers) before any
    CUDA call: with every pointer NULL and every integer 0 it returns
    NAM_ERR_INVALID_ARG and leaves a message, on a machine without a GPU."""
    import ctypes as C
    lib = libnam.lib()
    for name in libnam.EXPORTS:
        if name in ("nam_status_string", "nam_last_error_message", "nam_now"):
            continue
        f = getattr(lib, name)
        st = f(*[None if t is C.c_void_p else 0 for t in f.argtypes])
        assert st == libnam.NAM_ERR_INVALID_ARG, (name, st)
        assert lib.nam_last_error_message().decode(), name
