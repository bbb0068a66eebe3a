"""CPU-only checks of the C-ABI library: it builds for sm_103a, loads, and
exports every entry point include/dfvrb.h declares; the binding declares the
same names; the oracle and the CUDA path share no code."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^(?:dfv_status|const char \*)\s*(dfv_\w+)\s*\(", txt, flags=re.M)
    return names


def test_header_declares_the_documented_calls():
    names = set(declared_functions())
    for required in ("dfv_create_grid", "dfv_add_material", "dfv_set_fields", "dfv_set_body", "dfv_compute_dt",
                     "dfv_step", "dfv_get_fields", "dfv_get_body", "dfv_destroy", "dfv_last_error"):
        assert required in names


def test_library_builds_loads_and_exports_every_symbol():
    from paper_2111_11806_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_2111_11806_gb300 import binding
    assert set(declared_functions()) <= set(binding.EXPORTS)


def test_oracle_and_cuda_path_are_independent():
    """No import, include or link between oracle/ and the package."""
    pkg = os.path.join(ROOT, "paper_2111_11806_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"\boracle\b", txt.replace("the oracle", "")), fn
    for fn in os.listdir(os.path.join(ROOT, "oracle")):
        if fn.endswith((".py", ".c", ".h")):
            txt = open(os.path.join(ROOT, "oracle", fn)).read()
            assert "paper_2111_11806_gb300" not in txt and "dfvrb" not in txt, fn


def test_product_fails_loudly_without_library(tmp_path):
    from paper_2111_11806_gb300 import binding
    with pytest.raises(binding.DfvError):
        binding._lib = None
        binding.load(str(tmp_path / "missing.so"))
    binding._lib = None


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C compiler's size
    and field offsets (a field added on one side only fails here)."""
    from paper_2111_11806_gb300 import binding
    structs = {"dfv_options": binding.dfv_options, "dfv_material_params": binding.dfv_material_params,
               "dfv_instance_desc": binding.dfv_instance_desc}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dfvrb.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = dict(line.rsplit(" ", 1) for line in subprocess.check_output([str(exe)]).decode().splitlines())
    for name, cls in structs.items():
        assert int(out[name + " sizeof"]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(out[name + " " + field]) == getattr(cls, field).offset, (name, field)
