"""The C ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/sedi.h declares; the Python binding's struct layouts
match the header (checked by compiling a probe against the header)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sedi.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1601_03801_gb300 import build
    build.build()
    from paper_1601_03801_gb300 import sedi
    return sedi.lib()


def declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sedi_[a-z_]+)\s*\(", txt)))


def test_header_declares_expected_entry_points():
    names = declared()
    for must in ("sedi_create", "sedi_set_particles", "sedi_set_fluid", "sedi_step", "sedi_average"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1601_03801_gb300 import sedi
    for name in declared():
        assert hasattr(lib, name), name
    assert sorted(sedi.EXPORTS) == declared()
    out = subprocess.run(["nm", "-D", "--defined-only", sedi.LIB_PATH], capture_output=True, text=True).stdout
    for name in declared():
        assert re.search(rf"\bT {name}\b", out), name


def test_struct_layout_matches_header(tmp_path, lib):
    from paper_1601_03801_gb300 import sedi
    probe = tmp_path / "probe.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sedi.h"', "int main(void){",
             'printf("%zu\\n", sizeof(sedi_params));', 'printf("%zu\\n", sizeof(sedi_stats));']
    for name, _ in sedi.SediParams._fields_:
        lines.append(f'printf("%zu\\n", offsetof(sedi_params, {name}));')
    lines.append("return 0;}")
    probe.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(probe), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(sedi.SediParams)
    assert vals[1] == ctypes.sizeof(sedi.SediStats)
    for (name, _), off in zip(sedi.SediParams._fields_, vals[2:]):
        assert getattr(sedi.SediParams, name).offset == off, name


def test_default_params_without_gpu(lib):
    from paper_1601_03801_gb300 import sedi
    p = sedi.default_params()
    assert p["precision_form"] == sedi.SEDI_FORM_SPLIT
    assert p["ncell"] == [10, 10, 20] and p["n_tau"] == 4 and p["nbr_capacity"] == 32
