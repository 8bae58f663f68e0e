"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/geoflood.h declares; the binding refuses to run without
the library (no CPU fallback).  No compute calls here."""
import ctypes
import os
import subprocess

import pytest

from paper_2403_15435_gb300 import _build, geoflood


@pytest.fixture(scope="module")
def libpath():
    return _build.build()


def test_library_exports_every_declared_symbol(libpath):
    names = geoflood.exported_symbols()
    assert "geoflood_init_forest" in names and "geoflood_step" in names
    out = subprocess.check_output(["nm", "-D", "--defined-only", libpath]).decode()
    defined = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in names if n not in defined]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for n in names:
        assert hasattr(lib, n)


def test_build_targets_sm_103a_only():
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_config_struct_matches_header():
    """The binding's struct has the header's field order."""
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "geoflood.h")).read()
    body = hdr[hdr.index("typedef struct {"):hdr.index("} geoflood_config;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b([a-z_0-9]+)(?:\[\d+\])?[,;]", body)
    assert [f[0] for f in geoflood._Cfg._fields_] == fields


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(geoflood, "_LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(geoflood, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        geoflood.lib()


def test_advance_stats_struct_matches_header():
    """The binding's advance statistics have the header's fields, in order
    and with the header's types (counts as long long, times as double)."""
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "geoflood.h")).read()
    end = hdr.index("} geoflood_advance_stats;")
    body = hdr[hdr.rindex("typedef struct {", 0, end):end]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        m = re.match(r"\s*(long long|double)\s+(.*)", decl.replace("typedef struct {", ""))
        if m:
            fields += [(n.strip(), m.group(1)) for n in m.group(2).split(",")]
    ctype = {"long long": ctypes.c_longlong, "double": ctypes.c_double}
    assert [(n, ctype[t]) for n, t in fields] == list(geoflood.AdvanceStats._fields_)
