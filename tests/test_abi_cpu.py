"""Host-side checks of the C ABI that need no GPU: the library builds and loads, exports
every entry point include/gcpush.h declares, its structures have the header's layout
(compiled C offsets vs the ctypes mirrors), and errors come back as status codes."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2403_06706_gb300 import gcpush

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gcpush.h")


@pytest.fixture(scope="module")
def lib():
    gcpush.build()
    return gcpush.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(gc_\w+)\s*\(", text, re.M)))


def test_exports_every_declared_function(lib):
    names = declared_functions()
    assert len(names) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", gcpush.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gc_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert set(gcpush.EXPORTS) == set(names)
    for n in names:
        assert hasattr(lib, n)


STRUCTS = {
    "gc_options": gcpush.Options, "gc_grid_desc": gcpush.GridDesc,
    "gc_ensemble_desc": gcpush.EnsembleDesc, "gc_tally_desc": gcpush.TallyDesc,
    "gc_tally_out": gcpush.TallyOut, "gc_particle_soa": gcpush.ParticleSoA,
    "gc_stats_out": gcpush.StatsOut,
}


def test_struct_layouts_match_header(tmp_path):
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void){"]
    for cname, cls in STRUCTS.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n"):
        if line:
            a, b, v = line.split()
            got[(a, b)] = int(v)
    for cname, cls in STRUCTS.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_errors_are_status_codes(lib):
    assert lib.gc_version() >= 100
    assert lib.gc_create(None, None) == -1
    assert b"null" in lib.gc_last_error()
    o = gcpush.Options()
    o.precision = 7
    h = ctypes.c_void_p()
    assert lib.gc_create(ctypes.byref(h), ctypes.byref(o)) == -1
    assert lib.gc_advance(None, 0.5, 1, 0.0) == -1
    assert lib.gc_stats(None, None) == -1


def test_create_without_gpu_fails_cleanly(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(gcpush.GcError) as e:
        gcpush.Context()
    assert e.value.code == -2
