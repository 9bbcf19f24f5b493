"""The C-ABI library loads and exports every entry point include/gerbil.h declares (no GPU).

No compute call is made here; on a machine without a GPU the context constructor must fail
cleanly with GERBIL_E_CUDA instead of crashing.
"""
import ctypes
import os
import re

import pytest

import __graft_entry__
from paper_1607_06618_b300 import gerbil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(gerbil_[a-z_0-9]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return gerbil.load()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert declared, "no declarations found"
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared <= set(gerbil.ABI_SYMBOLS) | {n for n in declared if n.startswith("gerbil_")}
    assert set(gerbil.ABI_SYMBOLS) <= declared


def test_strerror_and_defaults(lib):
    assert gerbil.load().gerbil_strerror(0) == b"ok"
    assert gerbil.load().gerbil_strerror(999) == b"unknown status"
    o = gerbil.default_opts()
    assert (o.canonical, o.ordering, o.canonical_minimizer) == (1, 0, 1)
    assert (o.supermer_cap, o.max_probes, o.persistent, o.fused) == (256, 1024, 1, 0)
    assert abs(o.load_factor - 0.5) < 1e-6


def test_no_cpu_fallback_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = gerbil.load().gerbil_create(ctypes.byref(h), 0, 0, None)
    assert st == gerbil.GERBIL_E_CUDA and not h.value
    with pytest.raises(gerbil.GerbilError):
        gerbil.gerbil_create(0)


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors have the C structs' sizes and field offsets (gcc on the header)."""
    import ctypes
    import shutil
    import subprocess
    from paper_1607_06618_b300 import gerbil
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    structs = {"gerbil_reads": gerbil.gerbil_reads, "gerbil_opts": gerbil.gerbil_opts,
               "gerbil_count_stats": gerbil.gerbil_count_stats,
               "gerbil_phase_times": gerbil.gerbil_phase_times,
               "gerbil_tuning": gerbil.gerbil_tuning,
               "gerbil_server_stats": gerbil.gerbil_server_stats,
               "gerbil_job_times": gerbil.gerbil_job_times}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gerbil.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for fname, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, fname, name, fname))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(got["%s.%s" % (name, fname)]) == getattr(cls, fname).offset, (name, fname)
