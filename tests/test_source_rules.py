"""Source-level rules of the CUDA path (no GPU): kernels report failures through an error word
and bounded waits, never by trapping; the library is built for sm_103a alone."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1607_06618_b300", "csrc")


def _sources():
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(CSRC, name)) as f:
                yield name, f.read()


def test_no_trap_or_device_assert():
    for name, text in _sources():
        assert "__trap" not in text, name
        assert re.search(r"\bassert\s*\(", text) is None, name
        assert "<cassert>" not in text and "<assert.h>" not in text, name


def test_every_nanosleep_spin_has_a_bound():
    """A loop that sleeps between polls also compares against a limit (an iteration count or
    %globaltimer) within a few lines of the sleep."""
    for name, text in _sources():
        lines = text.splitlines()
        for i, line in enumerate(lines):
            if "__nanosleep" not in line:
                continue
            window = "\n".join(lines[max(0, i - 8): i + 3])
            assert re.search(r"limit|wait_ns|globaltimer", window), (name, i + 1)


def test_built_for_sm_103a_only():
    with open(os.path.join(ROOT, "paper_1607_06618_b300", "build.py")) as f:
        text = f.read()
    arches = set(re.findall(r"arch=compute_(\w+),code=sm_(\w+)", text))
    assert arches == {("103a", "103a")}, arches
