"""Pure-Python brute force for tiny inputs -- TEST INFRASTRUCTURE ONLY.

A second, independent restatement of the definitions in kmer_oracle.cpp, written with Python
strings and dicts.  It exists to pin the C++ oracle: on tiny random inputs the two must agree
exactly.  Nothing here is fast; keep inputs to a few thousand bases.
"""
from __future__ import annotations

_COMP = {"A": "T", "C": "G", "G": "C", "T": "A"}


def revcomp(s: str) -> str:
    """Sec. 2.4.2: reverse, then swap A<->T and C<->G."""
    return "".join(_COMP[c] for c in reversed(s))


def reads_from(seq: bytes, offsets) -> list[str]:
    return [seq[int(offsets[i]):int(offsets[i + 1])].decode("latin-1")
            for i in range(len(offsets) - 1)]


def _clean(window: str) -> str | None:
    up = window.upper()
    return up if all(c in "ACGT" for c in up) else None


def count(reads: list[str], k: int, canonical: bool = True, min_count: int = 1) -> dict[str, int]:
    hist: dict[str, int] = {}
    for r in reads:
        for i in range(len(r) - k + 1):
            x = _clean(r[i:i + k])
            if x is None:
                continue
            if canonical:
                x = min(x, revcomp(x))
            hist[x] = hist.get(x, 0) + 1
    return {key: c for key, c in hist.items() if c >= min_count}


def value(s: str) -> int:
    v = 0
    for c in s:
        v = 4 * v + "ACGT".index(c)
    return v


def kmc2_demoted(s: str) -> bool:
    return s.startswith("AAA") or s.startswith("ACA") or ("AA" in s[1:])


def rank(s: str, ordering: str = "kmc2") -> int:
    if ordering == "lex":
        return value(s)
    return value(s) + (4 ** len(s) if kmc2_demoted(s) else 0)


def minimizer(kmer: str, m: int, ordering: str = "kmc2", canonical_min: bool = True) -> str:
    """The m-mer of smallest rank in a k-mer (Sec. 2.1), after optional canonicalisation."""
    cands = []
    for q in range(len(kmer) - m + 1):
        s = kmer[q:q + m]
        if canonical_min:
            s = min(s, revcomp(s))
        cands.append(s)
    return min(cands, key=lambda s: rank(s, ordering))


def supermers(read: str, k: int, m: int, ordering: str = "kmc2", canonical_min: bool = True,
              lmax: int = 10 ** 9, base_offset: int = 0) -> list[tuple[int, str, str]]:
    """(global start, super-mer string, minimizer) for one read, by Fig. 1's definition."""
    out: list[tuple[int, str, str]] = []
    prev = None  # minimizer of the previous counted window, None if it was not counted
    for p in range(len(read) - k + 1):
        x = _clean(read[p:p + k])
        if x is None:
            prev = None
            continue
        mz = minimizer(x, m, ordering, canonical_min)
        g = base_offset + p
        if prev is None or mz != prev or g % lmax == 0:
            out.append((g, x, mz))
        else:
            start, s, z = out[-1]
            out[-1] = (start, s + x[-1], z)
        prev = mz
    return out
