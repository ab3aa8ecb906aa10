"""Split-lattice tables (head/tail blocks of the transition graph, Sec. II-A.3)
checked on the CPU, bit for bit.

The tables are built by the library's host code; these tests walk them the way
the split backward kernel does (4-parent runs, head-block descriptors, tail
child rows) and compare every child index that the kernel would form
with the plain transition graph of the same layer, which is itself pinned
against brute-force enumeration (test_abi_cpu.py).  They also check that every
index a kernel forms stays inside the buffer it addresses.
"""
import math

import numpy as np
import pytest

from paper_2602_11092_gb300 import binding

CHUNK = 4  # states per warp run (the chunk tables' granularity)

# (m, n): head/tail splits of 6 + 2, 6 + 6, 8 + 5 and 8 + 8 modes
SHAPES = [(8, 4), (12, 5), (13, 4), (16, 4), (16, 8)]


@pytest.fixture(scope="module")
def lib():
    return binding.load()


def _layers(m, n):
    return [k for k in range(2, n + 1)]


@pytest.mark.parametrize("m,n", SHAPES)
def test_split_backward_walk_matches_child_table(lib, m, n):
    tail = binding.host_split_tail(m, n)
    h = tail["h"]
    mL = m - h
    ctab_rows = tail["ctab"].reshape(-1, 8)
    for k in _layers(m, n):
        L = binding.host_split_layer(m, n, k)
        Fk, Fp = math.comb(m + k - 1, k), math.comb(m + k - 2, k - 1)
        _, _, ctab = binding.host_transition_table(m, k)
        bdesc, bhead, bchunk = L["bdesc"], L["bhead"], L["bchunk"]
        assert bdesc[0, 0] == 0
        assert np.array_equal(bdesc[1:, 0], bdesc[:-1, 0] + bdesc[:-1, 1])
        assert bdesc[-1, 0] + bdesc[-1, 1] == Fp
        assert bchunk.size == (Fp + CHUNK - 1) // CHUNK
        step = 17 if (m, n, k) == (16, 8, 8) else 1
        for ch in range(0, bchunk.size, step):
            c0, cend = ch * CHUNK, min(ch * CHUNK + CHUNK, Fp)
            b, c = int(bchunk[ch]), c0
            while c < cend:
                base, size, lc, rho = (int(x) for x in bdesc[b])
                assert base <= c < base + size and rho <= k - 1
                stop = min(base + size, cend)
                hoff = [int(bhead[b, j]) - base for j in range(h)]
                row = int(tail["coff"][rho]) + (c - base)
                for cc in range(c, stop):
                    assert row < ctab_rows.shape[0]
                    got = [cc + hoff[j] for j in range(h)] + [lc + int(ctab_rows[row, j]) for j in range(mL)]
                    assert all(0 <= x < Fk for x in got)
                    assert got == [int(x) for x in ctab[cc]], (m, n, k, cc)
                    row += 1
                c = stop
                b += 1


def _compositions_desc(parts, total):
    """All compositions of total into parts, in descending lexicographic order."""
    if parts == 1:
        return [(total,)]
    out = []
    for first in range(total, -1, -1):
        out += [(first,) + rest for rest in _compositions_desc(parts - 1, total - first)]
    return out


@pytest.mark.parametrize("m,n", [(8, 4), (12, 5), (16, 4)])
def test_split_tail_child_rows_by_enumeration(lib, m, n):
    """Row r of rho's block is the r-th tail composition of rho photons in
    descending-lex order; entry j is the position of t_L + e_j among the
    compositions of rho + 1 photons (enumerated here independently), and
    the entries past the m - h tail modes are 0."""
    t = binding.host_split_tail(m, n)
    mL = m - t["h"]
    rows = t["ctab"].reshape(-1, 8)
    assert int(t["coff"][0]) == 0 and int(t["coff"][n]) == rows.shape[0]
    for rho in range(n):
        comps = _compositions_desc(mL, rho)
        nxt = {c: i for i, c in enumerate(_compositions_desc(mL, rho + 1))}
        assert int(t["coff"][rho + 1]) - int(t["coff"][rho]) == len(comps)
        for r, c in enumerate(comps):
            row = rows[int(t["coff"][rho]) + r]
            want = [nxt[c[:j] + (c[j] + 1,) + c[j + 1:]] for j in range(mL)] + [0] * (8 - mL)
            assert [int(x) for x in row] == want, (m, n, rho, c)


def test_split_eligibility(lib):
    with pytest.raises(binding.SlosError):
        binding.host_split_tail(6, 3)       # too few modes to split
    with pytest.raises(binding.SlosError):
        binding.host_split_tail(20, 6)      # tail wider than 8 modes
    assert binding.host_split_tail(16, 8)["h"] == 8
    assert binding.host_split_tail(12, 6)["h"] == 6
