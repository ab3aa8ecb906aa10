"""Split-lattice tables (head/tail blocks of the transition graph, Sec. II-A.3)
checked on the CPU, bit for bit.

The tables are built by the library's host code; these tests walk them the way
the split kernels do (4-state runs, head-block descriptors, tail slot and
child rows) and compare every parent and child index that a kernel would form
with the plain transition graph of the same layer, which is itself pinned
against brute-force enumeration (test_abi_cpu.py).  They also check that every
index a kernel forms stays inside the buffer it addresses.
"""
import math

import numpy as np
import pytest

from paper_2602_11092_gb300 import binding

EMPTY = 24  # padding slot: parent 0, the zero row of U
CHUNK = 4  # states per warp run (the chunk tables' granularity)

# (m, n): head/tail splits of 6 + 2, 6 + 6, 8 + 5 and 8 + 8 modes
SHAPES = [(8, 4), (12, 5), (13, 4), (16, 4), (16, 8)]


@pytest.fixture(scope="module")
def lib():
    return binding.load()


def _layers(m, n):
    return [k for k in range(2, n + 1)]


@pytest.mark.parametrize("m,n", SHAPES)
def test_split_forward_walk_matches_transition_graph(lib, m, n):
    tail = binding.host_split_tail(m, n)
    h = tail["h"]
    mL = m - h
    slots = tail["slots"]
    for k in _layers(m, n):
        if k == n and (m, n) == (16, 8):
            step = 29  # every 29th run of the 490314-state layer
        else:
            step = 1
        L = binding.host_split_layer(m, n, k)
        assert L["h"] == h
        Fk, Fp = math.comb(m + k - 1, k), math.comb(m + k - 2, k - 1)
        rowptr, entries, _ = binding.host_transition_table(m, k)
        fdesc, fhead, fchunk = L["fdesc"], L["fhead"], L["fchunk"]
        # blocks tile the layer in rank order
        assert fdesc[0, 0] == 0
        assert np.array_equal(fdesc[1:, 0], fdesc[:-1, 0] + fdesc[:-1, 1])
        assert fdesc[-1, 0] + fdesc[-1, 1] == Fk
        assert fchunk.size == (Fk + CHUNK - 1) // CHUNK
        for ch in range(0, fchunk.size, step):
            c0, cend = ch * CHUNK, min(ch * CHUNK + CHUNK, Fk)
            b, c = int(fchunk[ch]), c0
            while c < cend:
                base, size, zb, w = (int(x) for x in fdesc[b])
                assert base <= c < base + size
                stop = min(base + size, cend)
                rho, qh = w & 255, (w >> 8) & 15
                assert 0 <= qh <= 8 and qh <= min(h, k)
                hoff = [(int(fhead[b, q]) >> 5) - base for q in range(qh)]
                hmode = [int(fhead[b, q]) & 31 for q in range(qh)]
                W = int(tail["tw"][rho])
                tr = int(tail["soff"][rho]) + (c - base) * W
                if W:
                    assert 0 <= zb and zb < Fp  # padding slots read parent row zb
                for cc in range(c, stop):
                    got = [(cc + hoff[q], hmode[q]) for q in range(qh)]
                    if W:
                        assert tr + W <= slots.size
                        for e in slots[tr:tr + W]:
                            e = int(e)
                            if e == EMPTY:
                                continue
                            assert h <= (e & 31) < m
                            got.append((zb + (e >> 5), e & 31))
                        tr += W
                    for p, _ in got:
                        assert 0 <= p < Fp
                    seg = entries[rowptr[cc]:rowptr[cc + 1]]
                    want = [(int(e >> 6), int((e >> 1) & 31)) for e in seg]
                    assert sorted(got, key=lambda x: x[1]) == want, (m, n, k, cc)
                c = stop
                b += 1
        assert mL >= 1


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


def test_split_tail_rows_are_padded_and_aligned(lib):
    for m, n in SHAPES:
        t = binding.host_split_tail(m, n)
        mL = m - t["h"]
        for rho in range(n + 1):
            W = int(t["tw"][rho])
            assert W == (0 if rho == 0 else ((min(mL, rho) + 3) & ~3))
            assert int(t["soff"][rho]) % 4 == 0  # 16-byte row loads
        # a tail state with q occupied modes has exactly q slots before the padding
        rho = n
        W = int(t["tw"][rho])
        rows = t["slots"][int(t["soff"][rho]):].reshape(-1, W)[:math.comb(rho + mL - 1, mL - 1)]
        occupied = (rows != EMPTY).sum(1)
        assert occupied.min() >= 1 and occupied.max() <= min(mL, rho)
        # padding only after the occupied slots
        for r in rows[:200]:
            nz = list(r != EMPTY)
            assert nz == sorted(nz, reverse=True)


def test_split_eligibility(lib):
    with pytest.raises(binding.SlosError):
        binding.host_split_tail(6, 3)       # too few modes to split
    with pytest.raises(binding.SlosError):
        binding.host_split_tail(20, 6)      # tail wider than 8 modes
    assert binding.host_split_tail(16, 8)["h"] == 8
    assert binding.host_split_tail(12, 6)["h"] == 6
