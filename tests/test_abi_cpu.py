"""C-ABI checks that need no GPU: the library loads, exports every function
declared in include/slos.h, and its host-side Fock ranking is bit-exact
against the oracle's brute-force enumeration."""
import math
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for mt in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                              text, flags=re.M):
            names.add(mt.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2602_11092_gb300 import buildlib as pkg_build
    pkg_build.build()
    from paper_2602_11092_gb300 import binding
    return binding.load()


def test_library_exports_every_declared_function(lib):
    names = header_functions()
    assert "slos_forward" in names and "mesh_unitary" in names
    for name in names:
        assert hasattr(lib, name), f"libslos.so does not export {name}"
    from paper_2602_11092_gb300 import binding, surrogate
    assert set(binding.exported_symbols()) | set(surrogate.symbols()) >= set(names)


@pytest.mark.parametrize("m", range(2, 13))
def test_host_rank_matches_enumeration(lib, m):
    from paper_2602_11092_gb300 import binding
    for k in range(0, 7):
        states = oracle.enumerate_fock(m, k)
        if states.shape[0] > 20000:
            states = states[:: max(1, states.shape[0] // 5000)]
            idx = np.arange(0, oracle.fock_dim(m, k), max(1, oracle.fock_dim(m, k) // 5000))[: states.shape[0]]
        else:
            idx = np.arange(states.shape[0])
        for r, t in zip(idx, states):
            assert binding.host_rank(m, t) == r
            assert binding.host_unrank(m, k, int(r)) == list(t)


def test_host_rank_large_sample(lib):
    from paper_2602_11092_gb300 import binding
    m, k = 20, 10
    total = math.comb(m + k - 1, k)
    rng = np.random.default_rng(0)
    pos = np.sort(rng.choice(total, size=300, replace=False))
    pos = np.concatenate([[0], pos, [total - 1]])
    states = oracle.enumerate_fock(m, k, pos)
    for r, t in zip(pos, states):
        assert binding.host_rank(m, t) == r
        assert binding.host_unrank(m, k, int(r)) == list(t)


def test_plan_argument_validation_without_gpu(lib):
    from paper_2602_11092_gb300 import binding
    with pytest.raises(binding.SlosError) as e:
        binding.Plan(25, [1] + [0] * 24)
    assert e.value.status == 2
    with pytest.raises(binding.SlosError) as e:
        binding.Plan(4, [1, 1, 0, 0], detection=7)
    assert e.value.status == 1
    with pytest.raises(binding.SlosError) as e:
        binding.Plan(4, [13, 0, 0, 0])
    assert e.value.status == 2
    with pytest.raises(binding.SlosError) as e:
        binding.host_unrank(5, 3, 10 ** 6)
    assert e.value.status == 1


@pytest.mark.parametrize("m,k", [(2, 1), (2, 5), (3, 3), (6, 3), (8, 4), (12, 6), (16, 4), (16, 8), (24, 3)])
def test_transition_graph_matches_enumeration(lib, m, k):
    """The plan's transition tables (Sec. II-A.3) against brute-force
    enumeration: CSR parent entries of every child, child table of every
    parent, all indices in range."""
    from paper_2602_11092_gb300 import binding
    from paper_2602_11092_gb300 import binding
    rowptr, entries, ctab = binding.host_transition_table(m, k)
    child = oracle.enumerate_fock(m, k)
    parent = oracle.enumerate_fock(m, k - 1)
    Fk, Fp = child.shape[0], parent.shape[0]
    assert rowptr[0] == 0 and rowptr[-1] == m * Fp == entries.size
    assert np.all(np.diff(rowptr) >= 1)
    pidx = (entries >> 6).astype(np.int64)
    mode = ((entries >> 1) & 31).astype(np.int64)
    last = (entries & 1).astype(bool)
    assert pidx.max() < Fp and mode.max() < m
    assert np.array_equal(np.nonzero(last)[0], rowptr[1:] - 1)
    # expected: for child c, the nonzero modes in increasing order, parent = rank(t - e_j)
    pkey = {tuple(t): i for i, t in enumerate(parent)}
    ckey = {tuple(t): i for i, t in enumerate(child)}
    step = max(1, Fk // 4000)
    for c in range(0, Fk, step):
        t = child[c]
        js = np.nonzero(t)[0]
        seg = slice(rowptr[c], rowptr[c + 1])
        assert list(mode[seg]) == list(js)
        for j, pi in zip(js, pidx[seg]):
            tt = t.copy(); tt[j] -= 1
            assert pkey[tuple(tt)] == pi
    stepp = max(1, Fp // 4000)
    assert ctab.min() >= 0 and ctab.max() < Fk
    for cp in range(0, Fp, stepp):
        for j in range(m):
            tt = parent[cp].copy(); tt[j] += 1
            assert ctab[cp, j] == ckey[tuple(tt)]


def test_dram_traffic_figures_are_used_only_for_the_sources_they_were_taken_on():
    """bench.py reports the dominant kernel's DRAM bytes from the committed ncu
    capture only while the single-shape kernel sources hash to what the
    capture records; after a kernel change it reports null until the next
    capture."""
    import json
    import os
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench

    d = json.load(open(os.path.join(root, "profiles", "slos_final_layers_train16_dram_traffic.json")))
    assert d["command"].startswith("python bench.py") and "--clock-control none" in d["command"]
    fresh = d["csrc_hash"] == bench.csrc_hash()
    for kernel in ("slos_bwd_final", "slos_fwd_final"):
        recorded = d["kernels"][kernel]["dram_bytes_per_launch"]
        assert recorded > 0
        assert bench.ncu_traffic(kernel) == (recorded if fresh else None), kernel


def test_surrogate_failure_rate_bound():
    """The one-sided Clopper-Pearson bound the checked inference decides with:
    closed form 1 - alpha^(1/n) with no failures, the beta quantile
    otherwise, and 1 when every check failed."""
    import scipy.stats

    from paper_2602_11092_gb300.surrogate import SurrogateLayer as S
    for n in (64, 512, 1024):
        assert abs(S.failure_rate_bound(0, n, 0.99) - (1 - 0.01 ** (1 / n))) < 1e-9
        for k in (1, 3, 10):
            ref = scipy.stats.beta.ppf(0.99, k + 1, n - k)
            assert abs(S.failure_rate_bound(k, n, 0.99) - ref) < 1e-7
    assert S.failure_rate_bound(7, 7) == 1.0
    # a clean spot check of 1024 rows passes a 1 % bound, one of 64 cannot
    assert S.failure_rate_bound(0, 1024) <= 0.01 < S.failure_rate_bound(0, 64)


def _slot_table(m, k):
    """Fixed-width slot rows (parent << 5 | mode, padded with 24) of layer k,
    formed from the library's CSR transition graph."""
    from paper_2602_11092_gb300 import binding
    rowptr, entries, ctab = binding.host_transition_table(m, k)
    kw = ((min(m, k) + 3) // 4) * 4
    Fk = rowptr.size - 1
    slots = np.full((Fk, kw), 24, dtype=np.uint32)
    for c in range(Fk):
        seg = entries[rowptr[c]:rowptr[c + 1]]
        slots[c, :seg.size] = ((seg >> 6) << 5) | ((seg >> 1) & 31)
    return kw, slots, np.ascontiguousarray(ctab.astype(np.int32))


@pytest.mark.parametrize("m,k", [(6, 3), (8, 5), (12, 4)])
def test_host_table_validation_rejects_corrupted_tables(lib, m, k):
    """The range check every plan runs before uploading its tables accepts the
    real tables and rejects each kind of corruption, naming the entry."""
    kw, slots, ctab = _slot_table(m, k)

    def check(sl, ct):
        return lib.slos_host_validate_tables(m, k, kw, sl.ctypes.data, ct.ctypes.data)

    assert check(slots, ctab) == 0
    Fp = ctab.shape[0]
    Fk = slots.shape[0]
    bad = slots.copy(); bad[Fk // 2, 0] = (Fp << 5) | (bad[Fk // 2, 0] & 31)   # parent past layer k-1
    assert check(bad, ctab) == 6 and b"out of range" in lib.slos_last_error()
    bad = slots.copy(); bad[3, 0] = (bad[3, 0] & ~np.uint32(31)) | m            # mode past the last one
    assert check(bad, ctab) == 6
    bad = slots.copy(); bad[Fk - 1, :] = 24                                     # a state with no parent
    assert check(bad, ctab) == 6 and b"no parent" in lib.slos_last_error()
    badc = ctab.copy(); badc[Fp - 1, m - 1] = Fk                                # child past layer k
    assert check(slots, badc) == 6
    badc = ctab.copy(); badc[0, 0] = -1                                         # no holes in the Fock lattice
    assert check(slots, badc) == 6
