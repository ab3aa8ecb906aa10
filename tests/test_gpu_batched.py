"""Uneven batches in one persistent launch (slos_batched_*), against the
single-shape path and the FP64 oracle."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2602_11092_gb300 import workloads

pytestmark = pytest.mark.gpu

P_TOL = 1e-5


def pack(Us, dev="cuda"):
    flat = np.concatenate([np.asarray(U, dtype=np.complex64).reshape(-1) for U in Us])
    return torch.tensor(flat, dtype=torch.complex64, device=dev)


def make_plan(slos, inst):
    ms = [it.m for it in inst]
    ns = [it.n for it in inst]
    det = [slos.THRESHOLD if it.threshold else slos.PNR for it in inst]
    return slos.BatchedPlan(ms, ns, [it.s for it in inst], det)


def small_uneven(rng, count=70):
    inst = []
    for i in range(count):
        m = int(rng.integers(3, 11))
        n = int(rng.integers(1, min(5, m) + 1))
        s = [0] * m
        for q in rng.choice(m, size=n, replace=True):
            s[q] += 1
        inst.append(workloads.UnevenInstance(m=m, n=n, s=s, threshold=bool(rng.integers(0, 2))))
    return inst


def test_batched_matches_single_shape_plans(slos):
    rng = np.random.default_rng(31)
    inst = small_uneven(rng)
    Us = [workloads.haar_unitaries(it.m, 1, rng)[0] for it in inst]
    bp = make_plan(slos, inst)
    ws = torch.empty(bp.workspace_bytes, dtype=torch.uint8, device="cuda")
    out = torch.full((bp.out_offsets[-1],), float("nan"), dtype=torch.float32, device="cuda")
    bp.forward(pack(Us), out, ws)
    bp.sync_status()
    out = out.cpu().numpy()
    for i, it in enumerate(inst):
        plan = slos.Plan(it.m, it.s, slos.THRESHOLD if it.threshold else slos.PNR)
        ref = plan.forward(torch.tensor(Us[i][None], dtype=torch.complex64, device="cuda")).cpu().numpy()[0]
        got = out[bp.out_offsets[i]:bp.out_offsets[i + 1]]
        assert got.shape == ref.shape
        assert np.abs(got - ref).max() <= P_TOL
    # oracle on a few
    for i in range(0, len(inst), 9):
        it = inst[i]
        Uq = np.asarray(Us[i], dtype=np.complex64).astype(np.complex128)
        outs = oracle.enumerate_fock(it.m, it.n)
        p = oracle.probabilities(Uq, it.s, outs)
        ref = oracle.threshold_probs(p, outs, it.m, it.n) if it.threshold else p
        got = out[bp.out_offsets[i]:bp.out_offsets[i + 1]]
        assert np.abs(got - ref).max() <= P_TOL


@pytest.mark.parametrize("det", ["pnr", "threshold"])
def test_batched_edge_shapes(slos, det):
    """More photons than modes, two modes, one photon, bunched inputs, and
    shapes with 1, 16 and 17 instances (one lane group, a full one, one
    more) against single-shape plans and the oracle."""
    rng = np.random.default_rng(41)
    thr = det == "threshold"
    specs = [(2, [3, 0], 1), (2, [1, 1], 3), (3, [2, 2, 1], 16), (4, [0, 7, 0, 0], 1), (5, [1, 0, 0, 0, 0], 17),
             (6, [2, 0, 1, 0, 0, 3], 2), (20, [1] * 3 + [0] * 17, 1)]
    inst = []
    for m, s, cnt in specs:
        inst += [workloads.UnevenInstance(m=m, n=sum(s), s=list(s), threshold=thr)] * cnt
    order = rng.permutation(len(inst))
    inst = [inst[i] for i in order]
    Us = [workloads.haar_unitaries(it.m, 1, rng)[0] for it in inst]
    bp = make_plan(slos, inst)
    ws = torch.empty(bp.workspace_bytes, dtype=torch.uint8, device="cuda")
    out = torch.full((bp.out_offsets[-1],), float("nan"), dtype=torch.float32, device="cuda")
    bp.forward(pack(Us), out, ws)
    bp.sync_status()
    out = out.cpu().numpy()
    for i, it in enumerate(inst):
        got = out[bp.out_offsets[i]:bp.out_offsets[i + 1]]
        plan = slos.Plan(it.m, it.s, slos.THRESHOLD if thr else slos.PNR)
        ref = plan.forward(torch.tensor(Us[i][None], dtype=torch.complex64, device="cuda")).cpu().numpy()[0]
        assert got.shape == ref.shape
        assert np.abs(got - ref).max() <= P_TOL
        Uq = np.asarray(Us[i], dtype=np.complex64).astype(np.complex128)
        outs = oracle.enumerate_fock(it.m, it.n)
        p = oracle.probabilities(Uq, it.s, outs)
        refo = oracle.threshold_probs(p, outs, it.m, it.n) if thr else p
        assert np.abs(got - refo).max() <= P_TOL


def test_uneven_full_workload_against_oracle(slos):
    """The 1024-instance workload (m in 8..20, n in 2..min(10, m/2), threshold
    for m >= 16): normalisation of every instance, and seeded outputs of the
    largest instances against the oracle."""
    inst, Us = workloads.uneven()
    bp = make_plan(slos, inst)
    ws = torch.empty(bp.workspace_bytes, dtype=torch.uint8, device="cuda")
    out = torch.empty((bp.out_offsets[-1],), dtype=torch.float32, device="cuda")
    bp.forward(pack(Us), out, ws)
    bp.sync_status()
    out = out.cpu().numpy()
    tot = np.array([out[bp.out_offsets[i]:bp.out_offsets[i + 1]].astype(np.float64).sum() for i in range(len(inst))])
    assert np.abs(tot - 1.0).max() < 2e-4
    order = sorted(range(len(inst)), key=lambda i: -workloads.fock_dim(inst[i].m, inst[i].n))
    rng = np.random.default_rng(5)
    for i in order[:3] + order[-2:]:
        it = inst[i]
        Uq = np.asarray(Us[i], dtype=np.complex64).astype(np.complex128)
        got = out[bp.out_offsets[i]:bp.out_offsets[i + 1]]
        if it.threshold:
            pats = oracle.threshold_patterns(it.m, it.n)
            for idx in rng.choice(len(pats), size=12, replace=False):
                ref = oracle.threshold_prob_of_pattern(Uq, it.s, pats[idx])
                assert abs(got[idx] - ref) <= P_TOL
        else:
            K = workloads.fock_dim(it.m, it.n)
            pos = np.sort(rng.choice(K, size=min(K, 200), replace=False))
            ref = oracle.probabilities(Uq, it.s, oracle.enumerate_fock(it.m, it.n, pos))
            assert np.abs(got[pos] - ref).max() <= P_TOL


def test_uneven_workload_every_shape_against_oracle(slos):
    """One instance of every (m, n, detection) shape of the 1024-instance
    workload against the oracle.  Full outputs where the Fock space has at most
    2e5 states (every PNR shape, and threshold shapes whose pattern sums the
    oracle can form from the full distribution): max |dp| <= 1e-5 and
    TV <= 1e-5.  Larger threshold shapes: 40 seeded patterns (and the first and
    last) summed by the oracle state by state."""
    inst, Us = workloads.uneven()
    bp = make_plan(slos, inst)
    ws = torch.empty(bp.workspace_bytes, dtype=torch.uint8, device="cuda")
    out = torch.empty((bp.out_offsets[-1],), dtype=torch.float32, device="cuda")
    bp.forward(pack(Us), out, ws)
    bp.sync_status()
    out = out.cpu().numpy()
    first = {}
    for i, it in enumerate(inst):
        first.setdefault((it.m, it.n, it.threshold), i)
    assert len(first) >= 70
    rng = np.random.default_rng(11)
    full = 0
    for (m, n, thr), i in sorted(first.items()):
        it = inst[i]
        Uq = np.asarray(Us[i], dtype=np.complex64).astype(np.complex128)
        got = out[bp.out_offsets[i]:bp.out_offsets[i + 1]].astype(np.float64)
        K = workloads.fock_dim(m, n)
        if K <= 200_000:
            outs = oracle.enumerate_fock(m, n)
            p = oracle.probabilities(Uq, it.s, outs)
            ref = oracle.threshold_probs(p, outs, m, n) if thr else p
            d = np.abs(got - ref)
            assert d.max() <= P_TOL, (m, n, thr, d.max())
            assert 0.5 * d.sum() <= 1e-5, (m, n, thr, 0.5 * d.sum())
            full += 1
        else:
            assert thr
            pats = oracle.threshold_patterns(m, n)
            idx = np.unique(np.concatenate([[0, len(pats) - 1], rng.choice(len(pats), size=40, replace=False)]))
            for j in idx:
                ref = oracle.threshold_prob_of_pattern(Uq, it.s, pats[j])
                assert abs(got[j] - ref) <= P_TOL, (m, n, j)
    assert full >= 50


def test_batched_graph_capture_and_replay(slos):
    rng = np.random.default_rng(8)
    inst = small_uneven(rng, 40)
    Us = [workloads.haar_unitaries(it.m, 1, rng)[0] for it in inst]
    bp = make_plan(slos, inst)
    ws = torch.empty(bp.workspace_bytes, dtype=torch.uint8, device="cuda")
    U = pack(Us)
    eager = torch.empty((bp.out_offsets[-1],), dtype=torch.float32, device="cuda")
    bp.forward(U, eager, ws)
    out = torch.zeros_like(eager)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            bp.forward(U, out, ws, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(3):
        out.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, eager)
    bp.sync_status()


def test_batched_autotune_and_cache(slos, tmp_path):
    rng = np.random.default_rng(9)
    inst = small_uneven(rng, 50)
    Us = [workloads.haar_unitaries(it.m, 1, rng)[0] for it in inst]
    bp = make_plan(slos, inst)
    ws = torch.empty(bp.workspace_bytes, dtype=torch.uint8, device="cuda")
    U = pack(Us)
    ref = torch.empty((bp.out_offsets[-1],), dtype=torch.float32, device="cuda")
    bp.forward(U, ref, ws)
    cache = str(tmp_path / "autotune.json")
    bp.autotune(U, torch.empty_like(ref), ws, cache_path=cache)
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 1
    entry = json.loads(lines[0])
    assert entry["chunk"] in (64, 128, 256, 512) and entry["threads"] in (128, 256)
    out = torch.empty_like(ref)
    bp.forward(U, out, ws)
    # every output is one fixed-order sum, whatever the launch shape
    assert torch.equal(out, ref)
    # a second plan with the same shapes reads the cache instead of timing
    bp2 = make_plan(slos, inst)
    bp2.autotune(U, torch.empty_like(ref), ws, cache_path=cache)
    assert len(open(cache).read().strip().splitlines()) == 1
    bp2.forward(U, out, ws)
    assert torch.equal(out, ref)


def test_bounded_wait_reports_timeout_and_context_survives(slos):
    """Fault injection without a GPU fault: one layer's completion counter is
    made unreachable; the waits give up after ~1 ms and the status word says
    SLOS_ERR_TIMEOUT; the next normal launch works."""
    rng = np.random.default_rng(10)
    inst = small_uneven(rng, 40)
    Us = [workloads.haar_unitaries(it.m, 1, rng)[0] for it in inst]
    bp = make_plan(slos, inst)
    ws = torch.empty(bp.workspace_bytes, dtype=torch.uint8, device="cuda")
    U = pack(Us)
    out = torch.empty((bp.out_offsets[-1],), dtype=torch.float32, device="cuda")
    bp.inject_stall(True)
    bp.forward(U, out, ws)
    with pytest.raises(slos.SlosError) as e:
        bp.sync_status()
    assert e.value.status == 5
    bp.inject_stall(False)
    bp.forward(U, out, ws)
    bp.sync_status()
    ref = torch.empty_like(out)
    bp.forward(U, ref, ws)
    assert torch.equal(out, ref)


def test_batched_widest_slot_rows(slos):
    """States with 11 or 12 occupied modes (m=12, n=11 and n=12) take the
    launcher's widest slot rows (12 slots; layers are sorted by occupied-mode
    count): against single-shape plans on every output and the oracle on
    sampled outputs and patterns."""
    rng = np.random.default_rng(57)
    specs = [(12, [1] * 11 + [0], False, 2), (12, [1] * 12, True, 1), (12, [2] + [1] * 10 + [0], False, 1)]
    inst = []
    for m, s, thr, cnt in specs:
        inst += [workloads.UnevenInstance(m=m, n=sum(s), s=list(s), threshold=thr)] * cnt
    Us = [workloads.haar_unitaries(it.m, 1, rng)[0] for it in inst]
    bp = make_plan(slos, inst)
    ws = torch.empty(bp.workspace_bytes, dtype=torch.uint8, device="cuda")
    out = torch.full((bp.out_offsets[-1],), float("nan"), dtype=torch.float32, device="cuda")
    bp.forward(pack(Us), out, ws)
    bp.sync_status()
    out = out.cpu().numpy()
    for i, it in enumerate(inst):
        got = out[bp.out_offsets[i]:bp.out_offsets[i + 1]]
        plan = slos.Plan(it.m, it.s, slos.THRESHOLD if it.threshold else slos.PNR)
        ref = plan.forward(torch.tensor(Us[i][None], dtype=torch.complex64, device="cuda")).cpu().numpy()[0]
        assert got.shape == ref.shape
        assert np.abs(got - ref).max() <= P_TOL
        Uq = np.asarray(Us[i], dtype=np.complex64).astype(np.complex128)
        if it.threshold:
            pats = oracle.threshold_patterns(it.m, it.n)
            for idx in list(rng.choice(len(pats), size=10, replace=False)) + [len(pats) - 1]:
                assert abs(got[idx] - oracle.threshold_prob_of_pattern(Uq, it.s, pats[idx])) <= P_TOL
        else:
            K = workloads.fock_dim(it.m, it.n)
            pos = np.sort(rng.choice(K, size=150, replace=False))
            refo = oracle.probabilities(Uq, it.s, oracle.enumerate_fock(it.m, it.n, pos))
            assert np.abs(got[pos] - refo).max() <= P_TOL
