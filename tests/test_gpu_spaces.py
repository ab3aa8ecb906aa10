"""Computation spaces and measurement strategies (Sec. II-A.3, QuantumLayer):
the collision-free (unbunched) space, per-mode photon-number expectations and
renormalisation, against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_11092_gb300 import workloads

pytestmark = pytest.mark.gpu

P_TOL = 1e-5
TV_TOL = 1e-5
G_TOL = 1e-3


def c64(U):
    return torch.tensor(np.asarray(U), dtype=torch.complex64, device="cuda")


def up(Ut):
    return Ut.detach().cpu().numpy().astype(np.complex128)


def check_dist(p_gpu, p_ref):
    d = np.abs(np.asarray(p_gpu, dtype=np.float64) - p_ref)
    assert d.max() <= P_TOL, f"max |dp| = {d.max():.3e}"
    assert 0.5 * d.sum() <= TV_TOL, f"TV = {0.5 * d.sum():.3e}"


UNB_CASES = [
    (6, [1, 1, 1, 0, 0, 0], 5),
    (12, [1, 0] * 6, 40),
    (8, [2, 0, 1, 0, 1, 0, 0, 0], 7),   # bunched input, collision-free outputs
    (5, [1, 1, 1, 1, 1], 3),            # n = m: one output
    (16, [1, 0] * 8, 33),               # 12870 outputs
    (9, [0, 0, 0, 0, 1, 0, 0, 0, 0], 4),  # one photon
]


@pytest.mark.parametrize("m,s,B", UNB_CASES)
def test_unbunched_forward_matches_oracle(slos, m, s, B):
    rng = np.random.default_rng(100 + m + B)
    U = c64(workloads.haar_unitaries(m, B, rng))
    plan = slos.Plan(m, s, space=slos.UNBUNCHED)
    outs = oracle.enumerate_unbunched(m, sum(s))
    assert plan.n_outputs == len(outs) == plan.fock_dim
    p = plan.forward(U).cpu().numpy()
    amps = plan.forward(U, slos.AMPS).cpu().numpy()
    layered = plan.forward(U, save_for_backward=True, workspace=plan.workspace(B, training=True)).cpu().numpy()
    Uh = up(U)
    for b in range(0, B, max(1, B // 6)):
        ref = oracle.probabilities(Uh[b], s, outs)
        check_dist(p[b], ref)
        check_dist(layered[b], ref)
        assert np.abs(amps[b] - oracle.amplitudes(Uh[b], s, outs)).max() <= P_TOL


def test_unbunched_equals_fock_restricted_to_collision_free(slos):
    m, s, B = 10, [1, 0, 1, 0, 1, 0, 1, 0, 0, 0], 64
    rng = np.random.default_rng(5)
    U = c64(workloads.haar_unitaries(m, B, rng))
    full = slos.Plan(m, s).forward(U).cpu().numpy()
    unb = slos.Plan(m, s, space=slos.UNBUNCHED).forward(U).cpu().numpy()
    keep = oracle.enumerate_fock(m, sum(s)).max(axis=1) <= 1
    assert np.abs(full[:, keep] - unb).max() <= 1e-6


def test_unbunched_rejects_bad_plans(slos):
    with pytest.raises(slos.SlosError):
        slos.Plan(3, [2, 1, 1], space=slos.UNBUNCHED)  # 4 photons, 3 modes
    with pytest.raises(slos.SlosError):
        slos.Plan(4, [1, 1, 0, 0], slos.THRESHOLD, space=slos.UNBUNCHED)


@pytest.mark.parametrize("m,s,B,shared", [
    (6, [1, 1, 1, 0, 0, 0], 5, True),
    (8, [2, 0, 1, 0, 1, 0, 0, 0], 7, False),
    (12, [1, 0] * 6, 9, True),
    (5, [1, 1, 1, 1, 1], 3, False),
    (16, [1, 0] * 3 + [0] * 10, 3, False),  # 16 modes: dU in tensor memory, holes in the child table
])
def test_unbunched_backward_matches_permanent_minors(slos, m, s, B, shared):
    rng = np.random.default_rng(200 + m)
    U = c64(workloads.haar_unitaries(m, B, rng))
    plan = slos.Plan(m, s, space=slos.UNBUNCHED)
    outs = oracle.enumerate_unbunched(m, sum(s))
    K = len(outs)
    c = rng.standard_normal(K) if shared else rng.standard_normal((B, K))
    ws = plan.workspace(B, training=True)
    plan.forward(U, save_for_backward=True, workspace=ws)
    dU = plan.backward(U, torch.tensor(c, dtype=torch.float32, device="cuda"), ws).cpu().numpy()
    Uh = up(U)
    for b in range(B):
        cb = c if shared else c[b]
        ref = oracle.grad_U_minors(Uh[b], s, cb.astype(np.float64), outs)
        assert np.linalg.norm(dU[b] - ref) / np.linalg.norm(ref) <= G_TOL


def test_unbunched_gradients_equal_fock_gradients_without_collision_outputs(slos):
    """The collision-free amplitudes are the Fock amplitudes on those outputs,
    so a loss on them has the same dL/dU on either lattice (probabilities and
    amplitudes, checkpointing on the collision-free plan)."""
    m, s, B = 9, [1, 0, 1, 0, 1, 0, 1, 0, 0], 40
    rng = np.random.default_rng(9)
    U = c64(workloads.haar_unitaries(m, B, rng))
    full = slos.Plan(m, s)
    unb = slos.Plan(m, s, space=slos.UNBUNCHED, mem_budget_bytes=1)
    assert unb.checkpoint_stride > 1
    keep = torch.tensor(oracle.enumerate_fock(m, sum(s)).max(axis=1) <= 1, device="cuda")
    for kind in (slos.PROBS, slos.AMPS):
        if kind == slos.PROBS:
            g = torch.tensor(rng.standard_normal((B, unb.n_outputs)), dtype=torch.float32, device="cuda")
            gf = torch.zeros((B, full.n_outputs), dtype=torch.float32, device="cuda")
        else:
            g = torch.tensor(rng.standard_normal((B, unb.n_outputs)) + 1j * rng.standard_normal((B, unb.n_outputs)),
                             dtype=torch.complex64, device="cuda")
            gf = torch.zeros((B, full.n_outputs), dtype=torch.complex64, device="cuda")
        gf[:, keep] = g
        res = []
        for plan, dout in ((unb, g), (full, gf)):
            ws = plan.workspace(B, training=True)
            plan.forward(U, kind, save_for_backward=True, workspace=ws)
            res.append(plan.backward(U, dout, ws, kind))
        rel = ((res[0] - res[1]).abs().norm() / res[1].abs().norm()).item()
        assert rel <= 1e-5


@pytest.mark.parametrize("m,s,det,space", [
    (8, [1, 0] * 4, 0, 0),
    (7, [1, 1, 0, 1, 0, 0, 0], 1, 0),
    (10, [1, 0] * 5, 0, 1),
    (5, [2, 0, 1, 0, 0], 0, 0),
])
def test_expectations_forward_and_backward(slos, m, s, det, space):
    rng = np.random.default_rng(300 + m)
    B = 6
    U = c64(workloads.haar_unitaries(m, B, rng))
    plan = slos.Plan(m, s, det, space=space)
    probs = plan.forward(U)
    E = plan.expectations(probs)
    n = sum(s)
    outs = oracle.enumerate_unbunched(m, n) if space == 1 else oracle.enumerate_fock(m, n)
    Uh = up(U)
    p64 = probs.double().cpu().numpy()
    for b in range(B):
        # the reduction itself, against FP64 sums of the same probabilities
        if det == 1:
            exact_sum = oracle.click_probabilities(p64[b], m, n)
        else:
            exact_sum = oracle.mode_expectations(p64[b], outs)
        assert np.abs(E[b].cpu().numpy() - exact_sum).max() <= 1e-5
        # and the physics: the oracle's distribution
        p_ref = oracle.probabilities(Uh[b], s, outs)
        if det == 1:
            ref = oracle.click_probabilities(oracle.threshold_probs(p_ref, outs, m, n), m, n)
        else:
            ref = oracle.mode_expectations(p_ref, outs)
        assert np.abs(E[b].cpu().numpy() - ref).max() <= 1e-4
        if det == 0 and space == 0:
            assert np.abs(E[b].cpu().numpy() - (np.abs(Uh[b]) ** 2) @ np.array(s, float)).max() <= 1e-4
    # backward: dprobs[b][t] = sum_j occ_j(t) dE[b][j]
    dE = torch.tensor(rng.standard_normal((B, m)), dtype=torch.float32, device="cuda")
    dp = plan.expectations_backward(dE).double().cpu().numpy()
    if det == 1:
        occ = np.zeros((plan.n_outputs, m))
        for i, b_ in enumerate(oracle.threshold_patterns(m, n)):
            occ[i, list(b_)] = 1.0
    else:
        occ = outs.astype(np.float64)
    assert np.abs(dp - dE.double().cpu().numpy() @ occ.T).max() <= 1e-5


def test_renormalise_forward_backward(slos):
    m, s, B = 8, [1, 0] * 4, 11
    rng = np.random.default_rng(17)
    U = c64(workloads.haar_unitaries(m, B, rng))
    plan = slos.Plan(m, s, space=slos.UNBUNCHED)
    p = plan.forward(U)
    q, Z = plan.renormalise(p)
    p64 = p.double().cpu().numpy()
    Zr = p64.sum(axis=1)
    assert np.abs(Z.double().cpu().numpy() - Zr).max() <= 1e-6
    assert np.abs(q.double().cpu().numpy() - p64 / Zr[:, None]).max() <= 1e-6
    Uh = up(U)
    for b in range(0, B, 5):
        ref = oracle.renormalise(oracle.probabilities(Uh[b], s, oracle.enumerate_unbunched(m, 4)))
        assert np.abs(q[b].double().cpu().numpy() - ref).max() <= 1e-4
    dq = torch.tensor(rng.standard_normal(p.shape), dtype=torch.float32, device="cuda")
    dp = plan.renormalise_backward(q, Z, dq).double().cpu().numpy()
    q64, dq64 = q.double().cpu().numpy(), dq.double().cpu().numpy()
    ref = (dq64 - (dq64 * q64).sum(axis=1, keepdims=True)) / Z.double().cpu().numpy()[:, None]
    assert np.abs(dp - ref).max() <= 1e-4 * np.abs(ref).max()
    # in place
    pc = p.clone()
    q2, _ = plan.renormalise(pc, q=pc)
    assert torch.equal(q2, q)


def test_layer_unbunched_renormalised_expectations_gradient(slos):
    """QuantumLayer(space=UNBUNCHED, renormalise=True, measurement=
    "expectations"): d loss / d phases through mesh, SLOS, renormalisation
    and expectations, against FP64 central differences of the oracle."""
    from paper_2602_11092_gb300.functions import QuantumLayer
    m, s, B = 6, [1, 0, 1, 0, 1, 0], 3
    rng = np.random.default_rng(21)
    mb = workloads.mesh_batch(m, B, seed=1000)
    layer = QuantumLayer(m, s, theta=torch.tensor(mb.theta, dtype=torch.float32),
                         w=torch.ones(m), space=slos.UNBUNCHED, renormalise=True, measurement="expectations")
    x = torch.tensor(mb.data, dtype=torch.float32, device="cuda", requires_grad=True)
    cw = rng.standard_normal((B, m))
    E = layer(x)
    (E * torch.tensor(cw, dtype=torch.float32, device="cuda")).sum().backward()
    outs = oracle.enumerate_unbunched(m, 3)

    def f(theta, data_b, b):
        U = oracle.mesh_unitary(m, theta, data_b)
        e = oracle.mode_expectations(oracle.renormalise(oracle.probabilities(U, s, outs)), outs)
        return float(e @ cw[b])

    th = layer.theta.detach().cpu().double().numpy()
    h = 1e-6
    g_th = np.zeros_like(th)
    for b in range(B):
        d = mb.data[b].astype(np.float64)
        for i in range(len(th)):
            tp, tm = th.copy(), th.copy()
            tp[i] += h
            tm[i] -= h
            g_th[i] += (f(tp, d, b) - f(tm, d, b)) / (2 * h)
        g_d = np.zeros_like(d)
        for i in range(len(d)):
            dp_, dm_ = d.copy(), d.copy()
            dp_[i] += h
            dm_[i] -= h
            g_d[i] = (f(th, dp_, b) - f(th, dm_, b)) / (2 * h)
        gx = x.grad[b].cpu().double().numpy()
        assert np.linalg.norm(gx - g_d) / np.linalg.norm(g_d) <= G_TOL
    g = layer.theta.grad.cpu().double().numpy()
    assert np.linalg.norm(g - g_th) / np.linalg.norm(g_th) <= G_TOL
