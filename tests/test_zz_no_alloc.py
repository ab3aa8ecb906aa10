"""slos_forward_noalloc: the forward pass for callers that cannot allocate
device memory (for example a plugin whose host application owns every device
allocation through its own pool).  It runs on a scratch array built into the
library; these tests call it through the C ABI and compare it with
slos_forward run on a caller-provided workspace, on two calls in a row.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest
import torch

from paper_2602_11092_gb300 import workloads

pytestmark = pytest.mark.gpu

P_TOL = 1e-5  # the same bound the forward parity tests use


def _case(slos, m, s, B, seed, detection):
    rng = np.random.default_rng(seed)
    U = torch.tensor(workloads.haar_unitaries(m, B, rng), dtype=torch.complex64, device="cuda")
    plan = slos.Plan(m, s, detection)
    return plan, U


@pytest.mark.parametrize("m,s,B,detection", [
    (6, [1, 1, 1, 0, 0, 0], 1, 0),
    (12, [1, 0] * 6, 40, 0),
    (8, [1, 0] * 4, 33, 1),
    (14, [1, 0] * 7, 32, 0),  # too large for the on-chip forward: layers go through the scratch
])
def test_noalloc_forward_matches_workspace_forward_twice(slos, m, s, B, detection):
    plan, U = _case(slos, m, s, B, 7 + m, detection)
    for call in range(2):
        if call == 1:  # a second call with other unitaries
            U = torch.tensor(workloads.haar_unitaries(m, B, np.random.default_rng(99 + m)),
                             dtype=torch.complex64, device="cuda")
        ref = plan.forward(U)  # slos_forward with a torch-allocated workspace
        out = torch.full_like(ref, float("nan"))
        plan.forward_noalloc(U, out)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert (out - ref).abs().max().item() <= P_TOL
    if detection == 0:
        ref = plan.forward(U, output=slos.AMPS)
        out = torch.zeros_like(ref)
        plan.forward_noalloc(U, out, output=slos.AMPS)
        assert (out - ref).abs().max().item() <= P_TOL
    if m == 14:
        # this plan is too large for the on-chip forward: its layers must have
        # gone through the built-in scratch, layer by layer
        slos.profile_reset()
        slos.profile_enable(True)
        plan.forward_noalloc(U, torch.empty_like(ref.real))
        torch.cuda.synchronize()
        names = set(slos.profile_collect())
        slos.profile_enable(False)
        assert "slos_fwd_final" in names and "slos_fwd_layer" in names, names
        assert "slos_fwd_fused" not in names, names


def test_noalloc_largest_batch_that_fits_the_scratch(slos):
    """The batch whose forward workspace is just under the scratch size runs
    and matches the workspace forward; one more instance is rejected when it
    no longer fits."""
    m, s = 14, [1, 0] * 7
    plan = slos.Plan(m, s)
    cap = slos.load().slos_noalloc_scratch_bytes()
    lo, hi = 1, 4096
    while lo < hi:  # largest B with workspace_bytes(B) <= cap
        mid = (lo + hi + 1) // 2
        if plan.workspace_bytes(mid, training=False) <= cap:
            lo = mid
        else:
            hi = mid - 1
    B = lo
    assert plan.workspace_bytes(B, training=False) <= cap < plan.workspace_bytes(B + 32, training=False)
    U = torch.tensor(workloads.haar_unitaries(m, B, np.random.default_rng(5)), dtype=torch.complex64, device="cuda")
    ref = plan.forward(U)
    out = torch.full_like(ref, float("nan"))
    plan.forward_noalloc(U, out)
    torch.cuda.synchronize()
    assert (out - ref).abs().max().item() <= P_TOL
    if plan.workspace_bytes(B + 1, training=False) > cap:
        U1 = torch.zeros((B + 1, m, m), dtype=torch.complex64, device="cuda")
        with pytest.raises(slos.SlosError):
            plan.forward_noalloc(U1, torch.empty((B + 1, plan.n_outputs), device="cuda"))


def test_noalloc_rejects_host_buffers_and_mismatched_outputs(slos):
    """Outputs that are not device memory of the current device are refused
    before any launch; a mismatched output dtype or shape is refused by the
    binding."""
    import ctypes
    m, s = 6, [1, 1, 1, 0, 0, 0]
    plan = slos.Plan(m, s)
    U = torch.tensor(workloads.haar_unitaries(m, 2, np.random.default_rng(1)), dtype=torch.complex64, device="cuda")
    host = np.zeros((2, plan.n_outputs), dtype=np.float32)
    st = slos.load().slos_forward_noalloc(plan._h, ctypes.c_void_p(U.data_ptr()), 2, slos.PROBS,
                                          ctypes.c_void_p(host.ctypes.data), None)
    assert st == 1  # SLOS_ERR_INVALID_ARG
    assert "device memory" in slos.load().slos_last_error().decode()
    with pytest.raises(ValueError):
        plan.forward_noalloc(U, torch.empty((2, plan.n_outputs), dtype=torch.float32, device="cuda"),
                             output=slos.AMPS)
    with pytest.raises(ValueError):
        plan.forward_noalloc(U, torch.empty((2, plan.n_outputs - 1), dtype=torch.float32, device="cuda"))


def test_noalloc_rejects_batches_beyond_the_scratch(slos):
    plan = slos.Plan(16, workloads.even_mode_input(16, 8))
    cap = slos.load().slos_noalloc_scratch_bytes()
    B = 256
    assert plan.workspace_bytes(B, training=False) > cap
    U = torch.zeros((B, 16, 16), dtype=torch.complex64, device="cuda")
    out = torch.empty((B, plan.n_outputs), dtype=torch.float32, device="cuda")
    with pytest.raises(slos.SlosError) as e:
        plan.forward_noalloc(U, out)
    assert e.value.status == 2
    assert "scratch" in str(e.value)
