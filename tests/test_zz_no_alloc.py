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
