"""Failure detection without a GPU fault.

Host-side injection makes the library's host calls fail the way the real
failure would (an allocation that runs out, a stream of another device);
the SLOS_DEBUG build's device-side bounds checks must stay silent on valid
inputs and leave the results unchanged.  Nothing here traps, faults or hangs
the GPU."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2602_11092_gb300 import workloads

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ALLOC, STREAM_DEV, NONE = 1, 2, 0


def _U(m, B, seed):
    return torch.tensor(workloads.haar_unitaries(m, B, np.random.default_rng(seed)), dtype=torch.complex64,
                        device="cuda")


def test_injected_allocation_failure_fails_the_plan_cleanly(slos):
    lib = slos.load()
    s = workloads.even_mode_input(16, 5)
    for nth in (1, 2, 5):
        assert lib.slos_inject_fault(ALLOC, nth) == 0
        with pytest.raises(slos.SlosError) as e:
            slos.Plan(16, s)
        assert e.value.status == 3 and "allocate" in str(e.value)
    lib.slos_inject_fault(NONE, 0)
    # one-shot: the next plan builds and computes the same as before the failures
    plan = slos.Plan(16, s)
    U = _U(16, 40, 3)
    p = plan.forward(U)
    ref = slos.Plan(16, s).forward(U)
    assert torch.equal(p, ref)


def test_misaligned_workspace_is_rejected_before_any_launch(slos):
    # the layer kernels move 16-byte pieces of the workspace; a workspace that
    # does not start on a 256-byte boundary is refused on the host
    plan = slos.Plan(8, workloads.even_mode_input(8, 4))
    U = _U(8, 33, 4)
    need = plan.workspace_bytes(33, training=True)
    raw = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    ws = raw[8:8 + need]
    out = torch.full((33, plan.n_outputs), -1.0, device="cuda")
    n0 = slos.launch_count()
    with pytest.raises(slos.SlosError) as e:
        plan.forward(U, save_for_backward=True, workspace=ws, out=out)
    assert e.value.status == 1 and "aligned" in str(e.value)
    with pytest.raises(slos.SlosError) as e:
        plan.backward(U, torch.ones(plan.n_outputs, device="cuda"), ws)
    assert e.value.status == 1 and "aligned" in str(e.value)
    assert slos.launch_count() == n0
    torch.cuda.synchronize()
    assert (out == -1.0).all()


def test_stream_of_another_device_is_rejected_before_any_launch(slos):
    lib = slos.load()
    plan = slos.Plan(8, workloads.even_mode_input(8, 4))
    U = _U(8, 33, 4)
    out = torch.full((33, plan.n_outputs), -1.0, device="cuda")
    ws = plan.workspace(33, training=True)
    lib.slos_inject_fault(STREAM_DEV, torch.cuda.current_device() + 1)
    try:
        n0 = slos.launch_count()
        with pytest.raises(slos.SlosError) as e:
            plan.forward(U, save_for_backward=True, workspace=ws, out=out)
        assert e.value.status == 1 and "device" in str(e.value)
        with pytest.raises(slos.SlosError):
            plan.backward(U, torch.ones(plan.n_outputs, device="cuda"), ws)
        assert slos.launch_count() == n0  # nothing was launched
        torch.cuda.synchronize()
        assert (out == -1.0).all()
    finally:
        lib.slos_inject_fault(NONE, 0)
    plan.forward(U, save_for_backward=True, workspace=ws, out=out)
    plan.sync_status()
    assert torch.isfinite(out).all()


_CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2602_11092_gb300 import binding, buildlib, workloads
binding.load(sys.argv[2])
res = {}
for m, n, B in [(6, 3, 5), (8, 4, 33), (16, 5, 64)]:
    s = workloads.even_mode_input(m, n) if m > 6 else [1, 1, 1, 0, 0, 0]
    plan = binding.Plan(m, s)
    U = torch.tensor(workloads.haar_unitaries(m, B, np.random.default_rng(m)), dtype=torch.complex64, device="cuda")
    ws = plan.workspace(B, training=True)
    p = plan.forward(U, save_for_backward=True, workspace=ws)
    c = torch.tensor(np.random.default_rng(m + 1).standard_normal(plan.n_outputs), dtype=torch.float32, device="cuda")
    dU = plan.backward(U, c, ws)
    plan.sync_status()
    res[f"{m}_{n}"] = [p.cpu().numpy().tobytes().hex(), dU.cpu().numpy().tobytes().hex()]
print(json.dumps(res))
"""


def _run_child(lib_path):
    r = subprocess.run([sys.executable, "-c", _CHILD, ROOT, lib_path], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_build_bounds_checks_stay_silent_and_change_nothing():
    """The SLOS_DEBUG library (device-side bounds checks on every gather index
    of the slot-table forward and the split-lattice backward) on valid plans:
    the status word stays clear (sync_status raises otherwise) and the
    probabilities and dU equal the release library's bit for bit."""
    from paper_2602_11092_gb300 import buildlib
    dbg = buildlib.build_debug()
    got = _run_child(dbg)
    ref = _run_child(buildlib.LIB)
    assert got.keys() == ref.keys()
    for k in ref:
        assert got[k] == ref[k], k
