"""Failure detection, exercised without faulting, trapping or hanging the GPU.

Faults are armed on the host (conv_fault_inject): a failed workspace allocation, a pass kernel's
bounded wait treated as given up, and a serving request lost before the dispatcher sees it.  Each
test checks that the failure is reported with its status and that the next call is correct.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2107_03958_gb300 import _native as N
from paper_2107_03958_gb300 import inputs
from paper_2107_03958_gb300.api import ConvPlan, Server, fault_inject

pytestmark = pytest.mark.gpu

SCALE = -1.0 / (2 * math.pi)


@pytest.fixture(autouse=True)
def _disarm():
    yield
    for k in ("alloc", "wait", "drop"):
        fault_inject(k, 0)


def _oracle(u, plan):
    g = O.ghat_full("log", plan.M, plan.b, plan.a, scale=SCALE)
    return np.stack([O.conv(x, plan.M, g).real for x in u])


def test_failed_workspace_allocation_reports_enomem_and_cleans_up():
    fault_inject("alloc", 1)
    with pytest.raises(N.ConvError) as e:
        ConvPlan("log", n=64, period=3, precision="fp64", scale=SCALE)
    assert e.value.status == 3 and "injected" in str(e.value)
    plan = ConvPlan("log", n=64, period=3, precision="fp64", scale=SCALE)
    u = inputs.bump_sums(64, 1, seed=3)
    out = plan.apply(torch.tensor(u[0], device="cuda")).cpu().numpy()
    ref = _oracle(u, plan)[0]
    assert np.max(np.abs(out - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_given_up_wait_is_reported_and_the_next_apply_is_correct():
    """Every prefetching pass kernel of one apply abandons its first work item as if its bounded
    wait had run out; the copy it issued still lands (drained with the ordinary bound) before the
    CTA leaves.  conv_device_status returns CONV_ETIMEOUT once and clears the word."""
    n, B = 1024, 2
    plan = ConvPlan("log", n=n, period=3, precision="fp32", batch_max=B, compact=True, scale=SCALE)
    assert plan.info.fused == 1 and plan.info.static_len == 2 * n
    u = torch.tensor(inputs.bump_sums(n, B, seed=11), dtype=torch.float32, device="cuda")
    plan.apply(u)
    plan.device_status()
    fault_inject("wait", 1)
    plan.apply(u)
    with pytest.raises(N.ConvError) as e:
        plan.device_status()
    assert e.value.status == 5
    plan.device_status()  # cleared
    out = plan.apply(u).cpu().numpy()
    plan.device_status()
    ref = _oracle(u.double().cpu().numpy(), plan)
    assert np.max(np.abs(out - ref)) <= 2e-6 * np.max(np.abs(ref))


def test_lost_request_times_out_and_is_cancelled_and_the_server_goes_on():
    n = 64
    srv = Server(mem_budget_bytes=1 << 30, max_inflight=8, conv_batch_max=4, ls_workers=1)
    u = torch.tensor(inputs.bump_sums(n, 1, seed=5)[0], device="cuda")
    out_lost = torch.empty_like(u)
    out_ok = torch.empty_like(u)
    fault_inject("drop", 1)
    lost = srv.submit_conv(u, out_lost, kernel="log", precision="fp64", scale=SCALE)
    ok = srv.submit_conv(u, out_ok, kernel="log", precision="fp64", scale=SCALE)
    r = srv.wait(ok, timeout_s=60)
    assert r["status"] == "CONV_OK"
    with pytest.raises(N.ConvError) as e:
        srv.wait(lost, timeout_s=0.2)
    assert e.value.status == 5
    srv.cancel(lost)
    assert srv.wait(lost, timeout_s=1)["status"] == "CONV_ECANCELLED"
    plan = ConvPlan("log", n=n, period=3, precision="fp64", scale=SCALE)
    ref = _oracle(u.cpu().numpy()[None], plan)[0]
    assert np.max(np.abs(out_ok.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
    st = srv.stats()
    assert st["failed"] == 1 and st["completed"] == 2
    srv.close()


def test_server_reports_a_failed_plan_build_and_serves_the_next_request():
    n = 96
    srv = Server(mem_budget_bytes=1 << 30, max_inflight=8, conv_batch_max=4, ls_workers=1)
    u = torch.tensor(inputs.bump_sums(n, 1, seed=6)[0], device="cuda")
    out = torch.empty_like(u)
    fault_inject("alloc", 1)
    t = srv.submit_conv(u, out, kernel="log", precision="fp64", scale=SCALE)
    assert srv.wait(t, timeout_s=60)["status"] == "CONV_ENOMEM"
    t = srv.submit_conv(u, out, kernel="log", precision="fp64", scale=SCALE)
    assert srv.wait(t, timeout_s=60)["status"] == "CONV_OK"
    plan = ConvPlan("log", n=n, period=3, precision="fp64", scale=SCALE)
    ref = _oracle(u.cpu().numpy()[None], plan)[0]
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
    srv.close()
