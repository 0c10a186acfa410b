"""Serving loop (continuous batching): each request's result in a mixed, overlapping stream of
requests equals its result alone; admission respects the memory budget."""
import threading
import time

import numpy as np
import pytest
import torch

from paper_2107_03958_gb300 import inputs
from paper_2107_03958_gb300.api import ConvPlan, Server, ls_solve

pytestmark = pytest.mark.gpu


def _conv_alone(n, kernel, kw, precision, io, u, compact):
    plan = ConvPlan(kernel, n=n, period=3, precision=precision, io=io, batch_max=1, compact=compact, **kw)
    return plan.apply(u)


@pytest.mark.parametrize("compact", [False, True])
def test_mixed_requests_equal_their_results_alone(compact):
    rng = np.random.default_rng(7)
    srv = Server(mem_budget_bytes=8 << 30, max_inflight=32, conv_batch_max=8, ls_workers=2, compact=compact)
    reqs = []
    kinds = [("log", {"scale": 1.0}), ("pow", {"gamma": -1.0}), ("helmholtz", {"kappa": 20.0})]
    for i in range(24):
        n = int(rng.choice([64, 128, 256]))
        if i % 6 == 5:
            kappa = float(rng.uniform(5, 30))
            m = torch.tensor(inputs.lippmann_contrast(n, "bump"), device="cuda")
            f = torch.tensor(inputs.plane_wave(n, kappa), device="cuda")
            x = torch.zeros_like(f)
            reqs.append(("ls", n, kappa, "fp64" if i % 12 == 5 else "fp32", (m, f, x)))
        else:
            kernel, kw = kinds[int(rng.integers(0, 3))]
            io = "r2c" if kernel == "helmholtz" else "r2r"
            prec = "fp32" if i % 2 else "fp64"
            dt = torch.float32 if prec == "fp32" else torch.float64
            u = torch.tensor(inputs.bump_sums(n, 1, seed=1000 + i)[0], dtype=dt, device="cuda")
            out = torch.empty((n, n), dtype=(dt if io == "r2r" else (torch.complex64 if prec == "fp32" else torch.complex128)),
                              device="cuda")
            reqs.append(("conv", n, (kernel, kw, io), prec, (u, out)))
    tickets = []

    def producer():
        for r in reqs:
            if r[0] == "ls":
                _, n, kappa, prec, (m, f, x) = r
                tickets.append(srv.submit_ls(m, f, x, kappa, precision=prec))
            else:
                _, n, (kernel, kw, io), prec, (u, out) = r
                tickets.append(srv.submit_conv(u, out, kernel=kernel, precision=prec, io=io, **kw))
            time.sleep(float(rng.exponential(0.002)))

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    results = [srv.wait(t, timeout_s=300) for t in tickets]
    stats = srv.stats()
    srv.close()
    assert all(r["status"] == "CONV_OK" for r in results), results
    assert stats["completed"] == len(reqs)
    for r, res in zip(reqs, results):
        if r[0] == "ls":
            _, n, kappa, prec, (m, f, x) = r
            plan = ConvPlan("helmholtz", n=n, period=3, precision=prec, io="c2c", kappa=kappa, compact=compact)
            xa, info = ls_solve(plan, m, f, refine=(prec == "fp32"))
            assert res["rel_residual"] <= 1.05e-10
            assert torch.equal(xa, x), (n, kappa, prec)
        else:
            _, n, (kernel, kw, io), prec, (u, out) = r
            alone = _conv_alone(n, kernel, kw, prec, io, u, compact)
            assert torch.equal(alone, out), (n, kernel, prec, res["batched_with"])


def test_budget_admission_and_rejection():
    n = 128
    srv = Server(mem_budget_bytes=64 << 20, max_inflight=4, conv_batch_max=4, ls_workers=1)
    u = torch.tensor(inputs.bump_sums(n, 1, seed=3)[0], device="cuda")
    outs = [torch.empty_like(u) for _ in range(6)]
    tks = [srv.submit_conv(u, o, kernel="log", precision="fp64") for o in outs]
    res = [srv.wait(t, timeout_s=120) for t in tks]
    assert all(r["status"] == "CONV_OK" for r in res)
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    big = torch.zeros(2048, 2048, dtype=torch.float64, device="cuda")
    bo = torch.empty_like(big)
    r = srv.wait(srv.submit_conv(big, bo, kernel="log", precision="fp64"), timeout_s=60)
    assert r["status"] == "CONV_ENOMEM"
    srv.close()


def test_cached_ls_plans_count_their_krylov_workspace():
    """An LS plan keeps its Krylov workspace (and its FP64 twin) after the solve, for as long as the
    server caches it: the budget counts them, and a second LS plan that would not fit beside the
    first evicts it instead of exceeding the budget."""
    n = 256
    basis = n * n * 16 * 51
    budget = int(1.6 * basis)
    srv = Server(mem_budget_bytes=budget, max_inflight=4, conv_batch_max=4, ls_workers=1, compact=True)
    m = torch.tensor(inputs.lippmann_contrast(n, "bump"), device="cuda")
    for i, kappa in enumerate((11.0, 23.0)):
        f = torch.tensor(inputs.plane_wave(n, kappa), device="cuda")
        x = torch.zeros_like(f)
        r = srv.wait(srv.submit_ls(m, f, x, kappa, precision="fp32"), timeout_s=120)
        assert r["status"] == "CONV_OK" and r["rel_residual"] <= 1.05e-10, r
        st = srv.stats()
        assert basis <= st["bytes_in_use"] <= budget, st
        assert st["plans_evicted"] == i, st
    srv.close()


def test_same_shape_requests_on_different_kernels_share_a_batch():
    """Convolutions of one transform shape (n, period, precision, io) on different kernels queue
    together while a batch of their shape runs, and go as one launch per pass with each density's
    own multiplier: fewer batches than requests, each result bitwise its own apply alone."""
    n = 256
    srv = Server(mem_budget_bytes=8 << 30, max_inflight=64, conv_batch_max=16, ls_workers=1, compact=True)
    kinds = [("log", {"scale": -1.0}), ("pow", {"gamma": -0.5}), ("pow", {"gamma": -1.0}), ("pow", {"gamma": -1.5})]
    reqs = []
    for i in range(24):
        kernel, kw = kinds[i % 4]
        u = torch.tensor(inputs.bump_sums(n, 1, seed=500 + i)[0], dtype=torch.float32, device="cuda")
        reqs.append((kernel, kw, u, torch.empty_like(u)))
    # warm the four plans so that every request below finds its plan resident
    for kernel, kw, u, out in reqs[:4]:
        srv.wait(srv.submit_conv(u, out, kernel=kernel, precision="fp32", **kw), timeout_s=120)
    before = srv.stats()
    tickets = [srv.submit_conv(u, out, kernel=kernel, precision="fp32", **kw) for kernel, kw, u, out in reqs]
    res = [srv.wait(t, timeout_s=120) for t in tickets]
    st = srv.stats()
    srv.close()
    assert all(r["status"] == "CONV_OK" for r in res)
    batches = st["batches"] - before["batches"]
    assert batches < len(reqs), (batches, st)
    assert max(r["batched_with"] for r in res) > 1
    for kernel, kw, u, out in reqs:
        assert torch.equal(_conv_alone(n, kernel, kw, "fp32", "r2r", u, True), out), kernel
