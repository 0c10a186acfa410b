"""Parity of the CUDA convolution path (through the C ABI) with the CPU oracle, element by element.

Tolerances (relative L-infinity, eq. (rel-err) normalisation by max |oracle|):
  FP64 passes: 1e-12.   FP32 passes: 2e-6 (single-precision FFTs of length up to 3*8192: about
  log2(M) * 6e-8 * a few, measured well below this bound).
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2107_03958_gb300 import inputs
from paper_2107_03958_gb300.api import ConvPlan

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-6}
INV2PI = 1.0 / (2.0 * math.pi)
KERNELS = {
    "log": dict(kernel="log", scale=-INV2PI),
    "pow-0.5": dict(kernel="pow", gamma=-0.5),
    "pow-1": dict(kernel="pow", gamma=-1.0),
    "pow-1.5": dict(kernel="pow", gamma=-1.5),
    "helm20": dict(kernel="helmholtz", kappa=20.0),
}


def _oracle_kw(kw):
    kind = {"log": "log", "pow": "pow", "helmholtz": "helm"}[kw["kernel"]]
    return kind, {k: v for k, v in kw.items() if k in ("gamma", "kappa", "scale")}


def _relerr(ref, got):
    return float(np.max(np.abs(ref - got)) / np.max(np.abs(ref)))


def _oracle_conv(u, plan, kw):
    kind, okw = _oracle_kw(kw)
    g = O.ghat_full(kind, plan.M, plan.b, plan.a, **okw)
    return O.conv(u, plan.M, g)


# ------------------------------------------------------------------ moments
@pytest.mark.parametrize("name", list(KERNELS))
@pytest.mark.parametrize("n", [16, 128])
def test_ghat_table_matches_oracle(name, n):
    kw = KERNELS[name]
    plan = ConvPlan(n=n, period=3, precision="fp64", io="r2c" if kw["kernel"] == "helmholtz" else "r2r", **kw)
    got = plan.ghat_quadrant()
    kind, okw = _oracle_kw(kw)
    h = plan.M // 2 + 1
    ref = np.zeros((h, h), dtype=complex)
    for k2 in range(h):
        for k1 in range(h):
            ref[k2, k1] = O.ghat_radial(kind, math.hypot(k1, k2), plan.b, plan.a, **okw)
    if kind != "helm":
        ref = ref.real
    # Helmholtz: outside the quadrature band the closed form divides by s^2 - kappa^2, so entries
    # a few percent from resonance carry ~|kappa^2/(s^2-kappa^2)| ulps on either side.
    tol = 1e-12 if kind == "helm" else 1e-13
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))


def test_helmholtz_ghat_near_resonance():
    """kappa chosen so that |k| = (3,4) sits 1e-6 from the resonance circle s = kappa."""
    b = 3.0
    kappa = 2 * math.pi * 5.0 / b * (1 + 1e-6)
    plan = ConvPlan("helmholtz", n=8, period=3, precision="fp64", io="c2c", kappa=kappa)
    got = plan.ghat_quadrant()
    ref = O.ghat_radial("helm", 5.0, b, plan.a, kappa=kappa)
    assert abs(got[4, 3] - ref) <= 1e-12 * abs(ref)
    assert abs(got[0, 0] - O.ghat_radial("helm", 0.0, b, plan.a, kappa=kappa)) <= 1e-13 * abs(ref)


# ------------------------------------------------------------------ the scheme
CASES = [
    # n, period, kernel, io
    (8, 3, "log", "r2r"), (16, 3, "pow-1", "r2r"), (32, 3, "pow-0.5", "r2r"), (64, 2, "log", "r2r"),
    (96, 3, "pow-1.5", "r2r"), (128, 3, "log", "r2r"), (256, 3, "pow-1", "r2r"),
    (48, 3, "helm20", "r2c"), (128, 3, "helm20", "c2c"), (64, 3, "log", "c2c"), (32, 3, "pow-1", "r2c"),
    (15, 2, "log", "r2r"),  # odd n: the last row pair is ragged (M = 30: generic radix-5 path)
    (9, 2, "pow-1", "r2r"),  # M = 18 = 2 * 3 * 3: generic path
    (3, 4, "log", "r2r"), (4, 3, "log", "c2c"), (2, 3, "pow-1", "r2c"),  # tiny transforms
    # R2C with the complex Helmholtz multiplier: the split pipeline (row pairs, one forward and two
    # inverse column transforms, packed inverse rows) wherever its fused passes exist
    (256, 3, "helm20", "r2c"), (15, 2, "helm20", "r2c"),
    (9, 8, "helm20", "r2c"),  # M = 72, h n = 333 odd: the second spectrum array is realigned
    (27, 4, "helm20", "r2c"),  # M = 108 = 4 * 3^3: FP64 E = 12 fused passes, h n odd
]


@pytest.mark.parametrize("compact", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,period,name,io", CASES)
def test_conv_matches_oracle(n, period, name, io, prec, compact):
    """Period-b passes and the compact (2n-periodic) embedding of the same quadrature weights."""
    kw = KERNELS[name]
    a = 0.0 if period == 3 else 0.45 * 2  # b = 2 needs an explicit radius
    plan = ConvPlan(n=n, period=period, trunc_a=a, precision=prec, io=io, batch_max=3, compact=compact, **kw)
    rng = np.random.default_rng(n * 7 + period)
    B = 3
    u = rng.standard_normal((B, n, n))
    if io == "c2c":
        u = u + 1j * rng.standard_normal((B, n, n))
    ut = torch.tensor(u, dtype=plan.in_dtype(), device="cuda")
    out = plan.apply(ut).cpu().numpy()
    plan.device_status()
    ref = _oracle_conv(u, plan, kw)
    if io == "r2r":
        assert np.max(np.abs(ref.imag)) <= 1e-12 * np.max(np.abs(ref))
        ref = ref.real
    for i in range(B):
        assert _relerr(ref[i], out[i]) <= TOL[prec], (i, _relerr(ref[i], out[i]))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mask_and_axpby(prec):
    n = 64
    kw = KERNELS["helm20"]
    plan = ConvPlan(n=n, period=3, precision=prec, io="c2c", batch_max=2, **kw)
    rng = np.random.default_rng(5)
    u = rng.standard_normal((2, n, n)) + 1j * rng.standard_normal((2, n, n))
    m = rng.uniform(0, 1, (n, n))
    ut = torch.tensor(u, dtype=plan.cplx_dtype, device="cuda")
    mt = torch.tensor(m, dtype=plan.real_dtype, device="cuda")
    alpha, beta = 400.0 + 3.0j, 1.0
    out = plan.apply(ut, mask=mt, alpha=alpha, beta=beta).cpu().numpy()
    ref = beta * u + alpha * _oracle_conv(u * m, plan, kw)
    for i in range(2):
        assert _relerr(ref[i], out[i]) <= TOL[prec]


def test_poisson_bump_config():
    """Single bump, -(1/2pi) log, n = 64, b = 2, a = 1.1: GPU == oracle, and both near the radial
    Poisson potential."""
    n = 64
    plan = ConvPlan("log", n=n, period=2, trunc_a=1.1, precision="fp64", io="r2r", scale=-INV2PI)
    u = inputs.poisson_bump(n)
    out = plan.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    ref = O.conv(u, plan.M, O.ghat_full("log", plan.M, 2.0, 1.1, scale=-INV2PI)).real
    assert _relerr(ref, out) <= 1e-12


def test_batch_results_independent_of_batch_position():
    n = 96
    plan = ConvPlan("pow", n=n, period=3, precision="fp32", io="r2r", batch_max=8, gamma=-1.0)
    u = torch.tensor(inputs.bump_sums(n, 8, seed=11), dtype=torch.float32, device="cuda")
    full = plan.apply(u)
    for i in (0, 5, 7):
        alone = plan.apply(u[i].contiguous())
        assert torch.equal(alone, full[i])


def test_caller_workspace_and_empty_batch():
    n = 32
    plan = ConvPlan("log", n=n, period=3, precision="fp64", io="r2r", batch_max=1, scale=-INV2PI)
    u = torch.randn(4, n, n, dtype=torch.float64, device="cuda")
    ws = torch.empty(plan.workspace_bytes(4), dtype=torch.uint8, device="cuda")
    out = plan.apply(u, workspace=ws)
    ref = np.stack([plan.apply(u[i].contiguous()).cpu().numpy() for i in range(4)])
    assert np.array_equal(out.cpu().numpy(), ref)
    empty = torch.empty(0, n, n, dtype=torch.float64, device="cuda")
    assert plan.apply(empty).shape == (0, n, n)


def test_invalid_arguments_are_reported():
    from paper_2107_03958_gb300._native import ConvError
    with pytest.raises(ConvError, match="EINVAL"):
        ConvPlan("log", n=0, period=3)
    with pytest.raises(ConvError, match="EINVAL"):
        ConvPlan("log", n=16, period=2)  # b < 1 + sqrt 2 and no explicit radius
    with pytest.raises(ConvError, match="EUNSUPPORTED"):
        ConvPlan("log", n=14, period=3)  # M = 42 = 2 * 3 * 7
    with pytest.raises(ConvError, match="EINVAL"):
        ConvPlan("helmholtz", n=16, period=3, io="r2r", kappa=5.0)
    with pytest.raises(ConvError, match="EUNSUPPORTED"):
        ConvPlan("pow", n=16, period=3, gamma=-0.3)
    with pytest.raises(ConvError, match="EUNSUPPORTED"):
        ConvPlan("log", n=5, period=3)  # M = 15 is odd
    with pytest.raises(ConvError, match="EUNSUPPORTED"):
        ConvPlan("log", n=1, period=3)  # M = 3
    plan = ConvPlan("log", n=16, period=3, batch_max=1)
    u = torch.zeros(2, 16, 16, dtype=torch.float64, device="cuda")
    with pytest.raises(ConvError, match="EINVAL"):
        plan.apply(u)  # batch > batch_max without a workspace
    with pytest.raises(ConvError, match="EINVAL"):
        plan.apply(u[0], out=u[0])  # aliasing


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_caller_workspace_r2c_split_and_alignment(prec):
    """R2C Helmholtz through a caller's workspace of exactly conv_workspace_size bytes (odd h n: the
    second spectrum array starts one element late) equals the plan's own workspace; misaligned
    workspaces and arrays are rejected."""
    from paper_2107_03958_gb300._native import ConvError
    n, B = 9, 3
    plan = ConvPlan("helmholtz", n=n, period=8, precision=prec, io="r2c", batch_max=B, kappa=20.0)
    u = torch.tensor(np.random.default_rng(2).standard_normal((B, n, n)), dtype=plan.real_dtype, device="cuda")
    ws = torch.empty(plan.workspace_bytes(B) + 64, dtype=torch.uint8, device="cuda")
    out = plan.apply(u, workspace=ws[16:16 + plan.workspace_bytes(B)])
    assert torch.equal(out, plan.apply(u))
    with pytest.raises(ConvError, match="EINVAL"):
        plan.apply(u, workspace=ws[8:8 + plan.workspace_bytes(B)])
    import ctypes
    from paper_2107_03958_gb300 import _native as N
    raw = torch.empty(B * n * n * u.element_size() + 8, dtype=torch.uint8, device="cuda")
    with pytest.raises(ConvError, match="EINVAL"):  # u one byte past an element boundary
        N.check(plan._lib.conv_apply(plan._h, ctypes.c_void_p(raw.data_ptr() + 1), None,
                                     ctypes.c_void_p(out.data_ptr()), B, None, None))
    plan.device_status()


@pytest.mark.parametrize("name,io,prec", [("log", "r2r", "fp32"), ("helm20", "r2c", "fp32"),
                                          ("helm20", "c2c", "fp64"), ("pow-1", "r2r", "fp64")])
def test_host_buffer_apply_equals_device_apply(name, io, prec):
    """conv_apply_host (chunks of ceil(batch_max/4) densities, uploads/passes/downloads overlapped)
    gives bitwise the device-buffer result, for a ragged last chunk, with a mask, from pinned and
    from pageable host memory."""
    n, B = 256, 11
    kw = KERNELS[name]
    plan = ConvPlan(n=n, period=3, precision=prec, io=io, batch_max=8, compact=True, **kw)
    rng = np.random.default_rng(12)
    u = rng.standard_normal((B, n, n))
    if io == "c2c":
        u = u + 1j * rng.standard_normal((B, n, n))
    u_host = torch.tensor(u, dtype=plan.in_dtype()).pin_memory()
    mask = torch.tensor(rng.uniform(0, 1, (n, n)), dtype=plan.real_dtype, device="cuda")
    ws = torch.empty(plan.workspace_bytes(B), dtype=torch.uint8, device="cuda")
    ref = plan.apply(u_host.cuda(), mask=mask, workspace=ws).cpu()
    s = torch.cuda.Stream()
    out = plan.apply_host(u_host, mask=mask, stream=s)
    s.synchronize()
    assert torch.equal(out, ref)
    pageable = torch.empty(ref.shape, dtype=ref.dtype)
    plan.apply_host(u_host.clone(), out=pageable, mask=mask)
    torch.cuda.synchronize()
    assert torch.equal(pageable, ref)
    plan.device_status()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_multi_plan_host_apply_equals_device_apply(prec):
    """conv_apply_host_multi (one upload per chunk, the plans' passes in turn, each result chunk
    downloaded behind the next plan): every plan's result is bitwise its device-buffer apply, for
    the kernel sweep's mix of R2R and R2C plans, more chunks than device slots, a ragged last
    chunk and a mask."""
    from paper_2107_03958_gb300.api import apply_host_multi
    n, B = 128, 11
    plans = [ConvPlan(n=n, period=3, precision=prec, io="r2c" if k == "helm20" else "r2r",
                      batch_max=5 + i, compact=i % 2 == 0, **KERNELS[k]) for i, k in enumerate(KERNELS)]
    u = inputs.bump_sums(n, B, seed=21)
    u_host = torch.tensor(u, dtype=plans[0].real_dtype).pin_memory()
    mask = torch.tensor(np.random.default_rng(3).uniform(0, 1, (n, n)), dtype=plans[0].real_dtype, device="cuda")
    ud = u_host.cuda()
    refs = []
    for p in plans:
        ws = torch.empty(p.workspace_bytes(B), dtype=torch.uint8, device="cuda")
        refs.append(p.apply(ud, mask=mask, workspace=ws).cpu())
    s = torch.cuda.Stream()
    for _ in range(2):  # the second call reuses the slots kept on the first plan
        outs = apply_host_multi(plans, u_host, mask=mask, stream=s)
        s.synchronize()
        for o, r in zip(outs, refs):
            assert torch.equal(o, r)
    for p in plans:
        p.device_status()
    with pytest.raises(Exception):
        apply_host_multi([plans[0], plans[0]], u_host)


def test_multi_plan_host_apply_rejects_mismatched_plans():
    """conv_apply_host_multi needs one n, precision and input type across its plans."""
    from paper_2107_03958_gb300.api import apply_host_multi
    from paper_2107_03958_gb300._native import ConvError
    a = ConvPlan("log", n=64, period=3, precision="fp32", io="r2r")
    b = ConvPlan("log", n=32, period=3, precision="fp32", io="r2r")
    c = ConvPlan("log", n=64, period=3, precision="fp64", io="r2r")
    d = ConvPlan("helmholtz", n=64, period=3, precision="fp32", io="c2c", kappa=5.0)
    u = torch.zeros((1, 64, 64), dtype=torch.float32).pin_memory()
    outs = [torch.empty((1, 64, 64), dtype=p.out_dtype()).pin_memory() for p in (a, a)]
    for other in (b, c, d):
        with pytest.raises((ConvError, ValueError)):
            apply_host_multi([a, other], u, outs=[outs[0], torch.empty((1, 64, 64), dtype=other.out_dtype()).pin_memory()])


@pytest.mark.parametrize("name,io", [("log", "r2r"), ("helm20", "r2c")])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_autotuned_plan_matches_oracle(name, io, prec):
    """The autotuner (per-pass options chosen by timing) changes launch shapes only: its plan still
    matches the oracle."""
    n, B = 256, 4
    kw = KERNELS[name]
    plan = ConvPlan(n=n, period=3, precision=prec, io=io, batch_max=B, compact=True, autotune=True, **kw)
    u = inputs.bump_sums(n, B, seed=21)
    out = plan.apply(torch.tensor(u, dtype=plan.real_dtype, device="cuda")).cpu().numpy()
    plan.device_status()
    ref = _oracle_conv(u, plan, kw)
    if io == "r2r":
        ref = ref.real
    for i in range(B):
        assert _relerr(ref[i], out[i]) <= TOL[prec]


@pytest.mark.parametrize("io", ["r2r", "r2c", "c2c"])
@pytest.mark.parametrize("n,prec", [(1024, "fp32"), (2048, "fp32"), (512, "fp64"), (1024, "fp64")])
def test_compile_time_lengths_match_oracle_and_runtime_stages(n, prec, io, monkeypatch):
    """Compact embedding, L = 2n = 2^10 ... 2^12: the transforms whose stage structure is fixed at
    compile time match the oracle and the runtime-descriptor transforms of the same plan."""
    kw = KERNELS["helm20" if io != "r2r" else "pow-1"]
    B = 2
    rng = np.random.default_rng(n + len(io))
    u = inputs.bump_sums(n, B, seed=n)
    if io == "c2c":
        u = u + 1j * rng.standard_normal((B, n, n)) * 0.1
    outs = []
    for fused in ("1", "2"):
        monkeypatch.setenv("WSCONV_FUSED", fused)
        plan = ConvPlan(n=n, period=3, precision=prec, io=io, batch_max=B, compact=True, **kw)
        info = plan.info
        assert info.fused == 1 and info.static_log2 == (int(np.log2(2 * n)) if fused == "1" else 0)
        assert info.static_len == (2 * n if fused == "1" else 0)
        outs.append(plan.apply(torch.tensor(u, dtype=plan.in_dtype(), device="cuda")).cpu().numpy())
        plan.device_status()
    ref = _oracle_conv(u, plan, kw)
    if io == "r2r":
        ref = ref.real
    for i in range(B):
        assert _relerr(ref[i], outs[0][i]) <= TOL[prec]
        assert _relerr(outs[1][i], outs[0][i]) <= (1e-6 if prec == "fp32" else 1e-13)


@pytest.mark.parametrize("io", ["r2r", "r2c", "c2c"])
@pytest.mark.parametrize("n", [128, 1024, 2048])
def test_compile_time_period_3_lengths_match_oracle_and_runtime_stages(n, io, monkeypatch):
    """The paper's period-3 grid, L = 3n = 3 2^l: FP32 transforms whose radix-8/radix-3 stage
    structure is fixed at compile time (inputs beyond n pruned in the first stage, outputs beyond
    n in the last) match the oracle and the runtime-descriptor transforms of the same plan."""
    kw = KERNELS["helm20" if io != "r2r" else "log"]
    B = 2
    rng = np.random.default_rng(3 * n + len(io))
    u = inputs.bump_sums(n, B, seed=n + 5)
    if io == "c2c":
        u = u + 1j * rng.standard_normal((B, n, n)) * 0.1
    outs = []
    for fused in ("1", "2"):
        monkeypatch.setenv("WSCONV_FUSED", fused)
        plan = ConvPlan(n=n, period=3, precision="fp32", io=io, batch_max=B, **kw)
        info = plan.info
        assert info.fused == 1 and info.static_len == (3 * n if fused == "1" else 0)
        outs.append(plan.apply(torch.tensor(u, dtype=plan.in_dtype(), device="cuda")).cpu().numpy())
        plan.device_status()
    ref = _oracle_conv(u, plan, kw)
    if io == "r2r":
        ref = ref.real
    for i in range(B):
        assert _relerr(ref[i], outs[0][i]) <= TOL["fp32"]
        assert _relerr(outs[1][i], outs[0][i]) <= 1e-6


@pytest.mark.parametrize("io", ["r2r", "r2c"])
def test_compile_time_length_on_the_period_2_grid(io):
    """b = 2 makes M = 2n a power of two without the compact embedding: the compile-time
    transforms (zero half pruned, cropped half) on the paper's own period-b multiplier."""
    n, B = 1024, 2
    kw = KERNELS["log" if io == "r2r" else "helm20"]
    plan = ConvPlan(n=n, period=2, trunc_a=0.9, precision="fp32", io=io, batch_max=B, **kw)
    assert plan.info.static_log2 == 11
    u = inputs.bump_sums(n, B, seed=77)
    out = plan.apply(torch.tensor(u, dtype=plan.real_dtype, device="cuda")).cpu().numpy()
    plan.device_status()
    ref = _oracle_conv(u, plan, kw)
    if io == "r2r":
        ref = ref.real
    for i in range(B):
        assert _relerr(ref[i], out[i]) <= TOL["fp32"]


@pytest.mark.parametrize("prec,n,compact", [("fp64", 128, True), ("fp32", 256, True), ("fp32", 128, False)])
def test_split_r2c_one_buffer(prec, n, compact, monkeypatch):
    """The split Helmholtz column pass with one buffer per CTA (the Im-ghat spectrum parked in a
    global scratch line), forced at small n: bitwise the two-buffer pass's results, and the
    oracle's.  FP64 at n = 4096 (L = 8192) takes it by default (test_full_size_helmholtz_r2c)."""
    B = 3
    kw = KERNELS["helm20"]
    u = inputs.bump_sums(n, B, seed=31)
    outs = {}
    for one in ("1", "0"):
        monkeypatch.setenv("WSCONV_SPLIT_ONE", one)
        plan = ConvPlan(n=n, period=3, precision=prec, io="r2c", batch_max=B, compact=compact, **kw)
        assert plan.info.r2c_split == 1
        assert plan.workspace_bytes(B) >= plan.workspace_bytes(1)
        outs[one] = plan.apply(torch.tensor(u, dtype=plan.real_dtype, device="cuda")).cpu().numpy()
        plan.device_status()
    assert np.array_equal(outs["1"], outs["0"])
    kind, okw = _oracle_kw(kw)
    g = O.ghat_full(kind, plan.M, plan.b, plan.a, **okw)
    for i in range(B):
        assert _relerr(O.conv(u[i], plan.M, g), outs["1"][i]) <= TOL[prec]


def test_fp64_helmholtz_n4096_runs_split():
    plan = ConvPlan("helmholtz", n=4096, period=3, precision="fp64", io="r2c", batch_max=16, compact=True,
                    kappa=20.0)
    assert plan.info.r2c_split == 1


@pytest.mark.parametrize("compact", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_helmholtz_r2c(prec, compact):
    """n = 4096, b = 3, batch 16, Helmholtz kappa = 20 (the benchmark's R2C line): densities 0 and
    13 against the oracle's full FFT convolution."""
    n, B = 4096, 16
    kw = KERNELS["helm20"]
    plan = ConvPlan(n=n, period=3, precision=prec, io="r2c", batch_max=B, compact=compact, **kw)
    u = inputs.bump_sums(n, B)
    out = plan.apply(torch.tensor(u, dtype=plan.real_dtype, device="cuda"))
    plan.device_status()
    kind, okw = _oracle_kw(kw)
    g = O.ghat_full(kind, plan.M, plan.b, plan.a, **okw)
    for i in (0, 13):
        ref = O.conv(u[i], plan.M, g)
        assert _relerr(ref, out[i].cpu().numpy()) <= TOL[prec]


@pytest.mark.parametrize("compact", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_kernel_sweep(prec, compact):
    """n = 4096, b = 3, batch 16 (the benchmark's launch configuration): densities 0 and 9 against
    the oracle's full FFT convolution."""
    n, B = 4096, 16
    kw = KERNELS["log"]
    plan = ConvPlan(n=n, period=3, precision=prec, io="r2r", batch_max=B, compact=compact, **kw)
    u = inputs.bump_sums(n, B)
    out = plan.apply(torch.tensor(u, dtype=plan.real_dtype, device="cuda"))
    g = O.ghat_full("log", plan.M, plan.b, plan.a, scale=-INV2PI)
    for i in (0, 9):
        ref = O.conv(u[i], plan.M, g).real
        assert _relerr(ref, out[i].cpu().numpy()) <= TOL[prec]


@pytest.mark.parametrize("n", [2048, 4096])
def test_pingpong_column_pass(n, monkeypatch):
    """The FP32 compact R2R passes at L = 4096 and 8192 alternate between two buffers per line
    (one barrier per stage): the same arithmetic as the one-buffer passes, so bitwise the same
    results, and the oracle's to the FP32 tolerance."""
    B = 4
    kw = KERNELS["pow-1"]
    u = inputs.bump_sums(n, B, seed=21)
    outs = {}
    for pp in ("7", "0"):  # all three passes / none
        monkeypatch.setenv("WSCONV_PP", pp)
        plan = ConvPlan(n=n, period=3, precision="fp32", io="r2r", batch_max=B, compact=True, **kw)
        assert plan.info.cols_pingpong == (pp == "7")
        outs[pp] = plan.apply(torch.tensor(u, dtype=plan.real_dtype, device="cuda")).cpu().numpy()
        plan.device_status()
    assert np.array_equal(outs["7"], outs["0"])
    g = O.ghat_full("pow", plan.M, plan.b, plan.a, gamma=-1.0)
    ref = O.conv(u[B - 1], plan.M, g).real
    assert _relerr(ref, outs["7"][B - 1]) <= TOL["fp32"]


# ------------------------------------------------------------------ Fourier smoothing (Sec. 2.4)
@pytest.mark.parametrize("shape,geom", [("disk", (0.5, 0.5, 0.3)), ("rect", (0.25, 0.75, 0.25, 0.75)),
                                        ("rect", (0.3, 0.7, 0.3, 0.7)), ("disk", (0.47, 0.55, 0.21))])
@pytest.mark.parametrize("n", [32, 128])
def test_fs_mask_matches_oracle(shape, geom, n):
    plan = ConvPlan("log", n=n, period=3, precision="fp64", io="r2r", scale=-INV2PI)
    got = plan.fs_mask(shape, geom, 0.15).cpu().numpy()
    ref = O.fs_mask(n, 3.0, shape, geom, 0.15)
    # the mask sums M^2 terms carrying J1 (disk) from two different Bessel implementations (CUDA
    # and the C library); they differ in the last bits, so the mask agrees to a few 1e-12
    assert np.max(np.abs(got - ref)) <= 5e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fourier_smoothed_convolution(prec):
    """Disk(0.3) indicator times a smooth bump: A_n(u~ chi^n psi) on the GPU equals the oracle's."""
    n = 256
    plan = ConvPlan("pow", n=n, period=3, precision=prec, io="r2r", gamma=-1.0)
    ut = inputs.smooth_extension(n)
    mask = plan.fs_mask("disk", (0.5, 0.5, 0.3), 0.15)
    out = plan.apply(torch.tensor(ut, dtype=plan.real_dtype, device="cuda"), mask=mask).cpu().numpy()
    om = O.fs_mask(n, 3.0, "disk", (0.5, 0.5, 0.3), 0.15)
    ref = O.conv(ut * om, plan.M, O.ghat_full("pow", plan.M, 3.0, plan.a, gamma=-1.0)).real
    assert _relerr(ref, out) <= TOL[prec]


def test_lines_beyond_one_cta_take_the_long_line_pipeline():
    """A pass holds a whole line of the transform in one CTA's shared memory; FP64 lines of 16384
    (n = 8192 compact) and 24576 (period 3), and FP32 lines of 24576, run as four-step FP64 line
    transforms instead (tests/test_gpu_long_lines.py checks their results)."""
    for prec, compact in (("fp64", True), ("fp32", False), ("fp64", False)):
        plan = ConvPlan("log", n=8192, period=3, precision=prec, io="r2r", compact=compact)
        assert plan.info.long_lines == 1, (prec, compact)
        del plan
    assert ConvPlan("log", n=4096, period=3, precision="fp64", io="r2r", compact=True).info.long_lines == 0


@pytest.mark.parametrize("io", ["r2r", "c2c"])
def test_split_plan_time_lines_equal_direct(io, monkeypatch):
    """The plan's FP64 line transforms split four-step (forced here at n = 64, where one CTA holds
    a line) give the same compact multiplier and FS mask as the direct transforms, to rounding."""
    n = 64
    kw = KERNELS["log"] if io == "r2r" else KERNELS["helm20"]
    u = inputs.bump_sums(n, 2, seed=31)
    if io == "c2c":
        u = u + 0.5j * inputs.bump_sums(n, 2, seed=32)
    outs, masks = [], []
    for split in ("0", "1"):
        monkeypatch.setenv("WSCONV_LINE_SPLIT", split)
        plan = ConvPlan(n=n, period=3, precision="fp64", io=io, compact=True, batch_max=2, **kw)
        outs.append(plan.apply(torch.tensor(u, dtype=plan.in_dtype(), device="cuda")).cpu().numpy())
        masks.append(plan.fs_mask("disk", (0.5, 0.5, 0.3)).cpu().numpy())
    assert _relerr(outs[0], outs[1]) <= 1e-13
    assert np.max(np.abs(masks[0] - masks[1])) <= 1e-13


def test_n8192_fp32_compact_matches_the_analytic_potential(monkeypatch):
    """n = 8192, FP32 passes on the compact grid (L = 16384: the compile-time transform at 1024
    threads, and the runtime stage structure; the plan's FP64 lines of 24576 and 16384 split
    four-step): the log potential of the Laplacian of a Gaussian sum (the setting of Table 7,
    alpha = 250) is minus the Gaussian sum.  FP32 rounding of 16384-point transforms sets the
    error, measured against that closed form; the two stage structures agree to it."""
    n = 8192
    centres = [(0.6, 0.6), (0.5, 0.5), (0.35, 0.6)]
    f = inputs.gaussian_sum_laplacian(n, 250.0, centres)
    ex = -inputs.gaussian_sum(n, 250.0, centres)
    ft = torch.tensor(f, dtype=torch.float32, device="cuda")
    outs = []
    for fused in ("1", "2"):
        monkeypatch.setenv("WSCONV_FUSED", fused)
        plan = ConvPlan("log", n=n, period=3, precision="fp32", io="r2r", compact=True, scale=-INV2PI)
        assert plan.info.transform_len == 16384
        assert plan.info.static_len == (16384 if fused == "1" else 0)
        outs.append(plan.apply(ft).cpu().numpy())
        plan.device_status()
        del plan
        torch.cuda.empty_cache()
    for out in outs:
        err = _relerr(ex, out)
        assert err <= 2e-5, err
    assert _relerr(outs[1], outs[0]) <= 2e-6
