"""Out-of-bounds writes and input mutation, checked without compute-sanitizer: every device array
a call touches (density, mask, output, caller's workspace) sits between two guard bands of a fixed
byte pattern, and after the call the bands must be intact, the density and mask unchanged and the
output finite.  Shapes: ragged and tiny n, R2R, split R2C (two-buffer and forced one-buffer), C2C,
the compile-time and runtime stage paths, a non-integer period, and conv_apply_multi.
"""
import numpy as np
import pytest
import torch

from paper_2107_03958_gb300 import inputs
from paper_2107_03958_gb300.api import ConvPlan, apply_multi, multi_workspace_bytes

pytestmark = pytest.mark.gpu

GUARD = 4096  # bytes on each side
PATTERN = 0xA5


class Guarded:
    """A device byte buffer of `nbytes` between two guard bands; .view(dtype, shape) is the
    payload (256-byte aligned)."""

    def __init__(self, nbytes):
        self.nbytes = int(nbytes)
        self.raw = torch.full((GUARD + self.nbytes + GUARD,), PATTERN, dtype=torch.uint8, device="cuda")

    def payload(self):
        return self.raw[GUARD:GUARD + self.nbytes]

    def view(self, dtype, shape):
        return self.payload().view(dtype).view(shape)

    def intact(self):
        lo = self.raw[:GUARD]
        hi = self.raw[GUARD + self.nbytes:]
        return bool(torch.all(lo == PATTERN)) and bool(torch.all(hi == PATTERN))


def _nbytes(dtype, shape):
    return int(np.prod(shape)) * torch.tensor([], dtype=dtype).element_size()


def _guarded_tensor(t):
    g = Guarded(_nbytes(t.dtype, t.shape))
    v = g.view(t.dtype, t.shape)
    v.copy_(t)
    return g, v


CASES = [
    # (kernel, kwargs, n, period, precision, io, compact, env); M = n b (or 2n) even and 2^a 3^b 5^c
    ("log", {}, 6, 3, "fp64", "r2r", False, {}),
    ("pow", {"gamma": -0.5}, 50, 3, "fp32", "r2r", False, {}),
    ("log", {}, 30, 3, "fp32", "r2r", True, {}),
    ("log", {}, 128, 3, "fp32", "r2r", True, {}),
    ("log", {}, 512, 3, "fp64", "r2r", True, {}),
    ("helmholtz", {"kappa": 9.0}, 27, 4, "fp64", "r2c", False, {}),  # h n odd: W2's alignment slot
    ("helmholtz", {"kappa": 9.0}, 128, 3, "fp32", "r2c", True, {}),
    ("helmholtz", {"kappa": 9.0}, 512, 3, "fp64", "r2c", True, {"WSCONV_SPLIT_ONE": "1"}),
    ("helmholtz", {"kappa": 9.0}, 64, 3, "fp32", "c2c", True, {}),
    ("log", {}, 40, 2.5, "fp32", "r2r", False, {}),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("use_ws", [False, True])
def test_apply_stays_in_bounds(case, use_ws, monkeypatch):
    kernel, kw, n, period, prec, io, compact, env = CASES[case]
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    B = 3
    plan = ConvPlan(kernel, n=n, period=period, precision=prec, io=io, batch_max=B, compact=compact, **kw)
    dt = plan.in_dtype()
    u0 = torch.tensor(inputs.bump_sums(n, B, seed=51), device="cuda")
    if io == "c2c":
        u0 = torch.complex(u0, 0.5 * u0)
    u0 = u0.to(dt)
    gu, u = _guarded_tensor(u0)
    gm, mask = _guarded_tensor(torch.linspace(0.5, 1.5, n * n, device="cuda").view(n, n).to(plan.real_dtype))
    go = Guarded(_nbytes(plan.out_dtype(), (B, n, n)))
    out = go.view(plan.out_dtype(), (B, n, n))
    ws, gw = None, None
    if use_ws:
        gw = Guarded(plan.workspace_bytes(B))
        ws = gw.payload()
    plan.apply(u, mask=mask, out=out, workspace=ws)
    plan.device_status()
    torch.cuda.synchronize()
    assert gu.intact() and gm.intact() and go.intact()
    assert gw is None or gw.intact()
    assert torch.equal(u, u0)
    assert bool(torch.all(torch.isfinite(torch.view_as_real(out) if out.is_complex() else out)))


def test_apply_multi_stays_in_bounds():
    n, B = 128, 2
    plans = [ConvPlan("log", n=n, period=3, precision="fp32", io="r2r", batch_max=B, compact=True),
             ConvPlan("helmholtz", n=n, period=3, precision="fp32", io="r2c", batch_max=B, compact=True,
                      kappa=20.0)]
    gu, u = _guarded_tensor(torch.tensor(inputs.bump_sums(n, B, seed=52), dtype=torch.float32, device="cuda"))
    gos = [Guarded(_nbytes(p.out_dtype(), (B, n, n))) for p in plans]
    outs = [g.view(p.out_dtype(), (B, n, n)) for g, p in zip(gos, plans)]
    gw = Guarded(multi_workspace_bytes(plans, B))
    apply_multi(plans, u, outs=outs, workspace=gw.payload())
    torch.cuda.synchronize()
    assert gu.intact() and gw.intact() and all(g.intact() for g in gos)

