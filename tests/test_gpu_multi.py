"""conv_apply_multi: several kernels on the same densities, pass 1 computed once (Sec. 2.1,
eq. (An); the paper's Tables 1-3 apply four kernels to one density).

  - every output is bitwise the output of conv_apply on its plan alone (the same kernels read the
    same row spectrum), with the plan's own or a caller's workspace, FP64 and FP32, with a mask;
  - one output per precision against the oracle (1e-12 FP64, 2e-6 FP32);
  - mismatched plans and unsupported pipelines are refused.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2107_03958_gb300 import inputs
from paper_2107_03958_gb300._native import ConvError
from paper_2107_03958_gb300.api import ConvPlan, apply_multi, multi_workspace_bytes

pytestmark = pytest.mark.gpu

INV2PI = 1.0 / (2.0 * math.pi)
SWEEP = [("log", dict(scale=-INV2PI)), ("pow", dict(gamma=-0.5)), ("pow", dict(gamma=-1.0)),
         ("pow", dict(gamma=-1.5)), ("helmholtz", dict(kappa=20.0))]
TOL = {"fp64": 1e-12, "fp32": 2e-6}


def _plans(n, prec, B, compact=True):
    return [ConvPlan(k, n=n, period=3, precision=prec, io="r2c" if k == "helmholtz" else "r2r", batch_max=B,
                     compact=compact, **kw) for k, kw in SWEEP]


@pytest.mark.parametrize("prec,n,compact,use_ws,masked", [("fp64", 128, True, False, False),
                                                         ("fp32", 256, True, True, True),
                                                         ("fp32", 128, False, False, False),
                                                         ("fp64", 4096, True, False, False)])
def test_multi_equals_single_applies(prec, n, compact, use_ws, masked):
    B = 2
    plans = _plans(n, prec, B, compact)
    u_np = inputs.bump_sums(n, B, seed=41)
    u = torch.tensor(u_np, dtype=plans[0].real_dtype, device="cuda")
    mask = None
    if masked:
        mask = plans[0].fs_mask("disk", (0.5, 0.5, 0.3)).to(plans[0].real_dtype)
    ws = None
    if use_ws:
        ws = torch.empty(multi_workspace_bytes(plans, B), dtype=torch.uint8, device="cuda")
    outs = apply_multi(plans, u, mask=mask, workspace=ws)
    for p, o in zip(plans, outs):
        ref = p.apply(u, mask=mask)
        p.device_status()
        assert torch.equal(o, ref), p.kernel
    # the log and Helmholtz outputs against the oracle (density 1)
    for k in (0, 4):
        kind = {"log": "log", "pow": "pow", "helmholtz": "helm"}[SWEEP[k][0]]
        g = O.ghat_full(kind, plans[k].M, plans[k].b, plans[k].a, **SWEEP[k][1])
        uu = u_np[1] if mask is None else u_np[1] * mask.double().cpu().numpy()
        ref = O.conv(uu.astype(np.float32).astype(np.float64) if prec == "fp32" else uu, plans[k].M, g)
        if kind != "helm":
            ref = ref.real
        got = outs[k][1].cpu().numpy()
        assert np.max(np.abs(got - ref)) <= TOL[prec] * np.max(np.abs(ref))


def test_multi_refuses_mismatched_and_unsupported_plans():
    a = ConvPlan("log", n=64, period=3, precision="fp32", io="r2r", compact=True)
    b = ConvPlan("log", n=128, period=3, precision="fp32", io="r2r", compact=True)
    c = ConvPlan("helmholtz", n=64, period=3, precision="fp32", io="c2c", compact=True, kappa=5.0)
    d = ConvPlan("log", n=64, period=3, precision="fp64", io="r2r", compact=True)
    u = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(ConvError, match="EINVAL"):
        multi_workspace_bytes([a, b], 1)  # another n
    with pytest.raises(ConvError, match="EINVAL"):
        multi_workspace_bytes([a, d], 1)  # another precision
    with pytest.raises(ConvError, match="EUNSUPPORTED"):
        multi_workspace_bytes([a, c], 1)  # a C2C plan
    with pytest.raises(ConvError, match="EINVAL"):
        apply_multi([a, a], u)  # the same plan twice
