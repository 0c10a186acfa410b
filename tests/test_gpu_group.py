"""Mixed-size batching through the C ABI (conv_group_create / conv_group_launch): one CUDA graph
launch over applies whose plans differ in n, kernel, period, precision and io.

Every item must equal its own conv_apply bit for bit (the graph holds the same pass kernels with
the same launch shapes), and an FP64 item must match the oracle of eq. (An) at 1e-12.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2107_03958_gb300 import _native as N
from paper_2107_03958_gb300 import inputs
from paper_2107_03958_gb300.api import ConvGroup, ConvPlan

pytestmark = pytest.mark.gpu

INV2PI = 1.0 / (2.0 * math.pi)


def _u(plan, batch, seed):
    re = torch.tensor(inputs.bump_sums(plan.n, batch, seed=seed), dtype=plan.real_dtype, device="cuda")
    if plan.io != "c2c":
        return re
    im = torch.tensor(inputs.bump_sums(plan.n, batch, seed=seed + 1), dtype=plan.real_dtype, device="cuda")
    return torch.complex(re, im)


def _plans():
    return [
        ConvPlan("log", n=64, period=3, precision="fp64", io="r2r", batch_max=2, scale=-INV2PI, compact=True),
        ConvPlan("helmholtz", n=96, period=3, precision="fp32", io="r2c", batch_max=3, kappa=20.0),
        ConvPlan("pow", n=128, period=3, precision="fp32", io="c2c", batch_max=1, gamma=-1.0, compact=True),
        ConvPlan("log", n=256, period=3, precision="fp32", io="r2r", batch_max=4, scale=-INV2PI, compact=True),
        ConvPlan("helmholtz", n=48, period=2.5, precision="fp64", io="c2c", batch_max=1, kappa=10.0),
    ]


def test_group_items_equal_their_own_apply():
    plans = _plans()
    items, refs = [], []
    batches = [2, 3, 1, 4, 1]
    for i, (p, b) in enumerate(zip(plans, batches)):
        u = _u(p, b, 100 + 10 * i)
        mask = None
        if i == 3:  # one masked item (a Fourier-smoothed disk, Sec. 2.4)
            mask = p.fs_mask("disk", (0.5, 0.5, 0.3))
        out = torch.full(u.shape, float("nan"), dtype=p.out_dtype(), device="cuda")
        items.append((p, u, out) if mask is None else (p, u, out, mask))
        refs.append(p.apply(u, mask=mask))
    # a second item on the first plan (its own buffers): runs after the first on its branch
    u2 = _u(plans[0], 1, 7)
    out2 = torch.empty(u2.shape, dtype=plans[0].out_dtype(), device="cuda")
    items.append((plans[0], u2, out2))
    refs.append(plans[0].apply(u2))
    g = ConvGroup(items)
    for _ in range(2):
        g.launch()
    torch.cuda.synchronize()
    for p in plans:
        p.device_status()
    for it, ref in zip(items, refs):
        assert torch.equal(it[2], ref), "item on n=%d differs from its conv_apply" % it[0].n


def test_group_fp64_item_matches_oracle_and_reads_new_contents():
    p = ConvPlan("log", n=64, period=3, precision="fp64", io="r2r", batch_max=2, scale=-INV2PI, compact=True)
    q = ConvPlan("pow", n=32, period=3, precision="fp32", io="r2r", batch_max=1, gamma=-0.5)
    u = _u(p, 2, 11)
    out = torch.empty_like(u)
    v = _u(q, 1, 12)
    vout = torch.empty_like(v)
    g = ConvGroup([(p, u, out), (q, v, vout)])
    g.launch()
    torch.cuda.synchronize()
    gh = O.ghat_full("log", p.M, p.b, p.a, scale=-INV2PI)
    ref = O.conv(u.cpu().numpy(), p.M, gh).real
    err = float(np.max(np.abs(ref - out.cpu().numpy())) / np.max(np.abs(ref)))
    assert err < 1e-12, err
    # the graph reads the buffers' current contents at every launch
    u.copy_(_u(p, 2, 13))
    g.launch()
    torch.cuda.synchronize()
    ref = O.conv(u.cpu().numpy(), p.M, gh).real
    err = float(np.max(np.abs(ref - out.cpu().numpy())) / np.max(np.abs(ref)))
    assert err < 1e-12, err


def _create(lib, plans, us, outs, batches, masks=None):
    k = len(plans)
    arr = ctypes.c_void_p * k
    h = ctypes.c_void_p()
    st = lib.conv_group_create(k, arr(*[p.handle.value for p in plans]), arr(*[u.data_ptr() for u in us]),
                               arr(*masks) if masks else None, arr(*[o.data_ptr() for o in outs]),
                               (ctypes.c_int * k)(*batches), ctypes.byref(h))
    if st == 0:
        lib.conv_group_destroy(h)
    return st


def test_group_rejects_bad_items():
    lib = N.load()
    p = ConvPlan("log", n=32, period=3, precision="fp32", io="r2r", batch_max=2, scale=-INV2PI)
    q = ConvPlan("log", n=32, period=3, precision="fp64", io="r2r", batch_max=1, scale=-INV2PI)
    u = _u(p, 2, 1)
    out = torch.empty_like(u)
    u64 = _u(q, 1, 2)
    out64 = torch.empty_like(u64)
    h = ctypes.c_void_p()
    assert lib.conv_group_create(0, None, None, None, None, None, ctypes.byref(h)) == 1
    assert _create(lib, [p], [u], [out], [3]) == 1            # batch above batch_max
    assert _create(lib, [p], [u], [u], [2]) == 1              # out aliases u
    assert _create(lib, [p, q], [u, u64], [out, u], [2, 1]) == 1  # q's out is p's input
    assert _create(lib, [p, q], [u, u64], [out, out], [2, 1]) == 1  # two items write one out
    p.timing(True)
    assert _create(lib, [p], [u], [out], [2]) == 1            # timing events cannot be captured
    p.timing(False)
    assert _create(lib, [p, q], [u, u64], [out, out64], [0, 1]) == 0  # a zero batch skips its item


def test_group_of_empty_items_launches_nothing():
    """Every item with batch 0: the group holds no graph and a launch is a no-op (outputs untouched)."""
    lib = N.load()
    p = ConvPlan("log", n=32, period=3, precision="fp32", io="r2r", batch_max=1, scale=-INV2PI)
    u = _u(p, 1, 5)
    out = torch.full_like(u, 7.0)
    k = 1
    arr = ctypes.c_void_p * k
    h = ctypes.c_void_p()
    assert lib.conv_group_create(k, arr(p.handle.value), arr(u.data_ptr()), None, arr(out.data_ptr()),
                                 (ctypes.c_int * k)(0), ctypes.byref(h)) == 0
    assert lib.conv_group_launch(h, None) == 0
    torch.cuda.synchronize()
    assert torch.all(out == 7.0)
    lib.conv_group_destroy(h)
