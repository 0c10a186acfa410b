"""Torch-facing binding of the C ABI (argument marshalling only; every step runs in the CUDA library).

    plan = ConvPlan("log", n=1024, period=3, precision="fp32", io="r2r", batch_max=16, scale=-1/(2*pi))
    out = plan.apply(u)            # u: CUDA tensor (B, n, n) or (n, n)
    x, info = ls_solve(plan_c2c_helmholtz, m, f)

Names follow the paper: n grid points per side on D = [0,1]^2, period b, truncation radius a,
moments ghat (Sec. 2.1-2.2).
"""
import ctypes
import math
from fractions import Fraction

import numpy as np
import torch

from . import _native as N

FAMILY = {"log": 0, "pow": 1, "helmholtz": 2, "helm": 2, "yukawa": 3, "dx1log": 4}
MOMENTS = {"closed": 0, "quadrature": 1, "localized": 2}
PRECISION = {"fp64": 0, "fp32": 1}
IO = {"r2r": 0, "r2c": 1, "c2c": 2}


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class ConvPlan:
    """A plan for A_n on an n x n grid with period b (Sec. 2.1, eq. (An))."""

    def __init__(self, kernel="log", n=64, period=3, trunc_a=0.0, precision="fp64", io="r2r",
                 batch_max=1, gamma=0.0, kappa=0.0, scale=1.0, device=None, compact=False,
                 autotune=False, moments="closed", moment_p=0, moment_nodes=0, beta=0.0):
        """moments: 'closed' (Sec. 2.2 closed forms), 'quadrature' (Sec. 2.3, rho = tau^p) or
        'localized' (Sec. 2.3, eq. (io_split), radius beta)."""
        self._lib = N.load()
        if device is not None:
            torch.cuda.set_device(device)
        frac = Fraction(period).limit_denominator(64)
        self.kernel, self.n, self.b = kernel, int(n), float(frac)
        self.precision, self.io = precision, io
        self.period = (frac.numerator, frac.denominator)
        k = N.ConvKernel(FAMILY[kernel], float(gamma), float(kappa), float(scale))
        h = ctypes.c_void_p()
        mo = N.ConvMoments(MOMENTS[moments], int(moment_p), int(moment_nodes), float(beta))
        N.check(self._lib.conv_plan_moments(ctypes.byref(k), frac.numerator, frac.denominator, int(n),
                                            float(trunc_a), PRECISION[precision], IO[io], int(batch_max),
                                            (1 if compact else 0) | (2 if autotune else 0), ctypes.byref(mo),
                                            ctypes.byref(h)))
        self._h = h
        self.info = self._info()
        self.M, self.a = self.info.M, self.info.a
        self.compact = bool(compact)
        self.real_dtype = torch.float64 if precision == "fp64" else torch.float32
        self.cplx_dtype = torch.complex128 if precision == "fp64" else torch.complex64
        self.batch_max = int(batch_max)

    def _info(self):
        inf = N.ConvPlanInfo()
        N.check(self._lib.conv_get_info(self._h, ctypes.byref(inf)))
        return inf

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.conv_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def in_dtype(self):
        return self.cplx_dtype if self.io == "c2c" else self.real_dtype

    def out_dtype(self):
        return self.real_dtype if self.io == "r2r" else self.cplx_dtype

    def workspace_bytes(self, batch):
        b = ctypes.c_size_t()
        N.check(self._lib.conv_workspace_size(self._h, int(batch), ctypes.byref(b)))
        return b.value

    def _check_grid(self, t, dtype, name):
        if not t.is_cuda:
            raise ValueError("%s must be a CUDA tensor" % name)
        if t.dtype != dtype:
            raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        if t.shape[-2:] != (self.n, self.n):
            raise ValueError("%s must end in (%d, %d)" % (name, self.n, self.n))

    def apply(self, u, mask=None, out=None, workspace=None, stream=None, alpha=1.0, beta=0.0):
        """out = beta u + alpha A_n(u * mask), batched over the leading dimension."""
        self._check_grid(u, self.in_dtype(), "u")
        batch = 1 if u.dim() == 2 else int(np.prod(u.shape[:-2]))
        if out is None:
            out = torch.empty(u.shape, dtype=self.out_dtype(), device=u.device)
        self._check_grid(out, self.out_dtype(), "out")
        if mask is not None:
            self._check_grid(mask, self.real_dtype, "mask")
            if mask.dim() != 2:
                raise ValueError("mask is one n x n array shared by the batch")
        ws = None
        if workspace is not None:
            if workspace.numel() * workspace.element_size() < self.workspace_bytes(batch):
                raise ValueError("workspace too small")
            ws = ctypes.c_void_p(workspace.data_ptr())
        a = complex(alpha)
        N.check(self._lib.conv_apply_axpby(
            self._h, ctypes.c_void_p(u.data_ptr()),
            ctypes.c_void_p(mask.data_ptr()) if mask is not None else None,
            ctypes.c_void_p(out.data_ptr()), batch, a.real, a.imag, float(beta), ws,
            _stream_ptr(stream)))
        return out

    __call__ = apply

    def apply_host(self, u, out=None, mask=None, stream=None):
        """A_n(u * mask) for densities in host memory (CPU tensors; pinned for overlap), with the
        host<->device copies pipelined against the passes; returns `out` (a CPU tensor).  Ordered
        on `stream`; synchronise it before reading `out`."""
        if u.device.type != "cpu":
            raise ValueError("apply_host takes host tensors")
        if u.dtype != self.in_dtype() or tuple(u.shape[-2:]) != (self.n, self.n) or not u.is_contiguous():
            raise ValueError("u must be a contiguous (..., n, n) %s host tensor" % self.in_dtype())
        batch = 1 if u.dim() == 2 else int(np.prod(u.shape[:-2]))
        if out is None:
            out = torch.empty(u.shape, dtype=self.out_dtype()).pin_memory()
        if out.device.type != "cpu" or out.dtype != self.out_dtype() or out.shape != u.shape or not out.is_contiguous():
            raise ValueError("out must be a contiguous host tensor of u's shape and %s" % self.out_dtype())
        if mask is not None:
            self._check_grid(mask, self.real_dtype, "mask")
        N.check(self._lib.conv_apply_host(
            self._h, ctypes.c_void_p(u.data_ptr()),
            ctypes.c_void_p(mask.data_ptr()) if mask is not None else None,
            ctypes.c_void_p(out.data_ptr()), batch, _stream_ptr(stream)))
        return out

    def fs_mask(self, shape, geom, delta=0.15, stream=None):
        """Fourier-smoothed indicator chi^n psi on the n x n grid (Sec. 2.4, eq. (tfs)).
        shape 'disk': geom = (c1, c2, r); 'rect': geom = (x0, x1, y0, y1)."""
        g = np.ascontiguousarray(geom, dtype=np.float64)
        mask = torch.empty((self.n, self.n), dtype=self.real_dtype, device="cuda")
        N.check(self._lib.conv_fs_mask(self._h, 0 if shape == "disk" else 1,
                                       g.ctypes.data_as(ctypes.c_void_p), float(delta),
                                       ctypes.c_void_p(mask.data_ptr()), _stream_ptr(stream)))
        return mask

    def device_status(self, stream=None):
        """Synchronise `stream` and raise if a pass kernel's bounded wait for an asynchronous copy
        gave up since the last check (the applies since then are incomplete)."""
        N.check(self._lib.conv_device_status(self._h, _stream_ptr(stream)))

    def timing(self, enable):
        """Record per-pass CUDA events on every apply (benchmark instrumentation)."""
        N.check(self._lib.conv_timing_enable(self._h, int(bool(enable))))

    def timing_read(self):
        """(ms per pass summed over recorded applies [3], number of applies); clears the record."""
        ms = (ctypes.c_double * 3)()
        cnt = ctypes.c_longlong()
        N.check(self._lib.conv_timing_read(self._h, ms, ctypes.byref(cnt)))
        return [ms[0], ms[1], ms[2]], cnt.value

    def ghat_quadrant(self):
        """FP64 moment table ghat(|k1|, |k2|), 0 <= k1, k2 <= M/2, as numpy [k2, k1]."""
        h = self.M // 2 + 1
        cplx = self.kernel in ("helmholtz", "helm")
        buf = np.zeros((h, h), dtype=np.complex128 if cplx else np.float64)
        N.check(self._lib.conv_ghat_to_host(self._h, buf.ctypes.data_as(ctypes.c_void_p)))
        return buf


def apply_kernels(shape, plans, u, out=None, mask=None, workspace=None, stream=None):
    """out[b] = A_n(u[b] * mask) with plans[b]'s kernel, every plan of shape's n, period, precision,
    io and embedding, in one launch of each pass on `shape` (see conv_apply_kernels)."""
    shape._check_grid(u, shape.in_dtype(), "u")
    batch = 1 if u.dim() == 2 else int(np.prod(u.shape[:-2]))
    if len(plans) != batch:
        raise ValueError("one plan per density")
    if out is None:
        out = torch.empty(u.shape, dtype=shape.out_dtype(), device=u.device)
    shape._check_grid(out, shape.out_dtype(), "out")
    arr = (ctypes.c_void_p * batch)(*[p.handle.value for p in plans])
    N.check(shape._lib.conv_apply_kernels(
        shape.handle, arr, ctypes.c_void_p(u.data_ptr()),
        ctypes.c_void_p(mask.data_ptr()) if mask is not None else None, ctypes.c_void_p(out.data_ptr()),
        batch, ctypes.c_void_p(workspace.data_ptr()) if workspace is not None else None, _stream_ptr(stream)))
    return out


def apply_multi(plans, u, outs=None, mask=None, workspace=None, stream=None):
    """A_n(u * mask) with every plan in `plans` (R2R or split R2C plans of one grid, precision and
    embedding) on the same device densities `u`, pass 1's row transforms computed once (see
    conv_apply_multi).  Returns the list of outputs."""
    p0 = plans[0]
    p0._check_grid(u, p0.in_dtype(), "u")
    batch = 1 if u.dim() == 2 else int(np.prod(u.shape[:-2]))
    if outs is None:
        outs = [torch.empty(u.shape, dtype=p.out_dtype(), device=u.device) for p in plans]
    for p, o in zip(plans, outs):
        p._check_grid(o, p.out_dtype(), "out")
    arr = (ctypes.c_void_p * len(plans))(*[p.handle.value for p in plans])
    oarr = (ctypes.c_void_p * len(plans))(*[o.data_ptr() for o in outs])
    N.check(p0._lib.conv_apply_multi(
        arr, len(plans), ctypes.c_void_p(u.data_ptr()),
        ctypes.c_void_p(mask.data_ptr()) if mask is not None else None, oarr, batch,
        ctypes.c_void_p(workspace.data_ptr()) if workspace is not None else None, _stream_ptr(stream)))
    return outs


def multi_workspace_bytes(plans, batch):
    arr = (ctypes.c_void_p * len(plans))(*[p.handle.value for p in plans])
    b = ctypes.c_size_t()
    N.check(plans[0]._lib.conv_multi_workspace_size(arr, len(plans), int(batch), ctypes.byref(b)))
    return b.value


def apply_host_multi(plans, u, outs=None, mask=None, stream=None):
    """A_n(u * mask) with every plan in `plans` for one batch of host densities `u` (a CPU tensor;
    pinned for overlap): each chunk is uploaded once and the plans run on it in turn.  The plans
    share n, precision and input type.  Returns the list of host results (pinned CPU tensors
    unless `outs` is given), ordered on `stream`; synchronise it before reading them."""
    plans = list(plans)
    if not plans:
        raise ValueError("at least one plan")
    p0 = plans[0]
    if u.device.type != "cpu" or u.dtype != p0.in_dtype() or tuple(u.shape[-2:]) != (p0.n, p0.n) or not u.is_contiguous():
        raise ValueError("u must be a contiguous (..., n, n) %s host tensor" % p0.in_dtype())
    batch = 1 if u.dim() == 2 else int(np.prod(u.shape[:-2]))
    if outs is None:
        outs = [torch.empty(u.shape, dtype=p.out_dtype()).pin_memory() for p in plans]
    if len(outs) != len(plans):
        raise ValueError("one output per plan")
    for p, o in zip(plans, outs):
        if o.device.type != "cpu" or o.dtype != p.out_dtype() or o.shape != u.shape or not o.is_contiguous():
            raise ValueError("each output must be a contiguous host tensor of u's shape and its plan's dtype")
    if mask is not None:
        p0._check_grid(mask, p0.real_dtype, "mask")
    k = len(plans)
    arr = ctypes.c_void_p * k
    N.check(p0._lib.conv_apply_host_multi(
        k, arr(*[p.handle.value for p in plans]), ctypes.c_void_p(u.data_ptr()),
        ctypes.c_void_p(mask.data_ptr()) if mask is not None else None,
        arr(*[o.data_ptr() for o in outs]), batch, _stream_ptr(stream)))
    return outs


class ConvGroup:
    """Several applies, on plans that may differ in n, kernel, precision and io, run as one CUDA
    graph launch (items on different plans run concurrently; items on one plan in order).

        g = ConvGroup([(plan_a, u_a, out_a), (plan_b, u_b, out_b, mask_b)])
        g.launch()      # out_i = A_n(u_i * mask_i) for every item, one graph launch

    The tensors are fixed at creation: launch() reads and writes the same storage every time
    (its contents may change between launches); the group keeps the plans and tensors alive."""

    def __init__(self, items):
        self._lib = N.load()
        plans, us, masks, outs, batches = [], [], [], [], []
        for it in items:
            plan, u, out = it[0], it[1], it[2]
            mask = it[3] if len(it) > 3 else None
            plan._check_grid(u, plan.in_dtype(), "u")
            plan._check_grid(out, plan.out_dtype(), "out")
            if out.shape != u.shape:
                raise ValueError("out must have u's shape")
            if mask is not None:
                plan._check_grid(mask, plan.real_dtype, "mask")
            plans.append(plan.handle.value)
            us.append(u.data_ptr())
            outs.append(out.data_ptr())
            masks.append(mask.data_ptr() if mask is not None else None)
            batches.append(1 if u.dim() == 2 else int(np.prod(u.shape[:-2])))
        k = len(plans)
        arr = ctypes.c_void_p * k
        h = ctypes.c_void_p()
        N.check(self._lib.conv_group_create(k, arr(*plans), arr(*us), arr(*masks), arr(*outs),
                                            (ctypes.c_int * k)(*batches), ctypes.byref(h)))
        self._h = h
        self._keep = list(items)

    def launch(self, stream=None):
        N.check(self._lib.conv_group_launch(self._h, _stream_ptr(stream)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.conv_group_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ls_solve(plan, m, f, x=None, restart=50, max_iters=2000, tol=1e-10, refine=False,
             inner_tol=1e-5, stream=None):
    """Solve u + kappa^2 A_n(m u) = f (Sec. 3.3, eq. (descretls)) by restarted GMRES.
    m: (n, n) float64 CUDA tensor; f: (n, n) complex128 CUDA tensor; x: optional initial guess."""
    if plan.io != "c2c" or plan.kernel not in ("helmholtz", "helm"):
        raise ValueError("ls_solve needs a C2C Helmholtz plan")
    plan._check_grid(m, torch.float64, "m")
    plan._check_grid(f, torch.complex128, "f")
    zero = x is None
    if x is None:
        x = torch.zeros_like(f)
    plan._check_grid(x, torch.complex128, "x")
    o = N.LsOpts(int(restart), int(max_iters), float(tol), int(bool(refine)), float(inner_tol), int(zero))
    inf = N.LsInfo()
    st = plan._lib.ls_solve(plan.handle, ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                            ctypes.c_void_p(x.data_ptr()), ctypes.byref(o), ctypes.byref(inf),
                            _stream_ptr(stream))
    info = {"iters": inf.iters, "restarts": inf.restarts, "refinements": inf.refinements,
            "rel_residual": inf.rel_residual, "status": N.STATUS.get(st, st)}
    if st not in (0, 6):
        N.check(st)
    return x, info


def ls_solve_multi(plan, m, F, X=None, restart=50, max_iters=2000, tol=1e-10, refine=False,
                   inner_tol=1e-5, stream=None):
    """Solve u_s + kappa^2 A_n(m u_s) = f_s for every right-hand side F[s] (one operator, one
    contrast m) as one stacked GMRES whose matvecs are batched applies.
    F: (K, n, n) complex128 CUDA tensor; returns (X, [info per system])."""
    if plan.io != "c2c" or plan.kernel not in ("helmholtz", "helm"):
        raise ValueError("ls_solve_multi needs a C2C Helmholtz plan")
    plan._check_grid(m, torch.float64, "m")
    plan._check_grid(F, torch.complex128, "F")
    if F.dim() != 3:
        raise ValueError("F must be (K, n, n)")
    K = int(F.shape[0])
    zero = X is None
    if X is None:
        X = torch.zeros_like(F)
    plan._check_grid(X, torch.complex128, "X")
    if X.shape != F.shape:
        raise ValueError("X must have F's shape")
    o = N.LsOpts(int(restart), int(max_iters), float(tol), int(bool(refine)), float(inner_tol), int(zero))
    infs = (N.LsInfo * K)()
    st = plan._lib.ls_solve_multi(plan.handle, K, ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(F.data_ptr()),
                                  ctypes.c_void_p(X.data_ptr()), ctypes.byref(o), infs, _stream_ptr(stream))
    status = N.STATUS.get(st, st)
    if st not in (0, 6):
        N.check(st)
    return X, [{"iters": i.iters, "restarts": i.restarts, "refinements": i.refinements,
                "rel_residual": i.rel_residual, "status": status} for i in infs]


class Server:
    """Continuous-batching request loop (C++ runtime in the library; see srv_* in wsconv.h).

    submit_conv / submit_ls return tickets; wait(ticket) returns the result record.  The tensors of
    a request must stay alive until its wait returns (the server keeps references until then)."""

    def __init__(self, mem_budget_bytes=150 << 30, max_inflight=64, conv_batch_max=16, ls_workers=4,
                 compact=False):
        self._lib = N.load()
        h = ctypes.c_void_p()
        N.check(self._lib.srv_create(int(mem_budget_bytes), int(max_inflight), int(conv_batch_max),
                                     int(ls_workers), 1 if compact else 0, ctypes.byref(h)))
        self.compact = bool(compact)
        self._h = h
        self._keep = {}

    def _submit(self, req, keep):
        t = ctypes.c_longlong()
        N.check(self._lib.srv_submit(self._h, ctypes.byref(req), ctypes.byref(t)))
        self._keep[t.value] = keep
        return t.value

    def submit_conv(self, u, out, kernel="log", period=3, precision="fp32", io="r2r", mask=None,
                    gamma=0.0, kappa=0.0, scale=1.0):
        frac = Fraction(period).limit_denominator(64)
        r = N.SrvRequest(0, N.ConvKernel(FAMILY[kernel], float(gamma), float(kappa), float(scale)),
                         int(u.shape[-1]), frac.numerator, frac.denominator, PRECISION[precision],
                         IO[io], u.data_ptr(), mask.data_ptr() if mask is not None else None, None,
                         out.data_ptr(), 0.0, 0, 0)
        return self._submit(r, (u, out, mask))

    def submit_ls(self, m, f, x, kappa, period=3, precision="fp64", tol=1e-10, restart=50,
                  max_iters=2000):
        frac = Fraction(period).limit_denominator(64)
        r = N.SrvRequest(1, N.ConvKernel(2, 0.0, float(kappa), 1.0), int(f.shape[-1]),
                         frac.numerator, frac.denominator, PRECISION[precision], IO["c2c"],
                         f.data_ptr(), None, m.data_ptr(), x.data_ptr(), float(tol), int(restart),
                         int(max_iters))
        return self._submit(r, (m, f, x))

    def wait(self, ticket, timeout_s=0.0):
        res = N.SrvResult()
        N.check(self._lib.srv_wait(self._h, int(ticket), float(timeout_s), ctypes.byref(res)))
        self._keep.pop(ticket, None)
        return {"status": N.STATUS.get(res.status, res.status), "t_submit": res.t_submit,
                "t_start": res.t_start, "t_done": res.t_done, "batched_with": res.batched_with,
                "iters": res.iters, "rel_residual": res.rel_residual,
                "latency_s": res.t_done - res.t_submit}

    def cancel(self, ticket):
        """Cancel a request that has not been admitted yet; its wait then reports CONV_ECANCELLED."""
        N.check(self._lib.srv_cancel(self._h, int(ticket)))

    def stats(self):
        st = N.SrvStats()
        N.check(self._lib.srv_get_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in N.SrvStats._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.srv_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_peaks(nbytes=1 << 30):
    """Measured HBM copy GB/s and FP64/FP32 FMA TFLOP/s on the current GPU."""
    lib = N.load()
    c, d, s = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    N.check(lib.conv_measure_peaks(int(nbytes), ctypes.byref(c), ctypes.byref(d), ctypes.byref(s)))
    return {"copy_gbs": c.value, "fp64_tflops": d.value, "fp32_tflops": s.value}


def fault_inject(kind, count=1):
    """Arm `count` host-side injected faults of one kind ('alloc', 'wait' or 'drop'; see
    conv_fault_inject in wsconv.h); count 0 disarms it."""
    N.check(N.load().conv_fault_inject(N.FAULT[kind], int(count)))


def measure_tc_stage(reps=2000):
    """One radix-16 stage of a length-8192 FP32 column on the CUDA cores and as a tensor-core
    DFT-matrix product (see conv_measure_tc_stage): microseconds per stage per column and the
    tensor-core result's max relative difference."""
    lib = N.load()
    a, b, e = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    N.check(lib.conv_measure_tc_stage(int(reps), ctypes.byref(a), ctypes.byref(b), ctypes.byref(e)))
    return {"us_cuda_core": a.value, "us_tensor": b.value, "max_rel_err": e.value}


def default_scale(kernel):
    """The paper's Laplace kernel is -(1/2pi) log|x|."""
    return -1.0 / (2.0 * math.pi) if kernel == "log" else 1.0
