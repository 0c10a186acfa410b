"""Plain FP64 CPU oracle for the FFT convolution of arXiv 2107.03958 (Tiwari, Pandey, Paul, Anand).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library: the arithmetic lives in
``orc.c`` (plain C, FP64/complex128, no pruning or fusion); this module only marshals numpy arrays.

Functions and the passage each follows:
  fft / ifft / fft2          discrete Fourier transform used by eq. (An), Sec. 2.1
  ghat_radial / ghat_full    moments ghat(k), eq. (ghat) and its closed forms, Sec. 2.2
  conv                       A_n u, eq. (An), Sec. 2.1
  direct                     quadrature form eq. (quad)/(quad_wts), Sec. 2.1 (O(n^4) sum)
  fs_mask                    chi^n_Omega psi, eq. (tfs) and the window psi, Sec. 2.4
  ls_apply / gmres           Nystrom system eq. (descretls), Sec. 3.3
  default_trunc_radius       the admissible truncation radius a of eq. (io), Sec. 2.1
  bessel_k / yukawa moments  K0, K1 and the Yukawa kernel K0(kappa|x|)/(2 pi) of Sec. 3.2
  ghat_numeric_full          moments by quadrature after rho = tau^p, eq. (cc_pts)/(cc_wts), Sec. 2.3
  eta / ghat_localized_full  localization, eq. (io_split), Sec. 2.3
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

LOG, POW, HELM, YUKAWA = 0, 1, 2, 3
_KIND = {"log": LOG, "pow": POW, "helmholtz": HELM, "helm": HELM, "yukawa": YUKAWA}

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        L.orc_fft.argtypes = [i, p, i]
        L.orc_fft2.argtypes = [i, i, p, i, d]
        L.orc_ghat_radial.argtypes = [i, d, d, d, d, d, d, p]
        L.orc_ghat_helm_resonant.argtypes = [d, d, d, p]
        L.orc_ghat_helm_quad.argtypes = [d, d, d, d, p]
        L.orc_ghat_full.argtypes = [i, d, d, d, d, d, i, p]
        L.orc_pow_moment.argtypes = [d, d]
        L.orc_pow_moment.restype = d
        L.orc_conv.argtypes = [i, i, p, p, p, i]
        L.orc_conv.restype = i
        L.orc_direct.argtypes = [i, i, p, p, p, i, i]
        L.orc_direct.restype = i
        L.orc_weights.argtypes = [i, i, p, p]
        L.orc_weights.restype = i
        L.orc_fs_mask.argtypes = [i, i, d, i, p, d, p]
        L.orc_fs_mask.restype = i
        L.orc_varkappa.argtypes = [d]
        L.orc_varkappa.restype = d
        L.orc_psi1.argtypes = [d, d]
        L.orc_psi1.restype = d
        L.orc_ls_apply.argtypes = [i, i, p, d, p, p, p]
        L.orc_gmres.argtypes = [i, i, p, d, p, p, p, i, i, d, p, p]
        L.orc_gmres.restype = i
        L.orc_max_threads.restype = i
        L.orc_bessel_k.argtypes = [i, d]
        L.orc_bessel_k.restype = d
        L.orc_yukawa_moment.argtypes = [d, d, d]
        L.orc_yukawa_moment.restype = d
        L.orc_cc_rule.argtypes = [i, d, p, p]
        L.orc_ghat_numeric_full.argtypes = [i, d, d, d, d, d, i, i, i, p]
        L.orc_ghat_numeric_full.restype = i
        L.orc_eta.argtypes = [d, d]
        L.orc_eta.restype = d
        L.orc_ghat_localized_full.argtypes = [i, d, d, d, d, d, i, d, i, i, p]
        L.orc_ghat_localized_full.restype = i
        L.orc_ghat_full_dx1log.argtypes = [d, d, d, i, p]
        L.orc_set_threads.argtypes = [i]
        _lib = L
    return _lib


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def threads():
    return lib().orc_max_threads()


def set_threads(t):
    lib().orc_set_threads(int(t))


# ---------------------------------------------------------------- DFT
def fft(x, sign=-1):
    """Unnormalised DFT  X[k] = sum_j x[j] exp(sign 2 pi i jk/N)."""
    a = _c128(x).copy()
    lib().orc_fft(a.size, _ptr(a), int(sign))
    return a


def fft2(x, sign=-1, scale=1.0):
    a = _c128(x).copy()
    R, C = a.shape
    lib().orc_fft2(R, C, _ptr(a), int(sign), float(scale))
    return a


# ---------------------------------------------------------------- moments (Sec. 2.2)
def default_trunc_radius(b):
    """Midpoint of the admissible interval sqrt(2) <= a <= b - 1 of eq. (io) for support D."""
    if b - 1.0 < math.sqrt(2.0):
        raise ValueError("period b=%g admits no truncation radius for support D" % b)
    return 0.5 * (math.sqrt(2.0) + b - 1.0)


def ghat_radial(kind, kmag, b, a, gamma=0.0, kappa=0.0, scale=1.0):
    out = np.zeros(2)
    lib().orc_ghat_radial(_KIND[kind], float(gamma), float(kappa), float(scale), float(b),
                          float(a), float(kmag), _ptr(out))
    return complex(out[0], out[1])


def ghat_helm_resonant(kappa, a, scale=1.0):
    out = np.zeros(2)
    lib().orc_ghat_helm_resonant(float(kappa), float(scale), float(a), _ptr(out))
    return complex(out[0], out[1])


def ghat_helm_quad(kappa, s, a, scale=1.0):
    out = np.zeros(2)
    lib().orc_ghat_helm_quad(float(kappa), float(scale), float(s), float(a), _ptr(out))
    return complex(out[0], out[1])


def pow_moment(gamma, z):
    """I(z) = int_0^z t^(1+gamma) J0(t) dt."""
    return lib().orc_pow_moment(float(gamma), float(z))


def ghat_full(kind, M, b, a, gamma=0.0, kappa=0.0, scale=1.0):
    """M x M table of ghat(k), k in F_n, at FFT index q (k = q for q < M/2 else q - M).
    kind 'dx1log': the non-radial kernel -x1/(2 pi |x|^2) of Sec. 3.1 (odd in k1)."""
    out = np.zeros((M, M), dtype=np.complex128)
    if kind == "dx1log":
        lib().orc_ghat_full_dx1log(float(scale), float(b), float(a), int(M), _ptr(out))
        return out
    lib().orc_ghat_full(_KIND[kind], float(gamma), float(kappa), float(scale), float(b),
                        float(a), int(M), _ptr(out))
    return out


# ---------------------------------------------------------------- moments without a closed form (Sec. 2.3)
def bessel_k(nu, x):
    """K_nu(x), nu in {0, 1}, by its integral representation."""
    return lib().orc_bessel_k(int(nu), float(x))


def yukawa_moment(kappa, s, a):
    """2 pi int_0^a K0(kappa rho)/(2 pi) J0(s rho) rho d rho (closed form), unscaled."""
    return lib().orc_yukawa_moment(float(kappa), float(s), float(a))


def cc_rule(npc, alpha):
    """Points and weights of eq. (cc_pts), (cc_wts) on [0, alpha]."""
    x, w = np.zeros(npc), np.zeros(npc)
    lib().orc_cc_rule(int(npc), float(alpha), _ptr(x), _ptr(w))
    return x, w


def ghat_numeric_full(kind, M, b, a, gamma=0.0, kappa=0.0, scale=1.0, p=4, npc=512):
    """M x M table of ghat(k) by the quadrature of Sec. 2.3 (rho = tau^p, npc-point rule)."""
    out = np.zeros((M, M), dtype=np.complex128)
    rc = lib().orc_ghat_numeric_full(_KIND[kind], float(gamma), float(kappa), float(scale), float(b),
                                     float(a), int(p), int(npc), int(M), _ptr(out))
    if rc:
        raise RuntimeError("orc_ghat_numeric_full failed (%d)" % rc)
    return out


def eta(rho, beta):
    return lib().orc_eta(float(rho), float(beta))


def ghat_localized_full(kind, n, b, a, beta, gamma=0.0, kappa=0.0, scale=1.0, p=4, npc=2048):
    """M x M multiplier of the localized scheme, eq. (io_split): moments of g eta_beta plus the
    DFT of the trapezoidal weights of g (1 - eta_beta)."""
    M = int(round(n * b))
    out = np.zeros((M, M), dtype=np.complex128)
    rc = lib().orc_ghat_localized_full(_KIND[kind], float(gamma), float(kappa), float(scale), float(b),
                                       float(a), int(n), float(beta), int(p), int(npc), _ptr(out))
    if rc:
        raise RuntimeError("orc_ghat_localized_full failed (%d)" % rc)
    return out


# ---------------------------------------------------------------- the scheme (Sec. 2.1)
def conv(u, M, ghat):
    """A_n u = crop_n(ifft2(ghat * fft2(zero-extend_M(u)))), eq. (An).  u: (n,n) or (B,n,n)."""
    u = _c128(u)
    single = u.ndim == 2
    if single:
        u = u[None]
    B, n, _ = u.shape
    g = _c128(ghat)
    assert g.shape == (M, M)
    out = np.zeros_like(u)
    rc = lib().orc_conv(n, M, _ptr(g), _ptr(u), _ptr(out), B)
    if rc:
        raise RuntimeError("orc_conv failed (%d)" % rc)
    return out[0] if single else out


def direct(u, M, ghat, rows=None):
    """Quadrature form eq. (quad): O(n^4) double sum with weights of eq. (quad_wts)."""
    u = _c128(u)
    n = u.shape[0]
    r0, r1 = (0, n) if rows is None else rows
    out = np.zeros((r1 - r0, n), dtype=np.complex128)
    g = _c128(ghat)
    rc = lib().orc_direct(n, M, _ptr(g), _ptr(u), _ptr(out), int(r0), int(r1))
    if rc:
        raise RuntimeError("orc_direct failed (%d)" % rc)
    return out


def weights(n, M, ghat):
    """w(d), d in [-(n-1), n-1]^2 (index d + n - 1), eq. (quad_wts)."""
    D = 2 * n - 1
    out = np.zeros((D, D), dtype=np.complex128)
    g = _c128(ghat)
    rc = lib().orc_weights(n, M, _ptr(g), _ptr(out))
    if rc:
        raise RuntimeError("orc_weights failed (%d)" % rc)
    return out


# ---------------------------------------------------------------- Fourier smoothing (Sec. 2.4)
def varkappa(t):
    return lib().orc_varkappa(float(t))


def psi1(t, delta):
    return lib().orc_psi1(float(t), float(delta))


def fs_mask(n, b, shape, geom, delta=0.15):
    """chi^n_Omega(x_j) psi(x_j) on the n x n grid.  shape 'disk' geom=(c1,c2,r);
    'rect' geom=(x0,x1,y0,y1)."""
    M = int(round(n * b))
    g = np.ascontiguousarray(geom, dtype=np.float64)
    out = np.zeros((n, n))
    rc = lib().orc_fs_mask(n, M, float(b), 0 if shape == "disk" else 1, _ptr(g), float(delta),
                           _ptr(out))
    if rc:
        raise RuntimeError("orc_fs_mask failed (%d)" % rc)
    return out


# ---------------------------------------------------------------- Lippmann-Schwinger (Sec. 3.3)
def ls_apply(x, M, ghat, kappa, m):
    """x + kappa^2 A_n(m x), the Nystrom operator of eq. (descretls)."""
    x = _c128(x)
    n = x.shape[0]
    mm = np.ascontiguousarray(m, dtype=np.float64)
    y = np.zeros_like(x)
    g = _c128(ghat)
    lib().orc_ls_apply(n, M, _ptr(g), float(kappa), _ptr(mm), _ptr(x), _ptr(y))
    return y


def gmres(f, M, ghat, kappa, m, x0=None, restart=50, maxit=2000, tol=1e-10):
    """Restarted GMRES (MGS Arnoldi, Givens) for eq. (descretls). Returns (x, iters, relres, ok)."""
    f = _c128(f)
    n = f.shape[0]
    x = np.zeros_like(f) if x0 is None else _c128(x0).copy()
    mm = np.ascontiguousarray(m, dtype=np.float64)
    g = _c128(ghat)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    rc = lib().orc_gmres(n, M, _ptr(g), float(kappa), _ptr(mm), _ptr(f), _ptr(x), int(restart),
                         int(maxit), float(tol), ctypes.byref(it), ctypes.byref(rr))
    return x, it.value, rr.value, rc == 0


# ---------------------------------------------------------------- error measures (Sec. 3)
def rel_err(exact, approx):
    """eq. (rel-err): max |U_exact - U_approx| / max |U_exact| over the grid."""
    exact = np.asarray(exact)
    return float(np.max(np.abs(exact - approx)) / np.max(np.abs(exact)))


def noc(e_n, e_2n):
    """eq. (ord-conv): log2(eps_n / eps_2n)."""
    return math.log2(e_n / e_2n)
