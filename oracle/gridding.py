"""Large-N mode of the FP64 oracle: Ker and A*b by a gridding NUFFT -- test infrastructure only.

Only the tests, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg may use
this module; the product path never does.

Ker (eq. kernel) and A*b (eq. backprojection) are type-1 non-uniform Fourier sums,
f(n) = sum_p c_p exp(+i <n, xi_p>) over the slice points xi_p of eq. forward-projector.
The direct sums in `oracle.firm` cost O(M |K| L^3) and stop being feasible near N = 64
with thousands of images.  This module evaluates the same sums as a type-1 NUFFT
(Dutt & Rokhlin 1993), the method the paper itself relies on (Fessler's NUFFT, Section 4):

  1. spread: tau[j] = sum_p c_p phi(j - u_p) on a periodic grid of G = sigma L points
     per axis, u_p = G xi_p / 2 pi, with a separable window phi of width W
     (oracle/gridding.c, plain C in FP64);
  2. F(n) = sum_j tau[j] exp(+2 pi i <n, j> / G), a library FFT (scipy.fft);
  3. f(n) = F(n) / (phi_hat(n1/G) phi_hat(n2/G) phi_hat(n3/G)) for n in [-L/2, L/2)^3,
     phi_hat(nu) = integral of phi(t) exp(2 pi i nu t) dt.

Step 3 is exact up to the aliased terms phi_hat(n/G - k), k != 0 (Poisson summation),
whose size the window sets.  Two windows:

  * "es": exponential of semicircle, exp(beta (sqrt(1 - (2t/W)^2) - 1)), beta = 2.3 W
    (Barnett, Magland & af Klinteberg 2019), phi_hat by Gauss-Legendre quadrature.
    With W = 12 at sigma = 2 the sums agree with the direct sums to ~1e-12 relative
    L2 (pinned in tests/test_oracle.py), which is what makes this the oracle at large N.
  * "kb": Kaiser-Bessel I0(beta sqrt(1 - (2t/W)^2)) with Beatty's beta
    (Beatty, Nishimura & Pauly 2005) and its analytic transform
    W sinh(z)/z, z = sqrt(beta^2 - (pi W nu)^2).  At W = 6 this is the NUFFT the
    configurations name, evaluated in FP64: the method's own approximation without
    any FP32 rounding.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import firm as _F

__all__ = ["build", "window_ft", "es_beta", "kb_beta", "type1_gridded", "kernel_gridded",
           "adjoint_gridded", "backproject_gridded", "default_threads"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gridding.c")
_SO = os.path.join(_HERE, "_gridding.so")
_lib = None


def build() -> str:
    """Compile oracle/gridding.c into oracle/_gridding.so (gcc, OpenMP) when stale."""
    if not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        lib.oracle_spread_slices.argtypes = [i, p, i, p, i, p, i, i, i, i, d, i, p]
        lib.oracle_spread_slices.restype = i
        lib.oracle_max_threads.restype = i
        _lib = lib
    return _lib


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def es_beta(W: int) -> float:
    """Exponential-of-semicircle shape parameter for sigma = 2 (Barnett et al. 2019)."""
    return 2.30 * W


def kb_beta(W: int, sigma: float = 2.0) -> float:
    """Kaiser-Bessel shape parameter of Beatty, Nishimura & Pauly (2005)."""
    return float(np.pi * np.sqrt((W / sigma) ** 2 * (sigma - 0.5) ** 2 - 0.8))


def _window(t, W, window, beta):
    s = np.sqrt(np.maximum(1.0 - (2.0 * np.asarray(t, float) / W) ** 2, 0.0))
    if window == "kb":
        return np.i0(beta * s)
    return np.exp(beta * (s - 1.0))


def window_ft(nu, W: int, window: str, beta: float, quadrature: bool | None = None) -> np.ndarray:
    """phi_hat(nu) = integral over [-W/2, W/2] of phi(t) cos(2 pi nu t) dt (phi is even).

    Kaiser-Bessel: the analytic transform W sinh(z)/z, z = sqrt(beta^2 - (pi W nu)^2)
    (sin for imaginary z); quadrature=True evaluates it by Gauss-Legendre instead (used
    to pin the formula).  Exponential of semicircle: Gauss-Legendre, 400 nodes."""
    nu = np.asarray(nu, float)
    if window == "kb" and not quadrature:
        a = (np.pi * W * nu) ** 2
        z2 = beta * beta - a
        z = np.sqrt(np.abs(z2))
        out = W * np.sinc(z / np.pi)                        # sin(z)/z where z2 < 0
        pos = z2 > 0
        out[pos] = W * np.sinh(z[pos]) / z[pos]
        return out
    x, wq = np.polynomial.legendre.leggauss(400)
    t = 0.5 * W * x
    phi = _window(t, W, window, beta) * (0.5 * W) * wq
    return np.cos(2.0 * np.pi * np.outer(nu.ravel(), t)) @ phi


def type1_gridded(R, K, N, weights, L, *, W=12, window="es", sigma=2, beta=None, threads=None,
                  chunk=1024, spread_only=False, timing=None):
    """f(n) = sum_{m,k} weights(m, k) exp(+i <n, xi_{m,k}>) for n in [-L/2, L/2)^3, stored
    [n3][n2][n1] (complex), by steps 1-3 of the module docstring.

    R is (M, 3, 3); K the disc (|K|, 2); weights a callable weights(a, b) returning the
    (b - a, |K|) weights of images a..b-1 (real or complex), so that no (M, |K|) array
    has to exist at once.  timing (a dict, optional) receives the seconds of step 1
    (with the weights) and of steps 2-3."""
    import time
    t_start = time.perf_counter()
    lib = _load()
    threads = threads or default_threads()
    beta = (es_beta(W) if window == "es" else kb_beta(W, sigma)) if beta is None else beta
    G = int(sigma * L)
    M = R.shape[0]
    Kc = np.ascontiguousarray(K, dtype=np.int32)
    Rf = np.ascontiguousarray(R.reshape(M, 9), dtype=np.float64)
    tau = None
    cplx = None
    for a in range(0, M, chunk):
        b = min(M, a + chunk)
        w = np.asarray(weights(a, b))
        if cplx is None:
            cplx = np.iscomplexobj(w)
            tau = np.zeros((G, G, G), complex if cplx else float)
        w = np.ascontiguousarray(w, dtype=complex if cplx else float)
        st = lib.oracle_spread_slices(b - a, Rf[a:].ctypes.data, Kc.shape[0], Kc.ctypes.data, int(N),
                                      w.ctypes.data, int(cplx), G, int(W), 0 if window == "kb" else 1,
                                      float(beta), int(threads), tau.ctypes.data)
        if st != 0:
            raise ValueError("oracle_spread_slices refused its arguments")
    if tau is None:
        tau = np.zeros((G, G, G))
    t_spread = time.perf_counter()
    if timing is not None:
        timing["spread_s"] = t_spread - t_start
    if spread_only:
        return tau
    import scipy.fft
    F = scipy.fft.ifftn(tau, workers=threads) * float(G) ** 3
    del tau
    n = np.arange(-L // 2, L // 2)
    sel = n % G
    F = F[np.ix_(sel, sel, sel)]
    d = window_ft(n / G, W, window, beta)
    out = F / (d[:, None, None] * d[None, :, None] * d[None, None, :])
    if timing is not None:
        timing["transform_s"] = time.perf_counter() - t_spread
    return out


def _group_h(N, K, groups, group_id):
    """Per-group CTF table (G, |K|) and the group of every image (all ones without groups)."""
    groups = np.asarray(groups, float).reshape(-1, 6)
    M = len(group_id)
    if groups.shape[0] == 0:
        return np.ones((1, K.shape[0])), np.zeros(M, np.int64)
    kk = np.sqrt((K.astype(float) ** 2).sum(1))
    table = np.stack([_F.ctf(kk / (N * g[4]), g) for g in groups])
    return table, np.asarray(group_id, np.int64)


def kernel_gridded(R, groups, group_id, K, N, **kw):
    """Ker(n) = sum_m sum_k h_m(|w_k|)^2 exp(+i <n, xi_{m,k}>), n in [-N, N)^3 (eq. kernel),
    as a gridding NUFFT.  Complex (2N)^3 stored [n3+N][n2+N][n1+N], like oracle.kernel."""
    table, gid = _group_h(N, K, groups, group_id)
    return type1_gridded(R, K, N, lambda a, b: table[gid[a:b]] ** 2, 2 * N, **kw)


def adjoint_gridded(g, R, h, K, N, **kw):
    """(A* g)(n) (eq. backprojection) for sample values g and CTF weights h, both (M, |K|)."""
    return type1_gridded(R, K, N, lambda a, b: h[a:b] * g[a:b], N, **kw)


def backproject_gridded(images, shifts, R, groups, group_id, K, **kw):
    """A*b of FIRM steps 1-2 (eq. measurement, eq. backprojection) as a gridding NUFFT: the
    image DFTs on the disc with the shift phase (oracle.image_dft), weighted by the CTF,
    spread and transformed.  Real N^3 volume (reading 7), images taken chunk by chunk."""
    N = images.shape[1]
    table, gid = _group_h(N, K, groups, group_id)

    def weights(a, b):
        return table[gid[a:b]] * _F.image_dft(np.asarray(images[a:b], np.float64), K, shifts[a:b])

    return type1_gridded(R, K, N, weights, N, **kw).real
