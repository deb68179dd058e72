"""FP64 oracle of the learned Fourier-domain CG preconditioner -- test infrastructure only.

Not in the paper (an addition to it; the paper's CG, Section 3.3, is
unpreconditioned).  Definitions:

  * bins: a frequency vector q (in units of the N-grid, |q| <= ~N/2) falls in shell
    s = min(63, floor(64 |q| / (N/2))) and cone c = min(15, floor(16 |<q/|q|, a>|))
    (q = 0: cone 0), a the principal axis of the viewing directions (the eigenvector
    of the largest eigenvalue of the second-moment tensor of R_m^T e3); bin = 16 s + c.
  * features: the h^2-weighted sample density per bin, f_b = sum of h_m(|k|)^2 over the
    slice samples xi_{m,k} (in N-grid units xi N / (2 pi)) falling in bin b, divided by
    the total sum of h^2.  A sample's shell uses |xi N / (2 pi)| = |k| exactly (rotations
    keep the norm), so samples on a shell edge are binned without rounding ambiguity.
  * target: the least-squares per-bin multiplier of the circulant spectrum kappa
    (T. Chan's circulant, oracle.firm.wrapped_spectrum) on the N^3 frequency grid,
    p_b = sum_{q in b} (kappa_q + lam) / sum_{q in b} (kappa_q + lam)^2, reported as
    t_b = log(p_b * Ker(0)) (scale-free); empty bins take the value of the nearest
    non-empty shell of the same cone.
  * network: x -> relu(W1 x + b1) -> relu(W2 . + b2) -> W3 . + b3, widths
    1024 -> 256 -> 256 -> 1024, input x_b = log(1024 f_b + 1e-3), loss = mean squared
    error against t; Adam (beta1 0.9, beta2 0.999, eps 1e-8).
  * baseline: t_b ~ -log(f_b / v_b + lambda / Ker(0)), v_b the fraction of the N^3
    frequency grid in bin b; the learned preconditioner is trained on target - baseline.
Pins: finite-difference gradients, closed-form targets for a constant spectrum, and
feature sums; bin volumes sum to 1 and match a direct count.
"""
from __future__ import annotations

import numpy as np

SHELLS, CONES = 64, 16
NBINS = SHELLS * CONES
WIDTHS = (NBINS, 256, 256, NBINS)


def principal_axis(R: np.ndarray) -> np.ndarray:
    """Eigenvector of the largest eigenvalue of mean(d d^T), d = R^T e3 (third rows of R)."""
    d = R[:, 2, :]
    Mt = d.T @ d / max(1, d.shape[0])
    w, V = np.linalg.eigh(Mt)
    a = V[:, -1]
    return a / np.linalg.norm(a)


def bin_index(q: np.ndarray, N: int, a: np.ndarray, r=None) -> np.ndarray:
    """Bin of each frequency vector q (..., 3) in N-grid units (r: its norm, if known exactly)."""
    if r is None:
        r = np.sqrt((q * q).sum(-1))
    s = np.minimum(SHELLS - 1, np.floor(SHELLS * r / (N / 2))).astype(np.int64)
    with np.errstate(invalid="ignore", divide="ignore"):
        cosv = np.abs(q @ a) / r
    cosv = np.where(r > 0, cosv, 0.0)
    c = np.minimum(CONES - 1, np.floor(CONES * cosv)).astype(np.int64)
    return CONES * s + c


def features(R: np.ndarray, h: np.ndarray, K: np.ndarray, N: int, a: np.ndarray) -> np.ndarray:
    """h^2-weighted sample density per bin (sums to 1)."""
    w = 2 * np.pi * K.astype(float) / N
    xi = (w[None, :, 0, None] * R[:, None, 0, :] + w[None, :, 1, None] * R[:, None, 1, :]) * N / (2 * np.pi)
    rk = np.broadcast_to(np.sqrt((K.astype(float) ** 2).sum(1))[None, :], xi.shape[:2])
    b = bin_index(xi.reshape(-1, 3), N, a, rk.reshape(-1))
    f = np.bincount(b, (h * h).reshape(-1), NBINS)
    return f / f.sum()


def target(kappa: np.ndarray, lam: float, ker0: float, a: np.ndarray) -> np.ndarray:
    """t_b = log(p_b Ker(0)), p_b the least-squares bin multiplier of 1 / (kappa + lam)."""
    N = kappa.shape[0]
    f = np.fft.fftfreq(N) * N                       # signed frequency of each FFT index
    q = np.stack(np.meshgrid(f, f, f, indexing="ij"), -1)[..., ::-1]   # kappa is [k3][k2][k1]
    b = bin_index(q.reshape(-1, 3), N, a)
    k = np.maximum(kappa.reshape(-1), 0.0) + lam
    s1 = np.bincount(b, k, NBINS)
    s2 = np.bincount(b, k * k, NBINS)
    t = np.full(NBINS, np.nan)
    ok = s2 > 0
    t[ok] = np.log(s1[ok] / s2[ok] * ker0)
    t = t.reshape(SHELLS, CONES)
    for c in range(CONES):                          # fill empty bins from the nearest shell
        col = t[:, c]
        good = np.nonzero(~np.isnan(col))[0]
        if good.size == 0:
            col[:] = np.nanmean(t)
            continue
        for s in np.nonzero(np.isnan(col))[0]:
            col[s] = col[good[np.argmin(np.abs(good - s))]]
    return t.reshape(-1)


def bin_volumes(N: int, a: np.ndarray) -> np.ndarray:
    """Fraction of the N^3 frequency grid (FFT index order) in each bin."""
    f = np.fft.fftfreq(N) * N
    q = np.stack(np.meshgrid(f, f, f, indexing="ij"), -1)
    return np.bincount(bin_index(q.reshape(-1, 3), N, a), minlength=NBINS) / float(N) ** 3


def baseline(feat: np.ndarray, vol: np.ndarray, rel_lam: float) -> np.ndarray:
    """Closed-form estimate of the target: a sampling operator's mean eigenvalue over a
    bin is about Ker(0) f_b / v_b, so t_b ~ -log(f_b / v_b + lambda / Ker(0))."""
    with np.errstate(divide="ignore", invalid="ignore"):
        dens = np.where(vol > 0, feat / np.where(vol > 0, vol, 1.0), 0.0)
    return -np.log(dens + rel_lam)


def table_diagonal(table_log: np.ndarray, N: int, ker0: float, a: np.ndarray) -> np.ndarray:
    """Fourier diagonal on the N^3 grid ([k3][k2][k1]) from a per-bin log table."""
    f = np.fft.fftfreq(N) * N
    q = np.stack(np.meshgrid(f, f, f, indexing="ij"), -1)[..., ::-1]
    b = bin_index(q.reshape(-1, 3), N, a)
    return (np.exp(table_log[b]) / ker0).reshape(N, N, N)


def net_input(feat: np.ndarray) -> np.ndarray:
    return np.log(NBINS * feat + 1e-3)


def mlp_forward(params, x):
    """params = [W1, b1, W2, b2, W3, b3] (W: out x in); x: (batch, 1024).  Returns y and
    the activations needed by the backward pass."""
    W1, b1, W2, b2, W3, b3 = params
    z1 = x @ W1.T + b1
    a1 = np.maximum(z1, 0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0)
    y = a2 @ W3.T + b3
    return y, (x, z1, a1, z2, a2)


def mlp_loss_grad(params, x, t):
    """Mean squared error over all outputs and its gradient (same layout as params)."""
    W1, b1, W2, b2, W3, b3 = params
    y, (x, z1, a1, z2, a2) = mlp_forward(params, x)
    n = y.size
    loss = float(((y - t) ** 2).sum() / n)
    gy = 2.0 * (y - t) / n
    gW3 = gy.T @ a2
    gb3 = gy.sum(0)
    ga2 = gy @ W3
    gz2 = ga2 * (z2 > 0)
    gW2 = gz2.T @ a1
    gb2 = gz2.sum(0)
    ga1 = gz2 @ W2
    gz1 = ga1 * (z1 > 0)
    gW1 = gz1.T @ x
    gb1 = gz1.sum(0)
    return loss, [gW1, gb1, gW2, gb2, gW3, gb3]


def adam_step(params, grads, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update in place (Kingma & Ba); step counts from 1."""
    for p, g, mm, vv in zip(params, grads, m, v):
        mm *= b1
        mm += (1 - b1) * g
        vv *= b2
        vv += (1 - b2) * g * g
        mh = mm / (1 - b1 ** step)
        vh = vv / (1 - b2 ** step)
        p -= lr * mh / (np.sqrt(vh) + eps)
