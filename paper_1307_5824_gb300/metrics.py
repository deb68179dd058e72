"""Resolution measures of a reconstruction (Section 4): the Fourier shell correlation
between two volumes, and its restriction to the frequencies inside or outside a
cone (the modified FCR the paper uses for a random conical tilt series, whose slices
miss a cone of Fourier space).  An evaluation utility on the host, outside the
reconstruction path.

FSC(i) = sum over j in Shell_i of F(V1)(j) conj(F(V2)(j)), divided by the square root
of sum |F(V1)(j)|^2 times sum |F(V2)(j)|^2, for i = 1 .. N/2 - 1 with
Shell_i = {j : 0.5 + (i - 1) + eps <= |j| < 0.5 + i + eps}, eps = 1e-4, j the
integer frequency of the 3D DFT (centred: each component in [-N/2, N/2)).  Against
the ground truth the FSC is the Fourier cross-resolution (FCR)."""
from __future__ import annotations

import numpy as np

EPS = 1e-4


def _freq(N: int) -> np.ndarray:
    return np.fft.fftfreq(N, 1.0 / N)          # integer frequencies in FFT order


def shell_index(N: int) -> np.ndarray:
    """Shell number i of every DFT frequency (FFT order [j3][j2][j1]); 0 for the
    frequencies in no shell (|j| < 0.5 + eps or |j| >= N/2 - 0.5 + eps)."""
    f = _freq(N)
    r = np.sqrt(f[:, None, None] ** 2 + f[None, :, None] ** 2 + f[None, None, :] ** 2)
    i = np.floor(r - 0.5 - EPS).astype(np.int64) + 1
    i[(r < 0.5 + EPS) | (i > N // 2 - 1)] = 0
    return i


def cone_mask(N: int, axis=(0.0, 0.0, 1.0), half_angle_deg: float = 30.0) -> np.ndarray:
    """Frequencies within half_angle_deg of the axis or of its opposite (FFT order,
    [j3][j2][j1]; axis given as (x, y, z)).  The origin is in no cone."""
    f = _freq(N)
    a = np.asarray(axis, float)
    a = a / np.linalg.norm(a)
    jx, jy, jz = f[None, None, :], f[None, :, None], f[:, None, None]
    dot = jx * a[0] + jy * a[1] + jz * a[2]
    r = np.sqrt(jx ** 2 + jy ** 2 + jz ** 2)
    with np.errstate(invalid="ignore", divide="ignore"):
        c = np.abs(dot) / r
    return (r > 0) & (c >= np.cos(np.deg2rad(half_angle_deg)))


def fsc(V1: np.ndarray, V2: np.ndarray, mask: np.ndarray | None = None) -> np.ndarray:
    """FSC(i), i = 1 .. N/2 - 1, of two N^3 volumes ([i3][i2][i1]); with mask (FFT order,
    see cone_mask) only the frequencies where it is True enter the sums.  Shells with
    no frequency (or a zero sum) give NaN."""
    N = V1.shape[0]
    F1 = np.fft.fftn(np.asarray(V1, np.float64))
    F2 = np.fft.fftn(np.asarray(V2, np.float64))
    sh = shell_index(N)
    if mask is not None:
        sh = np.where(mask, sh, 0)
    n = N // 2
    num = np.bincount(sh.ravel(), weights=(F1 * np.conj(F2)).real.ravel(), minlength=n)[1:n]
    d1 = np.bincount(sh.ravel(), weights=(np.abs(F1) ** 2).ravel(), minlength=n)[1:n]
    d2 = np.bincount(sh.ravel(), weights=(np.abs(F2) ** 2).ravel(), minlength=n)[1:n]
    with np.errstate(invalid="ignore", divide="ignore"):
        return num / np.sqrt(d1 * d2)
