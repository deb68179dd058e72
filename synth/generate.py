"""Seeded generators for phantoms, poses, images, shifts and defocus groups.

Every function takes a numpy Generator or an integer seed; nothing here
depends on global random state.  See the package docstring for conventions.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def _rng(seed):
    return seed if isinstance(seed, np.random.Generator) else np.random.default_rng(seed)


@dataclass
class Blobs:
    """Isotropic 3D Gaussians: centres (B,3) in voxels (x,y,z), sigma (B,), amplitude (B,)."""
    centres: np.ndarray
    sigma: np.ndarray
    amp: np.ndarray


def phantom_blobs(n_blobs: int, N: int, seed, sigma_range=(1.5, 4.0), amp_range=(0.5, 1.0),
                  radius_frac: float = 0.6) -> Blobs:
    """Blob phantom: centres uniform in the ball of radius radius_frac*N/2 voxels."""
    rng = _rng(seed)
    d = rng.standard_normal((n_blobs, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius_frac * (N / 2) * rng.uniform(0.0, 1.0, n_blobs) ** (1.0 / 3.0)
    centres = d * r[:, None]
    sigma = rng.uniform(*sigma_range, n_blobs)
    amp = rng.uniform(*amp_range, n_blobs)
    return Blobs(centres, sigma, amp)


def blob_volume(blobs: Blobs, N: int) -> np.ndarray:
    """Sample the phantom on the voxel grid n in [-N/2, N/2)^3 -> float64 [i3][i2][i1]."""
    n = np.arange(N) - N // 2
    V = np.zeros((N, N, N))
    for c, s, a in zip(blobs.centres, blobs.sigma, blobs.amp):
        gx = np.exp(-(n - c[0]) ** 2 / (2 * s * s))
        gy = np.exp(-(n - c[1]) ** 2 / (2 * s * s))
        gz = np.exp(-(n - c[2]) ** 2 / (2 * s * s))
        V += a * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return V


def _quat_to_rot(q: np.ndarray) -> np.ndarray:
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((q.shape[0], 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def haar_rotations(M: int, seed) -> np.ndarray:
    """Haar-uniform SO(3): normalised 4D Gaussian quaternions.  Returns (M,3,3)."""
    return _quat_to_rot(_rng(seed).standard_normal((M, 4)))


def _frame_from_direction(d: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Rotations whose third row (viewing direction R^T e3) is d, with in-plane angle psi."""
    M = d.shape[0]
    a = np.where(np.abs(d[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    e1 = np.cross(a, d)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(d, e1)
    c, s = np.cos(psi)[:, None], np.sin(psi)[:, None]
    r1 = c * e1 + s * e2
    r2 = -s * e1 + c * e2
    R = np.empty((M, 3, 3))
    R[:, 0, :], R[:, 1, :], R[:, 2, :] = r1, r2, d
    return R


def _vmf_directions(M: int, kappa: float, mu: np.ndarray, rng) -> np.ndarray:
    """Von Mises--Fisher on S^2 by Wood's (1994) rejection-free sampler for p=3."""
    mu = np.asarray(mu, float)
    mu = mu / np.linalg.norm(mu)
    u = rng.uniform(0.0, 1.0, M)
    w = 1.0 + np.log(u + (1.0 - u) * np.exp(-2.0 * kappa)) / kappa
    phi = rng.uniform(0.0, 2 * np.pi, M)
    s = np.sqrt(np.maximum(0.0, 1.0 - w * w))
    local = np.stack([s * np.cos(phi), s * np.sin(phi), w], axis=1)
    ez = mu
    a = np.array([1.0, 0.0, 0.0]) if abs(mu[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    ex = np.cross(a, ez)
    ex /= np.linalg.norm(ex)
    ey = np.cross(ez, ex)
    return local[:, 0:1] * ex + local[:, 1:2] * ey + local[:, 2:3] * ez


def vmf_rotations(M: int, kappa: float, axis, seed) -> np.ndarray:
    """Viewing directions von Mises--Fisher(kappa) about `axis`, in-plane angle uniform."""
    rng = _rng(seed)
    d = _vmf_directions(M, kappa, np.asarray(axis, float), rng)
    return _frame_from_direction(d, rng.uniform(0, 2 * np.pi, M))


def cap_rotations(M: int, cap_deg: float, pole, seed) -> np.ndarray:
    """Viewing directions uniform on the spherical cap of half-angle cap_deg about `pole`."""
    rng = _rng(seed)
    pole = np.asarray(pole, float)
    pole = pole / np.linalg.norm(pole)
    cmin = np.cos(np.deg2rad(cap_deg))
    w = rng.uniform(cmin, 1.0, M)
    phi = rng.uniform(0, 2 * np.pi, M)
    s = np.sqrt(1 - w * w)
    a = np.array([1.0, 0.0, 0.0]) if abs(pole[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    ex = np.cross(a, pole)
    ex /= np.linalg.norm(ex)
    ey = np.cross(pole, ex)
    d = (s * np.cos(phi))[:, None] * ex + (s * np.sin(phi))[:, None] * ey + w[:, None] * pole
    return _frame_from_direction(d, rng.uniform(0, 2 * np.pi, M))


def rct_rotations(M: int, tilt_deg: float, seed) -> np.ndarray:
    """Random conical tilt: every viewing direction at polar angle tilt_deg from the
    z axis, azimuth uniform on [0, 2 pi), in-plane angle uniform.  The slices then miss
    the cone of half-angle 90 - tilt_deg about z in Fourier space."""
    rng = _rng(seed)
    t = np.deg2rad(tilt_deg)
    phi = rng.uniform(0, 2 * np.pi, M)
    d = np.stack([np.sin(t) * np.cos(phi), np.sin(t) * np.sin(phi), np.full(M, np.cos(t))], axis=1)
    return _frame_from_direction(d, rng.uniform(0, 2 * np.pi, M))


def mixed_rotations(M: int, seed, frac_vmf=0.7, kappa=20.0, n_axes=3) -> np.ndarray:
    """frac_vmf of the views vMF(kappa) about n_axes random axes, the rest Haar."""
    rng = _rng(seed)
    n_v = int(round(frac_vmf * M))
    axes = rng.standard_normal((n_axes, 3))
    which = rng.integers(0, n_axes, n_v)
    R = np.empty((M, 3, 3))
    for a in range(n_axes):
        sel = np.nonzero(which == a)[0]
        if sel.size:
            R[sel] = vmf_rotations(sel.size, kappa, axes[a], rng)
    R[n_v:] = haar_rotations(M - n_v, rng)
    return R[rng.permutation(M)]


def uniform_shifts(M: int, seed, max_px: float = 2.0) -> np.ndarray:
    """Per-image in-plane shifts (x, y) in pixels, uniform in [-max_px, max_px]^2."""
    return _rng(seed).uniform(-max_px, max_px, (M, 2))


def project_blobs(blobs: Blobs, R: np.ndarray, N: int, shifts: np.ndarray | None = None,
                  dtype=np.float32, chunk: int = 2048) -> np.ndarray:
    """Analytic line integrals along x3 of the rotated phantom, sampled at pixel centres.

    A blob (c, sigma, a) projects to a * sigma * sqrt(2 pi) * exp(-|x - p|^2 / (2 sigma^2))
    with p = (R c)_{1,2} + s.  Returns (M, N, N) [m][i2][i1]."""
    M = R.shape[0]
    x = np.arange(N) - N // 2
    out = np.empty((M, N, N), dtype)
    s2 = 2.0 * blobs.sigma ** 2
    pref = blobs.amp * blobs.sigma * np.sqrt(2 * np.pi)
    for a in range(0, M, chunk):
        b = min(M, a + chunk)
        P = np.einsum('mij,cj->mci', R[a:b, :2, :], blobs.centres)        # (m, blob, 2)
        if shifts is not None:
            P = P + shifts[a:b, None, :]
        gx = np.exp(-(x[None, None, :] - P[:, :, 0:1]) ** 2 / s2[None, :, None])   # (m, blob, x)
        gy = np.exp(-(x[None, None, :] - P[:, :, 1:2]) ** 2 / s2[None, :, None])   # (m, blob, y)
        gy *= pref[None, :, None]
        out[a:b] = np.matmul(gy.transpose(0, 2, 1), gx)                   # (m, y, x)
    return out


def add_noise(images: np.ndarray, snr: float, seed) -> tuple[np.ndarray, float]:
    """White Gaussian noise with variance var(clean images) / snr.  Returns (noisy, sigma)."""
    if snr is None or snr <= 0 or np.isinf(snr):
        return images, 0.0
    rng = _rng(seed)
    sigma = float(np.sqrt(np.var(images, dtype=np.float64) / snr))
    noisy = np.empty_like(images)
    for a in range(0, images.shape[0], 4096):
        b = min(images.shape[0], a + 4096)
        noisy[a:b] = images[a:b] + sigma * rng.standard_normal(images[a:b].shape, dtype=np.float32)
    return noisy, sigma


def ctf_group_table(defocus_um, kV=300.0, Cs_mm=2.0, amp_contrast=0.07, pixel_A=2.8,
                    bfactor_A2=0.0) -> np.ndarray:
    """Defocus-group parameters as an (G, 6) float64 table, one row per group:
    (defocus in Angstrom, kV, Cs in mm, amplitude contrast, pixel size in Angstrom, B-factor)."""
    d = np.atleast_1d(np.asarray(defocus_um, float))
    t = np.empty((d.size, 6))
    t[:, 0] = d * 1e4
    t[:, 1], t[:, 2], t[:, 3], t[:, 4], t[:, 5] = kV, Cs_mm, amp_contrast, pixel_A, bfactor_A2
    return t


# The five workloads.  Counts, sizes and distributions follow the configuration
# list of the build; the seeds make each one reproducible.
CONFIGS = {
    "C1": dict(N=32, M=200, n_blobs=10, views="haar", shift_px=0.0, defocus_um=None,
               snr=None, lam=0.0, iters=10, rel_tol=0.0, seeds=(1, 2, 3)),
    "C2": dict(N=64, M=5000, n_blobs=30, views="mixed", shift_px=2.0,
               defocus_um=[1.5, 2.0, 2.5, 3.0], snr=0.1, lam=1e-3, iters=30, rel_tol=0.0,
               seeds=(11, 12, 13)),
    "C3": dict(N=128, M=50000, n_blobs=60, views="haar", shift_px=2.0,
               defocus_um=list(np.linspace(1.0, 3.5, 20)), snr=0.05, lam=1e-3, iters=2000,
               rel_tol=1e-4, seeds=(21, 22, 23)),
    "C5": dict(N=128, M=40000, n_blobs=60, views="cap", shift_px=2.0,
               defocus_um=list(np.linspace(1.0, 3.5, 8)), snr=0.1, lam=1e-3, iters=2000,
               rel_tol=1e-4, seeds=(41, 42, 43)),
    # random conical tilt series (tilt 60 deg, azimuth uniform), SNR 1, shaped like the
    # paper's simulation (90^3 volume, 10,000 images; N = 96 is the nearest supported
    # size); no CTF in the images (the generator holds none), so none in the solve
    "RCT": dict(N=96, M=10000, n_blobs=40, views="rct", shift_px=2.0, defocus_um=None,
                snr=1.0, lam=1e-3, iters=2000, rel_tol=1e-4, seeds=(51, 52, 53), tilt_deg=60.0),
}


def config_inputs(name: str, M: int | None = None, N: int | None = None, images: bool = True,
                  image_dtype=np.float32) -> dict:
    """Build one workload: poses (M,3,3) float64, shifts (M,2), group ids (M,) int32,
    defocus-group table (G,6) (G may be 0: no CTF), images (M,N,N) and the phantom."""
    cfg = dict(CONFIGS[name])
    if M is not None:
        cfg["M"] = M
    if N is not None:
        cfg["N"] = N
    N, M = cfg["N"], cfg["M"]
    s_ph, s_pose, s_noise = cfg["seeds"]
    blobs = phantom_blobs(cfg["n_blobs"], N, s_ph)
    rng = np.random.default_rng(s_pose)
    if cfg["views"] == "haar":
        R = haar_rotations(M, rng)
    elif cfg["views"] == "mixed":
        R = mixed_rotations(M, rng)
    elif cfg["views"] == "rct":
        R = rct_rotations(M, cfg["tilt_deg"], rng)
    elif cfg["views"] == "cap":
        n_cap = int(round(0.85 * M))
        R = np.concatenate([cap_rotations(n_cap, 15.0, [0, 0, 1], rng),
                            haar_rotations(M - n_cap, rng)])
        R = R[rng.permutation(M)]
    else:
        raise ValueError(cfg["views"])
    shifts = uniform_shifts(M, rng, cfg["shift_px"]) if cfg["shift_px"] > 0 else np.zeros((M, 2))
    if cfg["defocus_um"] is None:
        groups = np.zeros((0, 6))
        gid = np.zeros(M, np.int32)
    else:
        groups = ctf_group_table(cfg["defocus_um"])
        gid = rng.integers(0, groups.shape[0], M).astype(np.int32)
    out = dict(cfg=cfg, N=N, M=M, R=R, shifts=shifts, groups=groups, group_id=gid, blobs=blobs)
    if images:
        clean = project_blobs(blobs, R, N, shifts, dtype=np.float32)
        noisy, sigma = add_noise(clean, cfg["snr"], s_noise)
        out["images"] = noisy.astype(image_dtype, copy=False)
        out["noise_sigma"] = sigma
    return out


# The batched workload: 64 independent reconstructions of uneven size.
BATCH = dict(n=64, N_choices=(48, 64, 80, 96), M_range=(1000, 8000), n_blobs=30, shift_px=2.0,
             defocus_um=(1.5, 2.0, 2.5, 3.0), snr=0.1, lam=1e-3, iters=25, seed0=31)


def batch_inputs(j: int, images: bool = True, image_dtype=np.float32) -> dict:
    """Problem j of the batched workload: N uniform over {48, 64, 80, 96}, M uniform in
    [1000, 8000], its own 30-blob phantom, views as the N=64 workload (70% von
    Mises-Fisher about 3 axes, 30% Haar), shifts U[-2, 2] px, 1-4 of the 4 defocus
    groups, SNR 0.1.  Seeds 31 + j."""
    rng = np.random.default_rng(BATCH["seed0"] + j)
    N = int(rng.choice(BATCH["N_choices"]))
    M = int(rng.integers(BATCH["M_range"][0], BATCH["M_range"][1] + 1))
    blobs = phantom_blobs(BATCH["n_blobs"], N, rng)
    R = mixed_rotations(M, rng)
    shifts = uniform_shifts(M, rng, BATCH["shift_px"])
    ng = int(rng.integers(1, 5))
    dfs = sorted(rng.choice(BATCH["defocus_um"], ng, replace=False))
    groups = ctf_group_table(dfs)
    gid = rng.integers(0, ng, M).astype(np.int32)
    out = dict(N=N, M=M, R=R, shifts=shifts, groups=groups, group_id=gid, blobs=blobs)
    if images:
        clean = project_blobs(blobs, R, N, shifts, dtype=np.float32)
        noisy, sigma = add_noise(clean, BATCH["snr"], rng)
        out["images"] = noisy.astype(image_dtype, copy=False)
        out["noise_sigma"] = sigma
    return out
