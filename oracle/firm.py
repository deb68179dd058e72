"""FP64 oracle of FIRM (Wang, Shkolnisky & Singer) -- test infrastructure only.

Definitions are written out as the paper states them, by direct summation in
double precision.  A library primitive (matrix product, numpy's FFT) serves as
a step where noted; the only reformulation used is the exact factorisation of
a plane wave into per-axis factors, exp(i<n,xi>) = prod_j exp(i n_j xi_j), and
for a single image exp(i<n, R^T w>) = exp(i<R n, w>).

Readings of the paper taken here (the CUDA path takes the same ones):
  1. Disc (eq. truncation): the symmetric set {k in Z^2 : |k| <= N/2}.  Sample
     values at k_j = +N/2 are taken from the DFT by periodicity.
     disc_mode=1 keeps only -N/2 <= k_j < N/2.
  2. Circulant index map (eq. embedding_index) is read 0-based: d(i) = i for
     0 <= i < N, d(i) = i - 2N for N < i < 2N.  The planes i_j = N hold lag +-N,
     which never reaches a cropped output (|n - l| <= N - 1); they are set to
     zero, which keeps the column even so that its FFT is real.
  3. CTF (Section 3.1): h(r) = -sin(chi(r) + A) * exp(-B r^2 / 4) with
     chi = pi*lambda*df*r^2 - (pi/2)*Cs*lambda^3*r^4, r = |k| / (N * pixel) in 1/A,
     lambda the relativistic electron wavelength; no defocus groups => h = 1.
  4. Shifts: the reconstruction multiplies b_m(k) by exp(+2 pi i <k, s_m> / N).
  5. Rotations: xi_{m,k} = R_m^{-1} (w_k1, w_k2, 0) = R_m^T (w_k1, w_k2, 0), w = 2 pi k / N.
  6. Regulariser: (A*A + lam_eff I) V = A*b with lam_eff = lam * Ker(0)
     (lambda_mode 0) or lam_eff = lam (lambda_mode 1).
  7. V is real; A*b and Ker * V are real under reading 1 (their real parts are
     taken, which under disc_mode 1 restricts the unknown to real volumes).

Index conventions: a volume is an array [i3][i2][i1] with n_j = i_j - N/2;
Ker over n in [-N, N)^3 is stored [n3+N][n2+N][n1+N]; images are [m][i2][i1].
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "disc", "electron_wavelength_A", "ctf", "ctf_weights", "slice_points",
    "forward", "adjoint", "kernel", "kernel_at", "adjoint_at", "image_dft",
    "backproject", "backproject_at", "circulant_column", "khat", "khat_half",
    "toeplitz_direct", "toeplitz_apply", "gradient_penalty", "lambda_eff", "cg", "projected_cg", "wrapped_spectrum",
    "circulant_preconditioner", "sums_at_voxels",
]


# ----------------------------------------------------------------------------
# Sample set, CTF, slice geometry
# ----------------------------------------------------------------------------

def disc(N: int, disc_mode: int = 0) -> np.ndarray:
    """Integer frequencies k = (k1, k2) with |k| <= N/2 (eq. truncation, Section 3.1).

    Returned as a (|K|, 2) int array in lexicographic (k1, k2) order."""
    if N % 2:
        raise ValueError("N must be even")
    h = N // 2
    k1, k2 = np.meshgrid(np.arange(-h, h + 1), np.arange(-h, h + 1), indexing="ij")
    mask = k1 * k1 + k2 * k2 <= h * h
    if disc_mode == 1:
        mask &= (k1 < h) & (k2 < h)
    return np.stack([k1[mask], k2[mask]], axis=1).astype(np.int64)


def electron_wavelength_A(kV: float) -> float:
    """Relativistic electron wavelength in Angstrom, lambda = h / sqrt(2 m e U (1 + e U / 2 m c^2)).

    Used by the CTF of Section 3.1 (Fig. 2 caption quotes lambda = 2.51 pm)."""
    U = kV * 1e3
    h = 6.62607015e-34
    m = 9.1093837015e-31
    e = 1.602176634e-19
    c = 299792458.0
    lam_m = h / np.sqrt(2 * m * e * U * (1 + e * U / (2 * m * c * c)))
    return lam_m * 1e10


def ctf(r_invA, group) -> np.ndarray:
    """CTF of Section 3.1 (reading 3) at spatial frequency r in 1/Angstrom.

    group = (defocus_A, kV, Cs_mm, amp_contrast, pixel_A, bfactor_A2)."""
    df, kV, cs_mm, A, _pix, B = (float(v) for v in group)
    lam = electron_wavelength_A(kV)
    cs = cs_mm * 1e7
    r2 = np.asarray(r_invA, float) ** 2
    chi = np.pi * lam * df * r2 - 0.5 * np.pi * cs * lam ** 3 * r2 * r2
    return -np.sin(chi + A) * np.exp(-B * r2 / 4.0)


def ctf_weights(N: int, K: np.ndarray, groups: np.ndarray, group_id: np.ndarray) -> np.ndarray:
    """h_m(|w_k|) for every image m and sample k (eq. forward-projector).  Shape (M, |K|)."""
    M = group_id.shape[0]
    groups = np.asarray(groups, float).reshape(-1, 6)
    if groups.shape[0] == 0:
        return np.ones((M, K.shape[0]))
    kk = np.sqrt((K.astype(float) ** 2).sum(1))
    table = np.stack([ctf(kk / (N * g[4]), g) for g in groups])      # (G, |K|)
    return table[np.asarray(group_id)]


def slice_points(R: np.ndarray, N: int, K: np.ndarray) -> np.ndarray:
    """xi_{m,k} = R_m^{-1} (w_k1, w_k2, 0), w = 2 pi k / N (Section 3.1, eq. forward-projector).

    R has shape (M, 3, 3); R^{-1} = R^T, so xi = w_1 * (row 0 of R) + w_2 * (row 1 of R).
    Returns (M, |K|, 3)."""
    w = 2 * np.pi * K.astype(float) / N
    return (w[None, :, 0, None] * R[:, None, 0, :] + w[None, :, 1, None] * R[:, None, 1, :])


# ----------------------------------------------------------------------------
# Forward projector, back-projector, kernel (direct sums)
# ----------------------------------------------------------------------------

def forward(V: np.ndarray, R: np.ndarray, h: np.ndarray, K: np.ndarray) -> np.ndarray:
    """A(V)(k, m) = h_m(|w_k|) sum_n V_n exp(-i <n, xi_{m,k}>)  (eq. forward-projector).

    V is [i3][i2][i1] (real or complex), h is (M, |K|).  Returns (M, |K|) complex."""
    N = V.shape[0]
    n = np.arange(N) - N // 2
    xi = slice_points(R, N, K)
    M, P = xi.shape[:2]
    out = np.empty((M, P), complex)
    Vf = V.reshape(N * N, N).astype(complex)
    for m in range(M):
        E1 = np.exp(-1j * np.outer(xi[m, :, 0], n))          # (P, n1)
        E2 = np.exp(-1j * np.outer(xi[m, :, 1], n))          # (P, n2)
        E3 = np.exp(-1j * np.outer(xi[m, :, 2], n))          # (P, n3)
        T = (Vf @ E1.T).reshape(N, N, P)                     # sum over n1 -> [n3][n2][p]
        T = np.einsum("zyp,py->zp", T, E2)                   # sum over n2
        out[m] = np.einsum("zp,pz->p", T, E3) * h[m]         # sum over n3
    return out


def _type1(xi: np.ndarray, w: np.ndarray, lo: int, L: int, chunk: int = 2048) -> np.ndarray:
    """sum_p w_p exp(+i <n, xi_p>) for n in [lo, lo+L)^3, stored [n3][n2][n1].

    xi is (P, 3), w is (P,).  Direct sum; the per-axis factorisation of the
    plane wave turns each chunk into one matrix product."""
    n = np.arange(lo, lo + L)
    out = np.zeros((L, L * L), complex)
    for a in range(0, xi.shape[0], chunk):
        b = min(xi.shape[0], a + chunk)
        E1 = np.exp(1j * np.outer(xi[a:b, 0], n))
        E2 = np.exp(1j * np.outer(xi[a:b, 1], n))
        E3 = np.exp(1j * np.outer(xi[a:b, 2], n)) * w[a:b, None]
        B = (E2[:, :, None] * E1[:, None, :]).reshape(b - a, L * L)
        out += E3.T @ B
    return out.reshape(L, L, L)


def adjoint(g: np.ndarray, R: np.ndarray, h: np.ndarray, K: np.ndarray, N: int) -> np.ndarray:
    """(A* g)(n) = sum_m sum_k exp(+i <n, xi_{m,k}>) h_m(|w_k|) g_{k,m}  (eq. backprojection).

    g and h are (M, |K|).  Returns the complex N^3 volume [i3][i2][i1]."""
    xi = slice_points(R, N, K).reshape(-1, 3)
    return _type1(xi, (h * g).reshape(-1), -(N // 2), N)


def kernel(R: np.ndarray, h: np.ndarray, K: np.ndarray, N: int) -> np.ndarray:
    """Ker(n) = sum_m sum_k exp(+i <n, xi_{m,k}>) h_m(|w_k|)^2 for n in [-N, N)^3  (eq. kernel).

    Returns complex (2N)^3 stored [n3+N][n2+N][n1+N]."""
    xi = slice_points(R, N, K).reshape(-1, 3)
    return _type1(xi, (h * h).reshape(-1), -N, 2 * N)


def _at_voxels(R, H, K, N, nvox, chunk=512):
    """sum_m sum_k exp(+i <n_v, xi_{m,k}>) H_m(k) at a list of voxels n_v (V,3 in (n1,n2,n3)).

    Uses exp(i <n, R^T w>) = exp(i (R n)_1 w_1) exp(i (R n)_2 w_2): per image the
    sum over the disc is e_a^T H_m e_b with H_m the weights placed on the
    (N+1) x (N+1) square of k.  H is (M, |K|) (or (1,|K|) shared by all images)."""
    h = N // 2
    kr = np.arange(-h, h + 1)
    w = 2 * np.pi * kr / N
    nv = np.asarray(nvox, float)
    out = np.zeros(nv.shape[0], complex)
    ia, ib = K[:, 0] + h, K[:, 1] + h
    M = R.shape[0]
    for a in range(0, M, chunk):
        b = min(M, a + chunk)
        Rn = np.einsum("mij,vj->mvi", R[a:b, :2, :], nv)                  # (m, v, 2)
        Ea = np.exp(1j * Rn[:, :, 0:1] * w[None, None, :])                 # (m, v, k1)
        Eb = np.exp(1j * Rn[:, :, 1:2] * w[None, None, :])                 # (m, v, k2)
        Hs = np.zeros((b - a, 2 * h + 1, 2 * h + 1), complex)
        Hm = H[a:b] if H.shape[0] == M else np.broadcast_to(H, (b - a, H.shape[1]))
        Hs[:, ia, ib] = Hm
        T = np.matmul(Ea, Hs)                                              # (m, v, k2)
        out += np.einsum("mvj,mvj->v", T, Eb)
    return out


def sums_at_voxels(R, group_id, h_groups, images, shifts, K, N, nvox):
    """Ker(n) and A*b(n) (eq. kernel, eq. backprojection) at the voxels nvox, summed over
    the images given (a slice of a large set: the caller adds the slices).  The weights
    are built per chunk of images from the per-group table h_groups (G, |K|) instead of
    an (M, |K|) array.  Also returns the l1 norms of the weights, sum h^2 and sum |h b|,
    which bound the size of every output value."""
    ker = np.zeros(len(nvox), complex)
    rhs = np.zeros(len(nvox), complex)
    l1k = l1r = 0.0
    for a in range(0, R.shape[0], 1024):
        b = min(R.shape[0], a + 1024)
        h = h_groups[group_id[a:b]]
        g = image_dft(images[a:b].astype(np.float64), K, shifts[a:b]) * h
        ker += _at_voxels(R[a:b], h * h, K, N, nvox)
        rhs += _at_voxels(R[a:b], g, K, N, nvox)
        l1k += float((h * h).sum())
        l1r += float(np.abs(g).sum())
    return ker, rhs, l1k, l1r


def kernel_at(R, h, K, N, nvox):
    """Ker(n) (eq. kernel) at the voxels nvox ((V,3) array of (n1, n2, n3))."""
    return _at_voxels(R, h * h, K, N, nvox)


def adjoint_at(g, R, h, K, N, nvox):
    """(A* g)(n) (eq. backprojection) at the voxels nvox."""
    return _at_voxels(R, h * g, K, N, nvox)


# ----------------------------------------------------------------------------
# Step 1 of FIRM: image DFT, disc truncation, shifts
# ----------------------------------------------------------------------------

def image_dft(images: np.ndarray, K: np.ndarray, shifts: np.ndarray | None = None) -> np.ndarray:
    """b_m(k) = sum_n I_m(n) exp(-2 pi i <k, n> / N) * exp(+2 pi i <k, s_m> / N).

    The centred DFT of Section 2.2 restricted to the disc (eq. measurement); the
    shift factor is reading 4.  images is (M, N, N) [m][i2][i1]; n1 pairs with k1."""
    M, N, _ = images.shape
    n = np.arange(N) - N // 2
    h = N // 2
    kr = np.arange(-h, h + 1)
    F = np.exp(-2j * np.pi * np.outer(kr, n) / N)                          # (k, n)
    out = np.empty((M, K.shape[0]), complex)
    ia, ib = K[:, 0] + h, K[:, 1] + h
    for a in range(0, M, 1024):
        b = min(M, a + 1024)
        I = images[a:b].astype(float)
        # S[m, k2, k1] = sum_{n2, n1} F[k2, n2] I[m, n2, n1] F[k1, n1]
        S = np.matmul(np.matmul(F[None], I), F.T[None])
        out[a:b] = S[:, ib, ia]
        if shifts is not None:
            ph = 2 * np.pi * (np.outer(shifts[a:b, 0], K[:, 0]) + np.outer(shifts[a:b, 1], K[:, 1])) / N
            out[a:b] *= np.exp(1j * ph)
    return out


def backproject(images, shifts, R, h, K):
    """A*b of FIRM steps 1-2 (eq. measurement, eq. backprojection): real N^3 volume (reading 7)."""
    N = images.shape[1]
    return adjoint(image_dft(images, K, shifts), R, h, K, N).real


def backproject_at(images, shifts, R, h, K, nvox):
    """A*b (eq. backprojection) at the voxels nvox (complex; real under reading 1)."""
    N = images.shape[1]
    return adjoint_at(image_dft(images, K, shifts), R, h, K, N, nvox)


# ----------------------------------------------------------------------------
# Toeplitz structure, circulant embedding, CG
# ----------------------------------------------------------------------------

FFT_WORKERS = -1     # host threads of the oracle's FFTs (-1: all); 1 for single-core timings


def _fftn(a):
    """Library 3-D FFT (exponent -i): scipy.fft on FFT_WORKERS host threads when scipy is
    present (the same transform; only the 1-D batches are split across threads), numpy
    otherwise."""
    try:
        import scipy.fft as sf
    except ImportError:
        return np.fft.fftn(a)
    return sf.fftn(a, workers=FFT_WORKERS)


def _ifftn(a):
    """Inverse of _fftn (exponent +i, divided by the number of points)."""
    try:
        import scipy.fft as sf
    except ImportError:
        return np.fft.ifftn(a)
    return sf.ifftn(a, workers=FFT_WORKERS)


def circulant_column(Ker: np.ndarray, lag_n_planes: str = "zero") -> np.ndarray:
    """First column of the 2N^3 circulant C^A (eq. embedding_circulant, reading 2).

    C[i1, i2, i3] = Ker(d(i1), d(i2), d(i3)); stored with the same axis order as Ker.
    The planes with some i_j = N are zero (lag_n_planes="zero") or hold Ker at lag -N
    ("ker"); the cropped Toeplitz product is the same either way."""
    N = Ker.shape[0] // 2
    i = np.arange(2 * N)
    d = np.where(i < N, i, np.where(i == N, -N, i - 2 * N))
    idx = d + N
    C = Ker[np.ix_(idx, idx, idx)].copy()
    if lag_n_planes == "zero":
        C[N], C[:, N], C[:, :, N] = 0, 0, 0
    return C


def khat(Ker: np.ndarray, lag_n_planes: str = "zero") -> np.ndarray:
    """Eigenvalues of C^A: the 3D FFT of its first column (eq. circ1).  Complex (2N)^3."""
    return _fftn(circulant_column(Ker, lag_n_planes))


def khat_half(Ker: np.ndarray) -> np.ndarray:
    """Real part of K-hat on the half spectrum j1 in [0, N], the CUDA path's storage of K-hat.

    Under reading 1 Ker(-n) = Ker(n) is real, so K-hat is real with K-hat(-j) = K-hat(j);
    the [j3][j2][j1] block with j1 <= N (2N x 2N x (N+1)) holds every value."""
    N = Ker.shape[0] // 2
    return khat(Ker).real[:, :, : N + 1].copy()


def toeplitz_direct(Ker: np.ndarray, V: np.ndarray) -> np.ndarray:
    """(Ker * V)(n) = sum_l Ker(n - l) V_l over n, l in [-N/2, N/2)^3 (eq. toeplitz, eq. property).

    O(N^6): for tiny N only."""
    N = V.shape[0]
    out = np.zeros(V.shape, complex)
    # n - l ranges over [-(N-1), N-1]; Ker index = n - l + N.
    for l3 in range(N):
        for l2 in range(N):
            for l1 in range(N):
                v = V[l3, l2, l1]
                if v == 0:
                    continue
                # for output index i: n - l = i - j  (both shifted by N/2)
                out += v * Ker[N - l3: 2 * N - l3, N - l2: 2 * N - l2, N - l1: 2 * N - l1]
    return out


def toeplitz_apply(Khat: np.ndarray, V: np.ndarray, lam_eff: float = 0.0) -> np.ndarray:
    """(Ker * V) + lam_eff V through the 2N circulant embedding (Section 3.2):
    zero-pad V to 2N^3, multiply its FFT by K-hat, inverse FFT, keep the first N^3."""
    N = V.shape[0]
    pad = np.zeros((2 * N,) * 3, complex)
    pad[:N, :N, :N] = V
    y = _ifftn(Khat * _fftn(pad))[:N, :N, :N]
    return y + lam_eff * V


def gradient_penalty(V: np.ndarray) -> np.ndarray:
    """D^T D V for the first differences D of V on its box with zero outside: the
    gradient of ||D V||^2 / 2, a Fourier-domain damping of high frequencies (Section 5
    names damping high frequencies as a regulariser that fits FIRM; reading: the
    first-difference penalty).  Per axis a and voxel n: 2 V_n - V_{n+e_a} - V_{n-e_a},
    with V = 0 outside the box, summed over the three axes."""
    P = np.pad(np.asarray(V), 1)
    c = P[1:-1, 1:-1, 1:-1]
    out = 6.0 * c
    out = out - P[2:, 1:-1, 1:-1] - P[:-2, 1:-1, 1:-1]
    out = out - P[1:-1, 2:, 1:-1] - P[1:-1, :-2, 1:-1]
    out = out - P[1:-1, 1:-1, 2:] - P[1:-1, 1:-1, :-2]
    return out


def lambda_eff(lam: float, mode: int, ker0: float) -> float:
    """Tikhonov weight actually added to A*A (reading 6)."""
    return float(lam) * float(ker0) if mode == 0 else float(lam)


def cg(apply, rhs: np.ndarray, max_iter: int, rel_tol: float = 0.0, x0=None, precond=None,
       callback=None):
    """Conjugate gradients on apply(x) = rhs from x0 = 0 (Section 3.3, FIRM step 4).

    Textbook Hestenes--Stiefel recurrences in float64, no restarts; with
    `precond` the preconditioned form (z = P r).  Stops after max_iter
    iterations, or earlier when ||r_k|| <= rel_tol ||rhs|| (reading 8: the
    recurrence residual).  Returns (x, residual-norm history, iterations)."""
    x = np.zeros_like(rhs) if x0 is None else x0.copy()
    r = rhs - apply(x) if x0 is not None else rhs.copy()
    z = precond(r) if precond is not None else r
    p = z.copy()
    rz = float(np.vdot(r, z).real)
    bnorm = float(np.linalg.norm(rhs))
    hist = [float(np.linalg.norm(r))]
    it = 0
    while it < max_iter:
        if rel_tol > 0 and hist[-1] <= rel_tol * bnorm:
            break
        q = apply(p)
        alpha = rz / float(np.vdot(p, q).real)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        hist.append(float(np.linalg.norm(r)))
        if callback is not None:
            callback(it, x, r)
        z = precond(r) if precond is not None else r
        rz_new = float(np.vdot(r, z).real)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, np.array(hist), it


def projected_cg(apply, rhs: np.ndarray, max_iter: int, rel_tol: float = 0.0):
    """Positivity-constrained FIRM solve (Section 5 names positivity constraints as prior
    knowledge FIRM can take in; reading: the quadratic of Section 3.3,
    min 1/2 <x, H x> - <rhs, x> over x >= 0 with H = apply, SPD), by conjugate
    gradients on the free variables with projection and restarts (Polyak's method for
    bound-constrained quadratics, a published method), in float64:

      restart: free = {x > 0 or r > 0} (r = rhs - H x), p = r on free, 0 elsewhere;
      step:    q = H p, alpha = <r_f, r_f> / <p, q>; the largest feasible step is
               amax = min over p_i < 0 of x_i / -p_i;
               if amax < alpha: x += amax p, r -= amax q, the blocking variables set to
               0 (x projected onto x >= 0), restart;
               else x += alpha p, r -= alpha q; if ||r_f|| <= rel_tol ||rhs||: stop when
               no bound variable has r_i > 0, else restart; otherwise
               p = r_f + (<r_f, r_f>_new / <r_f, r_f>) p.

    Every step costs one apply; stops after max_iter applies.  Returns (x, applies,
    converged)."""
    x = np.zeros_like(rhs)
    r = rhs.copy()
    bnorm = float(np.linalg.norm(rhs))
    its = 0
    restart = True
    free = p = None
    rz = 0.0
    while True:
        if restart:
            free = (x > 0) | (r > 0)
            rf = np.where(free, r, 0.0)
            rz = float(np.vdot(rf, rf))
            if np.sqrt(rz) <= rel_tol * bnorm:
                return x, its, True
            p = rf
            restart = False
        if its >= max_iter:
            return x, its, False
        q = apply(p)
        its += 1
        alpha = rz / float(np.vdot(p, q))
        neg = p < 0
        ratio = np.full(x.shape, np.inf)
        ratio[neg] = x[neg] / -p[neg]
        amax = float(ratio.min())
        if amax < alpha:
            x = x + amax * p
            r = r - amax * q
            x[neg & (ratio <= amax)] = 0.0        # the blocking variables
            x = np.maximum(x, 0.0)
            restart = True
            continue
        x = x + alpha * p
        r = r - alpha * q
        rf = np.where(free, r, 0.0)
        rz_new = float(np.vdot(rf, rf))
        if np.sqrt(rz_new) <= rel_tol * bnorm:
            if not np.any(~free & (r > 0)):
                return x, its, True
            restart = True
            continue
        p = rf + (rz_new / rz) * p
        rz = rz_new


# ----------------------------------------------------------------------------
# Circulant preconditioner (an addition to the paper; built on the circulant
# diagonalisation of Section 2.3, eq. circ1)
# ----------------------------------------------------------------------------

def wrapped_spectrum(Ker: np.ndarray, weighted: bool = True) -> np.ndarray:
    """Eigenvalues of an N-periodic circulant built from the Toeplitz kernel (Section 2.3).

    weighted=True: T. Chan's optimal circulant (the circulant nearest to the Toeplitz
    matrix in Frobenius norm): c(m) = sum over n = m (mod N), n in (-N, N)^3, of
    Ker(n) prod_a (N - |n_a|) / N.  weighted=False: the plain wrap, whose spectrum is
    K-hat at even frequencies.  The lag -N planes are excluded (reading 2).
    Returns the real N^3 spectrum (FFT_N of c)."""
    N = Ker.shape[0] // 2
    K = Ker.real.copy()
    K[0], K[:, 0], K[:, :, 0] = 0.0, 0.0, 0.0          # lag -N planes
    if weighted:
        w = (N - np.abs(np.arange(-N, N))) / N
        K = K * w[:, None, None] * w[None, :, None] * w[None, None, :]
    c = np.zeros((N, N, N))
    # storage block a covers n in [-N + aN, aN); its index i is n + N - aN == n (mod N)
    for a in range(2):
        for b in range(2):
            for d in range(2):
                c += K[a * N:(a + 1) * N, b * N:(b + 1) * N, d * N:(d + 1) * N]
    return np.fft.fftn(c).real


def circulant_preconditioner(kappa: np.ndarray, lam_eff: float):
    """z = F^-1 diag(1 / (max(kappa, 0) + floor)) F r, floor = lam_eff (or 1e-6 kappa(0)
    when lam_eff = 0): the inverse of the circulant approximation of (A*A + lam_eff I)."""
    floor = lam_eff if lam_eff > 0 else 1e-6 * float(kappa[0, 0, 0])
    d = 1.0 / (np.maximum(kappa, 0.0) + floor)
    return lambda r: np.fft.ifftn(d * np.fft.fftn(r)).real
