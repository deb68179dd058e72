"""Pins of the FP64 oracle against facts fixed outside it.

Each test names the passage of the paper it pins and the independent fact it
uses: a library routine (numpy's FFT, dense solve), a closed form, an
invariant, or a number printed in the paper (tests/golden/).
"""
import os

import numpy as np
import pytest

import oracle as O
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand_rot(M, seed):
    return synth.haar_rotations(M, seed)


def _groups():
    return synth.ctf_group_table([1.5, 2.5], pixel_A=2.8)


# -- sample set and CTF ------------------------------------------------------

def test_disc_sizes_match_row_count_fixture():
    """eq. truncation: |K| against the integer row-count fixture."""
    rows = [l.split() for l in open(os.path.join(GOLD, "disc_counts.txt")) if not l.startswith("#")]
    for N, cnt in ((int(a), int(b)) for a, b in rows):
        K = O.disc(N)
        assert K.shape[0] == cnt
        assert np.all((K ** 2).sum(1) <= (N // 2) ** 2)
        # symmetric: -k in K for every k (reading 1)
        s = {tuple(k) for k in K}
        assert all((-a, -b) in s for a, b in s)
    assert O.disc(32, disc_mode=1).shape[0] == 795


def test_wavelength_matches_paper_fig2():
    """Fig. 2 caption: lambda = 2.51 pm, the 200 kV wavelength; 300 kV gives 1.9687 pm."""
    kV, pm, tol = np.loadtxt(os.path.join(GOLD, "ctf_wavelength.txt"))
    assert abs(O.electron_wavelength_A(kV) * 100 - pm) < tol
    assert abs(O.electron_wavelength_A(300.0) * 100 - 1.9687) < 1e-3


def test_ctf_special_values():
    """CTF (Section 3.1): h(0) = -sin(A); first zero near 1/sqrt(lambda*df) (thin-lens
    Scherzer relation, corrected for A); |h| <= 1; B-factor damps."""
    g = (20000.0, 300.0, 2.0, 0.07, 2.8, 0.0)
    assert O.ctf(0.0, g) == pytest.approx(-np.sin(0.07), abs=1e-15)
    lam = O.electron_wavelength_A(300.0)
    r0 = np.sqrt((1 - 0.07 / np.pi) / (lam * 20000.0))        # Cs term negligible here
    r = np.linspace(0.5 * r0, 1.5 * r0, 20001)
    h = O.ctf(r, g)
    zero = r[np.nonzero(np.diff(np.sign(h)))[0][0]]
    assert abs(zero - r0) / r0 < 5e-3
    rr = np.linspace(0, 0.2, 1000)
    assert np.all(np.abs(O.ctf(rr, g)) <= 1 + 1e-15)
    gB = (20000.0, 300.0, 2.0, 0.07, 2.8, 100.0)
    assert O.ctf(0.1, gB) == pytest.approx(O.ctf(0.1, g) * np.exp(-100 * 0.01 / 4), rel=1e-12)


# -- forward projector against numpy's FFT (special rotations) ------------------

def _centered_fft2(img, K):
    """Centred DFT (Section 2.2) read off numpy's FFT: sum_i x_i e^{-2pi i k (i-N/2)/N} = (-1)^k fft[k]."""
    N = img.shape[-1]
    F = np.fft.fft2(img)                      # axes (-2, -1) = (k on axis0, k on axis1)
    sgn = (-1.0) ** (K[:, 0] + K[:, 1])
    return F[..., K[:, 0] % N, K[:, 1] % N] * sgn


def test_forward_identity_rotation_is_dft_of_line_sum():
    """eq. forward-projector with R = I: A(V)(k) = h * 2D DFT of sum_{n3} V (numpy fft2)."""
    N = 8
    rng = np.random.default_rng(5)
    V = rng.standard_normal((N, N, N))
    K = O.disc(N)
    R = np.eye(3)[None]
    h = rng.uniform(0.5, 1.5, (1, K.shape[0]))
    A = O.forward(V, R, h, K)[0]
    line = V.sum(axis=0)                      # [i2][i1]; k1 pairs with n1 (axis 1)
    ref = _centered_fft2(line.T, K) * h[0]    # transpose so axis0 = n1
    np.testing.assert_allclose(A, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_forward_quarter_turn_projects_along_x():
    """R with rows (0,0,1), (0,1,0), (-1,0,0): xi = (0, w2, w1), so A(V) is the DFT of the
    line sum along n1 with k1 <-> n3 and k2 <-> n2.  Using R instead of R^T flips k1."""
    N = 8
    rng = np.random.default_rng(6)
    V = rng.standard_normal((N, N, N))
    K = O.disc(N)
    R = np.array([[[0.0, 0, 1], [0, 1, 0], [-1, 0, 0]]])
    h = np.ones((1, K.shape[0]))
    A = O.forward(V, R, h, K)[0]
    line = V.sum(axis=2)                      # [n3][n2]
    ref = _centered_fft2(line, K)             # axis0 = n3 <-> k1, axis1 = n2 <-> k2
    np.testing.assert_allclose(A, ref, rtol=0, atol=1e-11 * np.abs(ref).max())
    bad = O.forward(V, R.transpose(0, 2, 1), h, K)[0]
    assert np.abs(bad - ref).max() > 1e-3 * np.abs(ref).max()


# -- adjoint, kernel, Toeplitz ----------------------------------------------------

@pytest.mark.parametrize("N,M", [(6, 5), (8, 7)])
def test_adjoint_identity(N, M):
    """Definition of A* (Section 3.2): <A V, g> = <V, A* g> for random V, g."""
    rng = np.random.default_rng(N * 100 + M)
    K = O.disc(N)
    R = _rand_rot(M, 7)
    gid = rng.integers(0, 2, M)
    h = O.ctf_weights(N, K, _groups(), gid)
    V = rng.standard_normal((N,) * 3) + 1j * rng.standard_normal((N,) * 3)
    g = rng.standard_normal((M, K.shape[0])) + 1j * rng.standard_normal((M, K.shape[0]))
    lhs = np.vdot(g, O.forward(V, R, h, K))           # <A V, g> = sum A(V) conj(g)
    rhs = np.vdot(O.adjoint(g, R, h, K, N), V)        # <V, A* g> = sum V conj(A* g)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_kernel_closed_form_at_origin_and_symmetry():
    """eq. kernel at n = 0 is sum_m sum_k h^2; Ker(-n) = conj Ker(n) (Section 3.4); under the
    symmetric disc Ker is real.  The DFT-range disc (disc_mode 1) is not real."""
    N, M = 8, 6
    rng = np.random.default_rng(1)
    K = O.disc(N)
    R = _rand_rot(M, 3)
    h = O.ctf_weights(N, K, _groups(), rng.integers(0, 2, M))
    Ker = O.kernel(R, h, K, N)
    assert Ker[N, N, N].real == pytest.approx((h * h).sum(), rel=1e-13)
    flip = Ker[:0:-1, :0:-1, :0:-1]           # n -> -n for n in (-N, N)
    np.testing.assert_allclose(Ker[1:, 1:, 1:], np.conj(flip), atol=1e-10 * abs(Ker).max())
    assert np.abs(Ker.imag).max() < 1e-10 * abs(Ker).max()
    K1 = O.disc(N, 1)
    Ker1 = O.kernel(R, O.ctf_weights(N, K1, _groups(), rng.integers(0, 2, M)), K1, N)
    assert np.abs(Ker1.imag).max() > 1e-6 * abs(Ker1).max()


def test_kernel_at_matches_full_kernel():
    """kernel_at (per-image factorisation) equals the chunked direct sum of eq. kernel."""
    N, M = 8, 9
    K = O.disc(N)
    R = _rand_rot(M, 4)
    h = O.ctf_weights(N, K, _groups(), np.arange(M) % 2)
    Ker = O.kernel(R, h, K, N)
    rng = np.random.default_rng(2)
    nv = rng.integers(-N, N, (20, 3))
    got = O.kernel_at(R, h, K, N, nv)
    ref = Ker[nv[:, 2] + N, nv[:, 1] + N, nv[:, 0] + N]
    np.testing.assert_allclose(got, ref, atol=1e-11 * abs(Ker).max())


def test_octahedral_invariance_and_axis_permutation():
    """eq. kernel: premultiplying every R_m by a quarter turn about the beam axis permutes the
    disc lattice, so Ker is unchanged; R_m P^T (P a permutation) permutes Ker's axes."""
    N, M = 8, 5
    K = O.disc(N)
    R = _rand_rot(M, 8)
    h = O.ctf_weights(N, K, _groups(), np.arange(M) % 2)
    Ker = O.kernel(R, h, K, N)
    Rz = np.array([[0.0, -1, 0], [1, 0, 0], [0, 0, 1]])
    Ker_z = O.kernel(np.einsum("ij,mjk->mik", Rz, R), h, K, N)
    np.testing.assert_allclose(Ker_z, Ker, atol=1e-10 * abs(Ker).max())
    # P maps (x, y, z) -> (y, z, x)
    P = np.array([[0.0, 1, 0], [0, 0, 1], [1, 0, 0]])
    Ker_p = O.kernel(np.einsum("mij,kj->mik", R, P), h, K, N)
    # Ker_p(n) = Ker(P^T n); P^T n = (n3, n1, n2) as (x, y, z)
    n = np.arange(-N, N)
    n1, n2, n3 = np.meshgrid(n, n, n, indexing="ij")          # axes: (x, y, z)
    ref = Ker[n2 + N, n1 + N, n3 + N]     # Ker stored [z][y][x] at (x,y,z) = (n3, n1, n2)
    got = Ker_p.transpose(2, 1, 0)        # to (x, y, z) axes
    np.testing.assert_allclose(got, ref, atol=1e-10 * abs(Ker).max())


def test_toeplitz_identity():
    """eq. toeplitz / eq. property: A*(A V) equals the convolution of Ker with V."""
    N, M = 6, 7
    rng = np.random.default_rng(9)
    K = O.disc(N)
    R = _rand_rot(M, 10)
    h = O.ctf_weights(N, K, _groups(), rng.integers(0, 2, M))
    V = rng.standard_normal((N,) * 3)
    lhs = O.adjoint(O.forward(V, R, h, K), R, h, K, N)
    rhs = O.toeplitz_direct(O.kernel(R, h, K, N), V)
    np.testing.assert_allclose(lhs, rhs, atol=1e-11 * abs(rhs).max())


def test_circulant_embedding_equals_direct_toeplitz():
    """eq. embedding_circulant with the 0-based map (reading 2): the FFT product on the 2N grid,
    cropped, equals the O(N^6) Toeplitz sum; the lag +-N plane never reaches the crop."""
    N, M = 8, 6
    rng = np.random.default_rng(11)
    K = O.disc(N)
    R = _rand_rot(M, 12)
    h = O.ctf_weights(N, K, _groups(), rng.integers(0, 2, M))
    Ker = O.kernel(R, h, K, N)
    V = rng.standard_normal((N,) * 3)
    ref = O.toeplitz_direct(Ker, V)
    got = O.toeplitz_apply(O.khat(Ker), V)
    np.testing.assert_allclose(got, ref, atol=1e-11 * abs(ref).max())
    # the lag -N planes never reach the crop: holding Ker there, or junk, changes nothing
    got_ker = O.toeplitz_apply(O.khat(Ker, lag_n_planes="ker"), V)
    np.testing.assert_allclose(got_ker, ref, atol=1e-11 * abs(ref).max())
    Ker2 = Ker.copy()
    Ker2[0], Ker2[:, 0], Ker2[:, :, 0] = 123.0, -7.0, 5.0      # the n_j = -N planes
    got2 = O.toeplitz_apply(O.khat(Ker2, lag_n_planes="ker"), V)
    np.testing.assert_allclose(got2, ref, atol=1e-11 * abs(ref).max())


def test_khat_real_and_half_spectrum():
    """Under reading 1 Ker(-n) = Ker(n) is real, so K-hat (eq. circ1) is real and K-hat(-j) =
    K-hat(j); the half spectrum j1 <= N holds all of it.  K-hat is not even per axis."""
    N, M = 8, 5
    K = O.disc(N)
    R = _rand_rot(M, 13)
    h = O.ctf_weights(N, K, _groups(), np.arange(M) % 2)
    Ker = O.kernel(R, h, K, N)
    Kh = O.khat(Ker)
    assert np.abs(Kh.imag).max() < 1e-9 * abs(Kh).max()
    j = np.arange(2 * N)
    neg = (-j) % (2 * N)
    np.testing.assert_allclose(Kh[np.ix_(neg, neg, neg)], Kh, atol=1e-9 * abs(Kh).max())
    H = O.khat_half(Ker)
    assert H.shape == (2 * N, 2 * N, N + 1)
    full = np.where((j <= N)[None, None, :], H[:, :, np.minimum(j, N)],
                    H[np.ix_(neg, neg, np.minimum(neg, N))])
    np.testing.assert_allclose(full, Kh.real, atol=1e-9 * abs(Kh).max())
    assert np.abs(Kh.real - Kh.real[:, :, neg]).max() > 1e-6 * abs(Kh).max()


# -- image DFT, shifts, analytic projections ------------------------------------------

def test_image_dft_against_numpy_and_integer_shift():
    """Step 1 / eq. measurement: the centred DFT equals numpy's fft2 read at the disc; an image
    rolled by an integer shift s and given s returns the unshifted samples (reading 4)."""
    N, M = 16, 3
    rng = np.random.default_rng(14)
    I = rng.standard_normal((M, N, N))
    K = O.disc(N)
    b = O.image_dft(I, K)
    ref = np.stack([_centered_fft2(I[m].T, K) for m in range(M)])   # axis0 = n1
    np.testing.assert_allclose(b, ref, atol=1e-11 * abs(ref).max())
    s = np.array([[2, -3], [0, 1], [-1, 0]], float)
    Is = np.stack([np.roll(I[m], (int(s[m, 1]), int(s[m, 0])), axis=(0, 1)) for m in range(M)])
    np.testing.assert_allclose(O.image_dft(Is, K, s), b, atol=1e-10 * abs(b).max())


def test_analytic_projection_matches_forward_projector():
    """Fourier slice theorem (eq. continuous_fps and its discrete form, Section 3.1): the DFT of
    the analytic projection of a band-limited blob phantom equals A(V) of the sampled phantom.
    Pins the rotation convention shared with the data generator."""
    N, M = 32, 4
    bl = synth.Blobs(np.array([[2.0, -3.0, 1.0], [-4.0, 1.0, 3.0]]), np.array([2.0, 2.2]),
                     np.array([1.0, 0.7]))
    V = synth.blob_volume(bl, N)
    R = _rand_rot(M, 15)
    img = synth.project_blobs(bl, R, N, dtype=np.float64)
    K = O.disc(N)
    b = O.image_dft(img, K)
    A = O.forward(V, R, np.ones((M, K.shape[0])), K)
    assert np.abs(b - A).max() < 1e-6 * np.abs(A).max()


def test_backprojection_of_real_images_is_real():
    """Reading 1/7: with the symmetric disc A*b of real, shifted images is real."""
    N, M = 8, 4
    rng = np.random.default_rng(16)
    I = rng.standard_normal((M, N, N))
    K = O.disc(N)
    R = _rand_rot(M, 17)
    h = O.ctf_weights(N, K, _groups(), rng.integers(0, 2, M))
    s = rng.uniform(-2, 2, (M, 2))
    full = O.adjoint(O.image_dft(I, K, s), R, h, K, N)
    assert np.abs(full.imag).max() < 1e-10 * np.abs(full.real).max()
    nv = rng.integers(-N // 2, N // 2, (6, 3))
    at = O.backproject_at(I, s, R, h, K, nv)
    np.testing.assert_allclose(at, full[nv[:, 2] + N // 2, nv[:, 1] + N // 2, nv[:, 0] + N // 2],
                               atol=1e-10 * abs(full).max())


# -- CG ------------------------------------------------------------------------------------

def test_cg_identity_operator_one_step():
    """CG (Section 3.3) on lam_eff * I (no images) converges in one iteration to rhs / lam_eff."""
    rng = np.random.default_rng(18)
    rhs = rng.standard_normal((4, 4, 4))
    x, hist, it = O.cg(lambda v: 2.5 * v, rhs, 10, rel_tol=1e-14)
    assert it == 1
    np.testing.assert_allclose(x, rhs / 2.5, rtol=1e-14)


def test_cg_matches_dense_solve_of_explicit_toeplitz_system():
    """CG (Section 3.3) on (Ker * . + lam I) equals numpy's dense solve of the explicit
    N^3 x N^3 Toeplitz matrix (eq. toep3) at N = 4."""
    N, M = 4, 6
    K = O.disc(N)
    R = _rand_rot(M, 19)
    h = O.ctf_weights(N, K, _groups(), np.arange(M) % 2)
    Ker = O.kernel(R, h, K, N).real
    lam = O.lambda_eff(1e-2, 0, Ker[N, N, N])
    n = np.stack(np.meshgrid(*(np.arange(N),) * 3, indexing="ij"), -1).reshape(-1, 3)   # (z,y,x)
    d = n[:, None, :] - n[None, :, :] + N
    T = Ker[d[..., 0], d[..., 1], d[..., 2]] + lam * np.eye(N ** 3)
    rng = np.random.default_rng(20)
    rhs = rng.standard_normal((N,) * 3)
    ref = np.linalg.solve(T, rhs.reshape(-1)).reshape((N,) * 3)
    Kh = O.khat(Ker)
    x, hist, it = O.cg(lambda v: O.toeplitz_apply(Kh, v, lam).real, rhs, 400, rel_tol=1e-13)
    np.testing.assert_allclose(x, ref, atol=1e-9 * abs(ref).max())
    # A-norm of the error decreases monotonically along the iterates (CG optimality)
    errs = []
    O.cg(lambda v: O.toeplitz_apply(Kh, v, lam).real, rhs, 30,
         callback=lambda i, xx, rr: errs.append(float((xx - ref).ravel() @ T @ (xx - ref).ravel())))
    assert all(b <= a * (1 + 1e-9) for a, b in zip(errs, errs[1:]))


def test_cg_recovers_blob_phantom_from_dense_noiseless_views():
    """FIRM steps 2-4 (Section 3.4) on noiseless data b = A(V0) from many uniform views recover V0.

    CG from zero stays in the range of A*; V0 = (A*A) V_blob lies there and is recovered to
    1e-6.  The raw blob also carries Fourier content outside the ball |xi| <= pi that A does
    not see (Section 3.3: ill-conditioning), so it is only approached slowly."""
    N, M = 8, 120
    bl = synth.phantom_blobs(3, N, 21, sigma_range=(1.0, 1.5))
    Vb = synth.blob_volume(bl, N)
    K = O.disc(N)
    R = synth.haar_rotations(M, 22)
    h = np.ones((M, K.shape[0]))
    Kh = O.khat(O.kernel(R, h, K, N))
    op = lambda v: O.toeplitz_apply(Kh, v).real
    V0 = op(Vb)
    V0 /= np.abs(V0).max()
    rhs = O.adjoint(O.forward(V0, R, h, K), R, h, K, N).real
    x, hist, it = O.cg(op, rhs, 100)
    assert np.linalg.norm(x - V0) / np.linalg.norm(V0) <= 1e-6
    rhs_b = O.adjoint(O.forward(Vb, R, h, K), R, h, K, N).real
    xb, _, _ = O.cg(op, rhs_b, 500)
    assert np.linalg.norm(xb - Vb) / np.linalg.norm(Vb) <= 5e-5


def test_wrapped_spectrum_is_khat_at_even_frequencies():
    """The 2N-point DFT of the circulant column at frequency 2k equals the N-point DFT of
    the column wrapped onto N (a DFT identity), so K-hat(2k) is the spectrum of the
    wrapped circulant used as preconditioner."""
    N, M = 8, 5
    K = O.disc(N)
    R = _rand_rot(M, 23)
    h = O.ctf_weights(N, K, _groups(), np.arange(M) % 2)
    Ker = O.kernel(R, h, K, N)
    kap = O.wrapped_spectrum(Ker, weighted=False)
    Kh = O.khat(Ker).real
    np.testing.assert_allclose(kap, Kh[::2, ::2, ::2], atol=1e-10 * abs(Kh).max())


def test_chan_circulant_is_the_frobenius_projection():
    """T. Chan's circulant is the orthogonal projection of the Toeplitz matrix (eq. toep3)
    onto circulants: its column m is the mean of T over the wrapped diagonal i - j = m
    (mod N).  Checked against the explicit N^3 x N^3 matrix at N = 4; its spectrum is
    positive for the positive semidefinite A*A."""
    N, M = 4, 6
    K = O.disc(N)
    R = _rand_rot(M, 26)
    h = O.ctf_weights(N, K, _groups(), np.arange(M) % 2)
    Ker = O.kernel(R, h, K, N).real
    n = np.stack(np.meshgrid(*(np.arange(N),) * 3, indexing="ij"), -1).reshape(-1, 3)
    d = n[:, None, :] - n[None, :, :]
    T = Ker[d[..., 0] + N, d[..., 1] + N, d[..., 2] + N]
    key = ((d % N) * np.array([N * N, N, 1])).sum(-1)
    c = np.bincount(key.ravel(), T.ravel(), N ** 3) / np.bincount(key.ravel(), None, N ** 3)
    ref = np.fft.fftn(c.reshape(N, N, N)).real
    kap = O.wrapped_spectrum(Ker)
    np.testing.assert_allclose(kap, ref, atol=1e-10 * abs(ref).max())
    assert kap.min() > -1e-10 * kap.max()


def test_preconditioned_cg_delta_kernel_one_step_and_matches_plain_cg():
    """With a delta kernel the operator is (c + lam) I and the circulant preconditioner is
    its exact inverse: one PCG step.  On a real kernel PCG and plain CG reach the same
    solution (the dense solve at N = 4)."""
    N = 4
    Ker = np.zeros((2 * N,) * 3)
    Ker[N, N, N] = 3.0
    Kh = O.khat(Ker).real
    rng = np.random.default_rng(24)
    b = rng.standard_normal((N,) * 3)
    P = O.circulant_preconditioner(O.wrapped_spectrum(Ker), 0.5)   # delta kernel: all weights 1 at n=0
    x, hist, it = O.cg(lambda v: O.toeplitz_apply(Kh, v, 0.5).real, b, 10, rel_tol=1e-12, precond=P)
    assert it == 1
    np.testing.assert_allclose(x, b / 3.5, rtol=1e-12)
    K = O.disc(N)
    R = _rand_rot(6, 25)
    h = O.ctf_weights(N, K, _groups(), np.arange(6) % 2)
    Ker = O.kernel(R, h, K, N).real
    lam = O.lambda_eff(1e-2, 0, Ker[N, N, N])
    Kh = O.khat(Ker).real
    op = lambda v: O.toeplitz_apply(Kh, v, lam).real
    n = np.stack(np.meshgrid(*(np.arange(N),) * 3, indexing="ij"), -1).reshape(-1, 3)
    d = n[:, None, :] - n[None, :, :] + N
    T = Ker[d[..., 0], d[..., 1], d[..., 2]] + lam * np.eye(N ** 3)
    ref = np.linalg.solve(T, b.reshape(-1)).reshape((N,) * 3)
    P = O.circulant_preconditioner(O.wrapped_spectrum(Ker), lam)
    x, _, it_pc = O.cg(op, b, 200, rel_tol=1e-13, precond=P)
    np.testing.assert_allclose(x, ref, atol=1e-9 * abs(ref).max())


# -- learned preconditioner (oracle/lpre.py) -------------------------------------------

from oracle import lpre as LP   # noqa: E402


def _small_params(seed):
    rng = np.random.default_rng(seed)
    sizes = LP.WIDTHS
    params = []
    for i in range(3):
        params.append(rng.standard_normal((sizes[i + 1], sizes[i])) / np.sqrt(sizes[i]))
        params.append(0.1 * rng.standard_normal(sizes[i + 1]))
    return params


def test_mlp_gradient_matches_finite_differences():
    """Backward pass of the preconditioner network against central differences of the loss."""
    params = _small_params(30)
    rng = np.random.default_rng(31)
    x = rng.standard_normal((3, LP.NBINS))
    t = rng.standard_normal((3, LP.NBINS))
    loss, grads = LP.mlp_loss_grad(params, x, t)
    eps = 1e-6
    for layer in range(6):
        p = params[layer]
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in p.shape)
            old = p[idx]
            p[idx] = old + eps
            lp, _ = LP.mlp_loss_grad(params, x, t)
            p[idx] = old - eps
            lm, _ = LP.mlp_loss_grad(params, x, t)
            p[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - grads[layer][idx]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-10


def test_adam_first_step_closed_form():
    """From zero moments the bias-corrected first Adam step is -lr * g / (|g| + eps)."""
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -4.0, 0.0])]
    m, v = [np.zeros(3)], [np.zeros(3)]
    LP.adam_step(p, g, m, v, 1, 0.01)
    np.testing.assert_allclose(p[0], [1.0 - 0.01, -2.0 + 0.01, 3.0], atol=1e-7)


def test_target_of_constant_spectrum_and_table_round_trip():
    """kappa = c everywhere: every bin's least-squares multiplier is 1 / (c + lam), so
    t_b = log(Ker(0) / (c + lam)) and the expanded diagonal is 1 / (c + lam)."""
    N, c, lam, ker0 = 8, 5.0, 0.5, 7.0
    a = np.array([0.0, 0.0, 1.0])
    t = LP.target(np.full((N, N, N), c), lam, ker0, a)
    np.testing.assert_allclose(t, np.log(ker0 / (c + lam)), rtol=1e-12)
    d = LP.table_diagonal(t, N, ker0, a)
    np.testing.assert_allclose(d, 1.0 / (c + lam), rtol=1e-12)


def test_features_sum_to_one_and_identity_rotation_lies_in_cone_zero():
    """All slices of R = I lie in the plane q3 = 0, perpendicular to the viewing axis e3:
    the density is in cone 0, and its shell profile is the h^2-weighted count of disc
    points per |k| ring (computed directly)."""
    N, M = 16, 3
    K = O.disc(N)
    R = np.repeat(np.eye(3)[None], M, 0)
    h = O.ctf_weights(N, K, _groups(), np.arange(M) % 2)
    a = LP.principal_axis(R)
    np.testing.assert_allclose(np.abs(a), [0, 0, 1], atol=1e-12)
    f = LP.features(R, h, K, N, a).reshape(LP.SHELLS, LP.CONES)
    assert abs(f.sum() - 1.0) < 1e-12
    assert np.all(f[:, 1:] == 0)
    r = np.sqrt((K ** 2).sum(1))
    shell = np.minimum(63, np.floor(64 * r / (N / 2))).astype(int)
    ref = np.zeros(64)
    np.add.at(ref, shell, (h * h).sum(0))
    np.testing.assert_allclose(f[:, 0], ref / ref.sum(), rtol=1e-12)


# -- sensitivity of the 10-iteration, lambda = 0 volume ------------------------

def test_c1_volume_sensitivity_to_rhs_perturbation():
    """Section 3.3 CG, N=32 workload (200 Haar views, lambda = 0, 10 iterations): a white
    perturbation of A*b of relative L2 size 1e-5 moves the oracle's own 10-iteration
    volume by about 2e-4 (about 21x).  This fixes how far any path whose A*b is within
    1e-5 of the exact one (a W=6, sigma=2 window is at ~5e-6) can land from the oracle
    volume, and is the basis of the W=6 volume gate of the GPU parity test."""
    inp = synth.config_inputs("C1")
    N = inp["N"]
    K = O.disc(N)
    h = np.ones((inp["M"], K.shape[0]))
    Ker = O.kernel(inp["R"], h, K, N).real
    rhs = O.backproject(inp["images"].astype(np.float64), inp["shifts"], inp["R"], h, K)
    Kh = O.khat(Ker).real
    op = lambda v: O.toeplitz_apply(Kh, v).real
    x0, _, _ = O.cg(op, rhs, 10)
    amp = []
    for seed in (0, 1):
        g = np.random.default_rng(seed).standard_normal(rhs.shape)
        g *= 1e-5 * np.linalg.norm(rhs) / np.linalg.norm(g)
        x1, _, _ = O.cg(op, rhs + g, 10)
        amp.append(np.linalg.norm(x1 - x0) / np.linalg.norm(x0) / 1e-5)
    assert 10 <= min(amp) and max(amp) <= 40, amp


def test_chunked_voxel_sums_equal_the_full_sums():
    """sums_at_voxels (per-group weights, chunks of images) equals eq. kernel and
    eq. backprojection evaluated by the full-array oracle at the same voxels, and the
    shards of an image set add up."""
    inp = synth.config_inputs("C2", M=30, N=8)
    N, M = inp["N"], inp["M"]
    K = O.disc(N)
    hg = O.ctf_weights(N, K, inp["groups"], np.arange(inp["groups"].shape[0], dtype=np.int32))
    h = O.ctf_weights(N, K, inp["groups"], inp["group_id"])
    vox = np.array([[0, 0, 0], [1, -2, 3], [-4, 3, 0], [3, 3, -4]])
    imgs = inp["images"].astype(np.float64)
    parts = [O.sums_at_voxels(inp["R"][a:b], inp["group_id"][a:b], hg, imgs[a:b], inp["shifts"][a:b], K, N, vox)
             for a, b in ((0, 11), (11, 30))]
    ker = parts[0][0] + parts[1][0]
    rhs = parts[0][1] + parts[1][1]
    Kfull = O.kernel(inp["R"], h, K, N)
    A = O.adjoint(O.image_dft(imgs, K, inp["shifts"]), inp["R"], h, K, N)
    for i, (n1, n2, n3) in enumerate(vox):
        assert abs(ker[i] - Kfull[n3 + N, n2 + N, n1 + N]) <= 1e-10 * abs(Kfull).max()
        assert abs(rhs[i] - A[n3 + N // 2, n2 + N // 2, n1 + N // 2]) <= 1e-10 * abs(A).max()
    assert abs(parts[0][2] + parts[1][2] - (h * h).sum()) <= 1e-10 * (h * h).sum()


def test_cg_trajectory_horizon_under_tiny_operator_noise():
    """Section 3.3 CG on a CTF-weighted problem (N=16, 60 views, 2 defocus groups,
    lambda = 1e-3 Ker(0)): a relative perturbation of 1e-9 of every operator apply moves
    the oracle's own FP64 iterate by < 1e-6 after 10 iterations but by > 1e-3 after 25
    (the iterate of a fixed, large iteration count is not a stable quantity; the FP32
    path's ~1e-7 rounding moves it by ~4e-2).  This fixes how many iterations a parity
    test of the iterate itself can span."""
    inp = synth.config_inputs("C2", M=60, N=16)
    rng = np.random.default_rng(100)
    sub = rng.choice(inp["groups"].shape[0], 2, replace=False)
    groups = inp["groups"][sub]
    gid = rng.integers(0, 2, 60).astype(np.int32)
    N = 16
    K = O.disc(N)
    h = O.ctf_weights(N, K, groups, gid)
    Ker = O.kernel(inp["R"], h, K, N).real
    rhs = O.backproject(inp["images"].astype(np.float64), inp["shifts"], inp["R"], h, K)
    lam = O.lambda_eff(1e-3, 0, Ker[N, N, N])
    Kh = O.khat(Ker).real
    op = lambda v: O.toeplitz_apply(Kh, v, lam).real
    noise = np.random.default_rng(9)

    def noisy(v):
        q = op(v)
        return q + 1e-9 * np.abs(q).mean() * noise.standard_normal(q.shape)

    dev = {}
    for it in (10, 25):
        xa, _, _ = O.cg(op, rhs, it)
        xb, _, _ = O.cg(noisy, rhs, it)
        dev[it] = np.linalg.norm(xb - xa) / np.linalg.norm(xa)
    assert dev[10] < 1e-6 and dev[25] > 1e-3, dev


def test_c1_fp32_fft_drift():
    """The N=32 workload's 10 CG iterations (lambda = 0) with the circulant apply done by a
    library FFT in FP32 (complex64) and FP32 CG vectors, everything else as the oracle:
    the iterate moves by ~8e-5 from the FP64 one (while white noise of the same size,
    1e-7 per apply, moves it by only ~3e-6).  This is the floor of any FP32-FFT path on
    this workload and the basis of its FP32 gates."""
    sf = pytest.importorskip("scipy.fft")
    inp = synth.config_inputs("C1")
    N = inp["N"]
    K = O.disc(N)
    h = np.ones((inp["M"], K.shape[0]))
    Ker = O.kernel(inp["R"], h, K, N).real
    rhs = O.backproject(inp["images"].astype(np.float64), inp["shifts"], inp["R"], h, K)
    Kh = O.khat(Ker).real
    Kh32 = Kh.astype(np.float32)

    def op32(v):
        P = np.zeros((2 * N,) * 3, np.complex64)
        P[:N, :N, :N] = v.astype(np.float32)
        Fv = sf.fftn(P)
        Fv *= Kh32
        return sf.ifftn(Fv)[:N, :N, :N].real.astype(np.float64)

    f32 = lambda v: v.astype(np.float32).astype(np.float64)
    x = np.zeros(rhs.shape)
    r = rhs.copy()
    p = f32(rhs)
    rr = float((r * r).sum())
    for _ in range(10):
        q = f32(op32(p))
        a = rr / float((p * q).sum())
        x = f32(x + a * p)
        r = r - a * q
        rr2 = float((r * r).sum())
        p = f32(rr2 / rr * p + r)
        rr = rr2
    xo, _, _ = O.cg(lambda v: O.toeplitz_apply(Kh, v).real, rhs, 10)
    drift = np.linalg.norm(x - xo) / np.linalg.norm(xo)
    assert 2e-5 <= drift <= 3e-4, drift


def test_bin_volumes_partition_the_grid_and_baseline_of_uniform_density():
    """Learned-preconditioner baseline: the bin volumes are the fractions of the N^3 grid
    per bin (they sum to 1 and equal a direct count), and a density proportional to the
    volumes (f = v) gives the constant table -log(1 + lambda / Ker(0))."""
    from oracle import lpre as LP
    N = 8
    a = np.array([0.3, -0.2, 0.93])
    a /= np.linalg.norm(a)
    v = LP.bin_volumes(N, a)
    assert abs(v.sum() - 1.0) < 1e-12
    cnt = np.zeros(LP.NBINS)
    for i in range(N):
        for j in range(N):
            for k in range(N):
                q = np.array([[(k + N // 2) % N - N // 2, (j + N // 2) % N - N // 2, (i + N // 2) % N - N // 2]], float)
                cnt[LP.bin_index(q, N, a)[0]] += 1
    assert np.allclose(v * N ** 3, cnt)
    b = LP.baseline(v, v, 1e-3)
    assert np.allclose(b[v > 0], -np.log(1.001))


# -- high-frequency damping (first-difference penalty) ------------------------------
def _stencil_ker(N):
    """The penalty as a convolution kernel on [-N, N)^3: 6 at lag 0, -1 at lags +-e_a."""
    K = np.zeros((2 * N,) * 3)
    K[N, N, N] = 6.0
    for a in range(3):
        for s in (-1, 1):
            idx = [N, N, N]
            idx[a] += s
            K[tuple(idx)] = -1.0
    return K


def test_gradient_penalty_is_the_first_difference_quadratic_form():
    """<V, D^T D V> = sum over the three axes of the squared first differences of V
    padded with zeros (each boundary edge to the zero exterior counted once)."""
    rng = np.random.default_rng(61)
    V = rng.standard_normal((5, 6, 7))
    q = sum(float((np.diff(np.pad(V, 1), axis=a)[tuple(slice(1, -1) if b != a else slice(None)
                                                      for b in range(3))] ** 2).sum()) for a in range(3))
    assert np.isclose(np.vdot(V, O.gradient_penalty(V)).real, q, rtol=1e-13)


def test_gradient_penalty_is_a_toeplitz_convolution_with_the_stencil():
    """D^T D V = (stencil * V) by the direct Toeplitz sum, and through the 2N circulant,
    whose spectrum is 6 - 2 sum_a cos(pi j_a / N) (the closed form the GPU adds to K-hat)."""
    N = 4
    rng = np.random.default_rng(62)
    V = rng.standard_normal((N, N, N))
    Ks = _stencil_ker(N)
    assert np.allclose(O.toeplitz_direct(Ks, V).real, O.gradient_penalty(V), atol=1e-12)
    Kh = O.khat(Ks)
    j = np.arange(2 * N)
    c = np.cos(np.pi * j / N)
    sym = 6.0 - 2.0 * (c[:, None, None] + c[None, :, None] + c[None, None, :])
    assert np.allclose(Kh.real, sym, atol=1e-12) and np.abs(Kh.imag).max() < 1e-12
    assert np.allclose(O.toeplitz_apply(Kh, V).real, O.gradient_penalty(V), atol=1e-12)


# -- positivity: projected CG (Polyak) ------------------------------------------------
def _explicit_system(N=4, lam=0.05, seed=71):
    """H = explicit matrix of (Ker * .) + lam I for a small random image set (columns by
    the direct Toeplitz sum), SPD."""
    inp = synth.config_inputs("C2", M=12, N=N)
    K = O.disc(N)
    h = O.ctf_weights(N, K, inp["groups"], inp["group_id"])
    Ker = O.kernel(inp["R"], h, K, N).real
    n = N ** 3
    H = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        H[:, j] = O.toeplitz_direct(Ker, e.reshape(N, N, N)).real.ravel()
    H = 0.5 * (H + H.T) + lam * Ker[N, N, N] * np.eye(n)
    return H


def test_projected_cg_equals_nonnegative_least_squares():
    """With H = C^T C (Cholesky), min 1/2 x^T H x - b^T x over x >= 0 is the NNLS problem
    min ||C x - C^-T b|| (scipy.optimize.nnls, Lawson-Hanson); the constraint binds."""
    from scipy.optimize import nnls
    H = _explicit_system()
    n = H.shape[0]
    rng = np.random.default_rng(72)
    b = rng.standard_normal(n) * np.abs(H).max()
    C = np.linalg.cholesky(H).T
    d = np.linalg.solve(C.T, b)
    ref, _ = nnls(C, d, maxiter=50 * n)
    x, its, ok = O.projected_cg(lambda v: (H @ v.ravel()).reshape(v.shape), b.reshape(4, 4, 4), 5000, 1e-13)
    assert ok and (ref == 0).sum() > 5                      # several bounds active
    assert np.linalg.norm(x.ravel() - ref) <= 1e-9 * np.linalg.norm(ref)
    # KKT: x >= 0, gradient >= 0 on the bound set, ~0 on the free set
    g = H @ x.ravel() - b
    assert x.min() >= 0
    assert g[x.ravel() == 0].min() >= -1e-9 * np.abs(b).max()
    assert np.abs(g[x.ravel() > 0]).max() <= 1e-9 * np.abs(b).max()


def test_projected_cg_is_cg_when_the_solution_is_positive():
    H = _explicit_system()
    n = H.shape[0]
    xt = 1.0 + np.random.default_rng(73).random(n)        # strictly positive solution
    b = H @ xt
    apply = lambda v: (H @ v.ravel()).reshape(v.shape)
    x, its, ok = O.projected_cg(apply, b.reshape(4, 4, 4), 500, 1e-12)
    assert ok and np.linalg.norm(x.ravel() - xt) <= 1e-9 * np.linalg.norm(xt)
    xc, _, _ = O.cg(apply, b.reshape(4, 4, 4), its)
    assert np.linalg.norm(x - xc) <= 1e-9 * np.linalg.norm(xc)   # no bound ever hit: the same iterates


# -- readings 1 and 2 written out on single entries -----------------------------------
def test_circulant_index_map_places_each_lag_at_its_wrapped_index():
    """Reading 2 (eq. embedding_index, read 0-based): a kernel that is 1 at one lag
    n in (-N, N)^3 and 0 elsewhere puts its 1 at index i_j = n_j mod 2N of the circulant
    column, and nowhere else; a lag with some n_j = -N (the planes i_j = N) is dropped."""
    N = 4
    for lag in [(0, 0, 0), (1, -2, 3), (-3, 3, -1), (-1, 0, 2)]:
        Ker = np.zeros((2 * N,) * 3)
        Ker[lag[0] + N, lag[1] + N, lag[2] + N] = 1.0
        C = O.circulant_column(Ker)
        assert C.sum() == 1.0
        assert C[tuple(l % (2 * N) for l in lag)] == 1.0
    Ker = np.zeros((2 * N,) * 3)
    Ker[0, N + 1, N] = 1.0                               # lag (-N, 1, 0)
    assert O.circulant_column(Ker).sum() == 0.0
    assert O.circulant_column(Ker, "ker")[N, 1, 0] == 1.0   # kept when asked, at i = N


def test_image_dft_at_plus_half_n_is_the_periodic_value():
    """Reading 1: the symmetric disc includes k_j = +N/2, whose value is the DFT's at
    -N/2 (the centred DFT of integer pixel positions is N-periodic in k); with a shift
    the phase exp(2 pi i <k, s>/N) differs between the two by exp(2 pi i N s_j / N)."""
    rng = np.random.default_rng(91)
    N = 8
    img = rng.standard_normal((2, N, N))
    K = np.array([[N // 2, 0], [-N // 2, 0], [0, N // 2], [0, -N // 2], [N // 2, N // 2 - 2]])
    b = O.image_dft(img, K)
    assert np.allclose(b[:, 0], b[:, 1]) and np.allclose(b[:, 2], b[:, 3])
    s = np.array([[0.3, -0.7], [1.25, 0.5]])
    bs = O.image_dft(img, K, s)
    assert np.allclose(bs[:, 0], b[:, 0] * np.exp(2j * np.pi * (N // 2) * s[:, 0] / N))
    assert np.allclose(bs[:, 1], b[:, 1] * np.exp(-2j * np.pi * (N // 2) * s[:, 0] / N))


# -- large-N mode: the gridding NUFFT (oracle/gridding.py, oracle/gridding.c) ----------

def test_gridded_kernel_and_adjoint_match_the_direct_sums():
    """eq. kernel, eq. backprojection: the gridding NUFFT against the direct sums (the
    definitions) at N = 8 and 16, with CTF weights, shifts and both windows.  The
    exponential-of-semicircle window at W = 12 must be at the ~1e-11 level (what makes it
    the oracle at large N), W = 8 at ~1e-7; Kaiser-Bessel at W = 6 carries the window
    error of the configurations' own NUFFT (~5e-6).  A dropped window factor, a wrong
    grid scale, sign or axis order fails all of them."""
    from oracle import gridding as Gr
    for N, M in ((8, 30), (16, 40)):
        inp = synth.config_inputs("C2", M=M, N=N)
        K = O.disc(N)
        h = O.ctf_weights(N, K, inp["groups"], inp["group_id"])
        Ker = O.kernel(inp["R"], h, K, N)
        b = O.image_dft(inp["images"].astype(float), K, inp["shifts"])
        A = O.adjoint(b, inp["R"], h, K, N)
        for W, win, tol in ((12, "es", 1e-10), (8, "es", 3e-7), (6, "kb", 2e-5)):
            Kg = Gr.kernel_gridded(inp["R"], inp["groups"], inp["group_id"], K, N, W=W, window=win)
            assert np.linalg.norm(Kg - Ker) / np.linalg.norm(Ker) < tol, (N, W, win)
            Ag = Gr.adjoint_gridded(b, inp["R"], h, K, N, W=W, window=win)
            assert np.linalg.norm(Ag - A) / np.linalg.norm(A) < tol, (N, W, win)
        Bg = Gr.backproject_gridded(inp["images"], inp["shifts"], inp["R"], inp["groups"],
                                    inp["group_id"], K, W=12)
        assert np.linalg.norm(Bg - A.real) / np.linalg.norm(A.real) < 1e-10


def test_gridded_kernel_matches_voxel_sums_at_n64():
    """eq. kernel at N = 64 (beyond the direct full-box sums): the gridding NUFFT at 200
    random lags against the oracle's one-voxel-at-a-time sums."""
    from oracle import gridding as Gr
    N, M = 64, 60
    inp = synth.config_inputs("C2", M=M, N=N)
    K = O.disc(N)
    h = O.ctf_weights(N, K, inp["groups"], inp["group_id"])
    Kg = Gr.kernel_gridded(inp["R"], inp["groups"], inp["group_id"], K, N, W=12)
    rng = np.random.default_rng(5)
    nv = rng.integers(-N, N, (200, 3))
    ref = O.kernel_at(inp["R"], h, K, N, nv)
    got = Kg[nv[:, 2] + N, nv[:, 1] + N, nv[:, 0] + N]
    assert np.max(np.abs(got - ref)) <= 1e-11 * float((h * h).sum())


def test_gridding_window_transform_and_thread_invariance():
    """The Kaiser-Bessel transform W sinh(z)/z (z = sqrt(beta^2 - (pi W nu)^2), sin past
    the cut-off) equals Gauss-Legendre quadrature of the window; the spread grid does not
    depend on the thread count (every grid value is the same sum in the same order)."""
    from oracle import gridding as Gr
    nu = np.linspace(0.0, 1.5, 301)
    for W in (6, 7, 8):
        beta = Gr.kb_beta(W)
        a = Gr.window_ft(nu, W, "kb", beta)
        q = Gr.window_ft(nu, W, "kb", beta, quadrature=True)
        assert np.max(np.abs(a - q)) <= 1e-12 * a[0]
    inp = synth.config_inputs("C2", M=20, N=16)
    K = O.disc(16)
    t1 = Gr.kernel_gridded(inp["R"], inp["groups"], inp["group_id"], K, 16, W=9, threads=1, spread_only=True)
    t3 = Gr.kernel_gridded(inp["R"], inp["groups"], inp["group_id"], K, 16, W=9, threads=3, spread_only=True)
    assert np.array_equal(t1, t3)
