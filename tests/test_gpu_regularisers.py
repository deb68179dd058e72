"""High-frequency damping (firm_set_damping): the system becomes
(A*A + mu_eff D^T D + lam_eff I) V = A*b with D the first differences on the box
(Section 5 names damping high frequencies as a Fourier-domain regulariser; the
first-difference penalty is the reading, oracle.gradient_penalty its definition).
The damped Toeplitz apply and CG are compared with the oracle's undamped apply plus
mu_eff D^T D (mu_eff = mu Ker(0), the relative reading of lambda)."""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def F():
    import __graft_entry__ as g
    g.build()
    import paper_1307_5824_gb300 as pkg
    return pkg


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _problem(N=16, M=37):
    inp = synth.config_inputs("C2", M=M, N=N)
    K = O.disc(N)
    h = O.ctf_weights(N, K, inp["groups"], inp["group_id"])
    Ker = O.kernel(inp["R"], h, K, N).real
    rhs = O.backproject(inp["images"].astype(np.float64), inp["shifts"], inp["R"], h, K)
    return inp, Ker, rhs


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("mu", [0.002, 0.02])
def test_damped_toeplitz_apply_and_cg_match_oracle(F, mu):
    N, M, W, lam = 16, 37, 7, 1e-3
    inp, Ker, rhs = _problem(N, M)
    ker0 = Ker[N, N, N]
    lam_o, mu_o = lam * ker0, mu * ker0
    Kh = O.khat(Ker).real

    def apply(v):
        return O.toeplitz_apply(Kh, v, lam_o).real + mu_o * O.gradient_penalty(v)

    rec = F.Reconstructor(N, M, groups=inp["groups"], W=W, lam=lam)
    rec.set_damping(mu)
    R, gid = _dev(inp["R"].reshape(M, 9)), _dev(inp["group_id"])
    rec.kernel(R, gid)
    rec.backproject(_dev(inp["images"]), _dev(inp["shifts"]), R, gid)
    V = np.random.default_rng(3).standard_normal((N, N, N)).astype(np.float32)
    y = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    rec.toeplitz_apply(_dev(V), y)
    torch.cuda.synchronize()
    e = rel(y.cpu().numpy(), apply(V.astype(np.float64)))
    # the damping is a visible part of the operator at this mu (a wrong or missing term fails the gate)
    share = np.linalg.norm(mu_o * O.gradient_penalty(V.astype(np.float64))) / np.linalg.norm(apply(V.astype(np.float64)))
    print(f"damped apply mu={mu}: rel err {e:.2e} (damping {share:.2f} of the result)")
    assert e <= 1e-5 and share > 1e-3           # the damping is far above the error
    x = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    st, it = rec.cg_solve(x, 10)
    assert st == 0 and it == 10
    xo, _, _ = O.cg(apply, rhs, 10)
    e = rel(x.cpu().numpy(), xo)
    print(f"damped CG mu={mu}, 10 iterations: rel err {e:.2e}")
    assert e <= 2e-4
    rec.close()


def test_damped_cg_in_fp64_mode_matches_oracle(F):
    N, M, W, lam, mu = 16, 37, 8, 1e-3, 0.005
    inp, Ker, rhs = _problem(N, M)
    ker0 = Ker[N, N, N]
    Kh = O.khat(Ker).real
    rec = F.Reconstructor(N, M, groups=inp["groups"], W=W, lam=lam, flags=F._lib.FIRM_FLAG_FP64_CG)
    rec.set_damping(mu)
    R, gid = _dev(inp["R"].reshape(M, 9)), _dev(inp["group_id"])
    rec.kernel(R, gid)
    rec.backproject(_dev(inp["images"]), _dev(inp["shifts"]), R, gid)
    x = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    st, it = rec.cg_solve(x, 25)
    assert st == 0 and it == 25
    xo, _, _ = O.cg(lambda v: O.toeplitz_apply(Kh, v, lam * ker0).real + mu * ker0 * O.gradient_penalty(v), rhs, 25)
    e = rel(x.cpu().numpy(), xo)
    print(f"damped CG, FP64 mode, 25 iterations: rel err {e:.2e}")
    assert e <= 1e-4
    rec.close()


def test_damping_off_restores_the_spectrum_and_bad_values_are_refused(F):
    N, M = 16, 37
    inp, _, _ = _problem(N, M)
    rec = F.Reconstructor(N, M, groups=inp["groups"], W=6, lam=1e-3)
    R, gid = _dev(inp["R"].reshape(M, 9)), _dev(inp["group_id"])
    kh = [torch.empty(rec.half_shape(), dtype=torch.float32, device="cuda") for _ in range(3)]
    rec.kernel(R, gid, khat_out=kh[0])
    rec.set_damping(0.01)
    rec.kernel(R, gid, khat_out=kh[1])
    rec.set_damping(0.0)
    rec.kernel(R, gid, khat_out=kh[2])
    torch.cuda.synchronize()
    k0, k1, k2 = (k.cpu().numpy().astype(np.float64) for k in kh)
    assert rel(k2, k0) <= 1e-6                      # run-to-run freedom of the FP64 grid sums only
    # the damped spectrum differs from the plain one by mu Ker(0) (6 - 2 sum cos(pi j / N))
    j = np.arange(2 * N)
    c = np.cos(np.pi * j / N)
    sym = 6.0 - 2.0 * (c[:, None, None] + c[None, :, None] + c[None, None, :N + 1])
    ker0 = rec.lambda_eff() / 1e-3
    assert rel(k1 - k0, 0.01 * ker0 * sym) <= 1e-3
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(F.FirmError):
            rec.set_damping(bad)
    rec.close()


def test_nonnegative_solve_matches_oracle_and_meets_kkt(F):
    """firm_solve_nonneg (projected CG, Polyak) against the oracle's projected CG run to a
    tight tolerance: both reach the unique minimiser of the strictly convex quadratic over
    V >= 0 (lam = 1e-2 keeps the system's condition number near 100, so FP32 residuals of
    1e-5 bound the volume's error near 1e-3).  The GPU result meets the KKT conditions
    (checked in FP64 with the oracle's operator), and the constraint binds on this data."""
    N, M, W, lam = 16, 37, 7, 1e-2
    inp, Ker, rhs = _problem(N, M)
    ker0 = Ker[N, N, N]
    Kh = O.khat(Ker).real

    def apply(v):
        return O.toeplitz_apply(Kh, v, lam * ker0).real

    xo, its_o, ok = O.projected_cg(apply, rhs, 20000, 1e-10)
    assert ok
    rec = F.Reconstructor(N, M, groups=inp["groups"], W=W, lam=lam)
    x = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    with pytest.raises(F.FirmError) as e:
        rec.solve_nonneg(x, 10, 1e-5)                   # no K-hat, no A*b yet
    assert e.value.code == F._lib.FIRM_ESTATE
    R, gid = _dev(inp["R"].reshape(M, 9)), _dev(inp["group_id"])
    rec.kernel(R, gid)
    rec.backproject(_dev(inp["images"]), _dev(inp["shifts"]), R, gid)
    st, its = rec.solve_nonneg(x, 5000, 1e-5)
    xg = x.cpu().numpy().astype(np.float64)
    e = rel(xg, xo)
    held = int((xg == 0).sum())
    print(f"non-negative solve: {its} applies (oracle {its_o}), rel err {e:.2e}, {held} voxels held at 0")
    assert st == 0 and xg.min() >= 0.0 and held > 50
    assert e <= 2e-3
    g = apply(xg) - rhs                                 # gradient of the quadratic
    scale = np.abs(rhs).max()
    assert g[xg == 0].min() >= -1e-3 * scale            # held voxels: the gradient points outward
    assert np.linalg.norm(g[xg > 0]) <= 1e-3 * np.linalg.norm(rhs)
    # host output, and refusals
    xh = np.empty((N, N, N), np.float32)
    st2, its2 = F._lib.firm_solve_nonneg(rec.plan, xh, 5000, 1e-5)
    assert st2 == 0 and rel(xh, xg) <= 1e-5
    for bad in ((-1, 1e-5), (10, -1.0), (10, float("nan"))):
        with pytest.raises(F.FirmError):
            rec.solve_nonneg(x, *bad)
    st3, its3 = rec.solve_nonneg(x, 3, 1e-5, allow=(F._lib.FIRM_ENOTCONV,))
    assert st3 == F._lib.FIRM_ENOTCONV and its3 == 3 and float(x.min()) >= 0.0
    rec.close()
