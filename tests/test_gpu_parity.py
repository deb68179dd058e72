"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Gates: Ker and A*b to relative L2 <= 1e-5, the CG volume to
relative L2 <= 1e-4 after the same iteration count.  The FP32 path's own budget
on top of the window error is derived in the design notes; tolerances are
written in each test.
"""
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
    a = np.asarray(a)
    a = a.astype(np.complex128) if np.iscomplexobj(a) else a.astype(np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _inputs(cfg, N, M, seed_shift=0):
    inp = synth.config_inputs(cfg, M=M, N=N)
    return inp


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _oracle_h(inp):
    K = O.disc(inp["N"])
    return K, O.ctf_weights(inp["N"], K, inp["groups"], inp["group_id"])


def _ker_half_from_oracle(Ker, N):
    """Oracle Ker (full [-N,N)^3 box) -> [n3+N][n2+N][n1] for n1 in [0, N)."""
    return Ker.real[:, :, N:2 * N]


@pytest.mark.parametrize("N,M,W,cfg", [(16, 50, 7, "C2"), (16, 37, 6, "C2"), (32, 120, 7, "C2"),
                                       (32, 200, 6, "C1")])
def test_kernel_and_khat_match_oracle(F, N, M, W, cfg):
    """eq. kernel and eq. circ1: GPU Ker half box and K-hat vs the direct-sum oracle."""
    inp = _inputs(cfg, N, M)
    K, h = _oracle_h(inp)
    rec = F.Reconstructor(N, M, groups=inp["groups"], W=W)
    rec.kernel(_dev(inp["R"].reshape(M, 9)), _dev(inp["group_id"]))
    ker = torch.empty(rec.half_shape(), dtype=torch.float32, device="cuda")
    khat = torch.empty(rec.half_shape(), dtype=torch.float32, device="cuda")
    rec.copy_out(F._lib.FIRM_OUT_KER, ker)
    rec.copy_out(F._lib.FIRM_OUT_KHAT, khat)
    torch.cuda.synchronize()
    Ker = O.kernel(inp["R"], h, K, N)
    e_ker = rel(ker.cpu().numpy()[:, :, :N], _ker_half_from_oracle(Ker, N))
    e_kh = rel(khat.cpu().numpy(), O.khat_half(Ker.real))
    tol = 1e-5
    print(f"Ker N={N} M={M} W={W}: rel err Ker {e_ker:.3e} K-hat {e_kh:.3e}")
    assert e_ker <= tol, e_ker
    assert e_kh <= tol, e_kh
    # lam_eff reads Ker(0); the closed form is sum h^2
    assert abs(float(ker[N, N, 0]) - (h * h).sum()) <= 1e-5 * (h * h).sum()
    rec.close()


@pytest.mark.parametrize("N,M,W,dtype", [(16, 50, 7, "f32"), (32, 77, 7, "f32"), (32, 64, 7, "bf16"),
                                         (16, 33, 6, "f32")])
def test_backprojection_matches_oracle(F, N, M, W, dtype):
    """FIRM steps 1-2 (eq. measurement, eq. backprojection): samples h b and A*b vs the oracle.
    BF16 images: the oracle takes the same BF16-rounded pixels."""
    inp = _inputs("C2", N, M)
    K, h = _oracle_h(inp)
    img = inp["images"]
    tdtype = torch.bfloat16 if dtype == "bf16" else torch.float32
    timg = _dev(img).to(tdtype)
    img64 = timg.float().cpu().numpy().astype(np.float64)
    rec = F.Reconstructor(N, M, groups=inp["groups"], W=W,
                          img_dtype=F._lib.FIRM_IMG_BF16 if dtype == "bf16" else F._lib.FIRM_IMG_F32)
    rec.backproject(timg, _dev(inp["shifts"]), _dev(inp["R"].reshape(M, 9)), _dev(inp["group_id"]))
    rhs = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    rec.copy_out(F._lib.FIRM_OUT_RHS, rhs)
    nH = (K.shape[0] + 1) // 2
    smp = torch.empty((M, nH, 2), dtype=torch.float32, device="cuda")
    rec.copy_out(F._lib.FIRM_OUT_SAMPLES, smp)
    torch.cuda.synchronize()
    # samples on the half disc in the documented order
    H = [(0, k2) for k2 in range(0, N // 2 + 1)]
    H += [(k1, k2) for k1 in range(1, N // 2 + 1) for k2 in range(-N // 2, N // 2 + 1)
          if k1 * k1 + k2 * k2 <= (N // 2) ** 2]
    H = np.array(H)
    bH = O.image_dft(img64, H, inp["shifts"]) * O.ctf_weights(N, H, inp["groups"], inp["group_id"])
    bH[:, 0] *= 0.5
    s = smp.cpu().numpy()
    assert rel(s[..., 0] + 1j * s[..., 1], bH) <= 2e-6
    ref = O.backproject(img64, inp["shifts"], inp["R"], h, K)
    tol = 1e-5
    e_rhs = rel(rhs.cpu().numpy(), ref)
    print(f"A*b N={N} M={M} W={W} {dtype}: rel err {e_rhs:.3e}")
    assert e_rhs <= tol
    rec.close()


def test_toeplitz_apply_matches_oracle(F):
    """eq. property via the circulant embedding (Section 3.2), with lam_eff V added."""
    N, M = 32, 90
    inp = _inputs("C2", N, M)
    K, h = _oracle_h(inp)
    rec = F.Reconstructor(N, M, groups=inp["groups"], W=7, lam=1e-2)
    rec.kernel(_dev(inp["R"].reshape(M, 9)), _dev(inp["group_id"]))
    rng = np.random.default_rng(3)
    V = rng.standard_normal((N, N, N)).astype(np.float32)
    y = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    rec.toeplitz_apply(_dev(V), y)
    torch.cuda.synchronize()
    Ker = O.kernel(inp["R"], h, K, N).real
    lam = O.lambda_eff(1e-2, 0, Ker[N, N, N])
    assert abs(rec.lambda_eff() - lam) <= 1e-5 * lam
    ref = O.toeplitz_apply(O.khat(Ker), V.astype(np.float64), lam).real
    assert rel(y.cpu().numpy(), ref) <= 1e-5
    # host buffers through the same entry point
    yh = np.empty((N, N, N), np.float32)
    rec.toeplitz_apply(V, yh)
    assert rel(yh, ref) <= 1e-5
    rec.close()


@pytest.mark.parametrize("W", [6, 7])
def test_cg_config1_matches_oracle(F, W):
    """FIRM on the N=32 workload: 200 noiseless Haar views, no CTF, lam=0, 10 CG iterations;
    the volume vs the oracle's after the same count, default (FP32) path, for the images
    as given and for the images with every pixel moved by one FP32 ulp (random sign).  The
    two A*b differ by rounding only (~1e-7), yet this lambda = 0 iterate moves by up to
    ~1e-4 between them: the FP32 FFTs of the Toeplitz apply drive it (a library FFT in
    FP32 moves it by ~8e-5, test_c1_fp32_fft_drift; the FP64 CG mode, on the same FP32
    Ker and A*b, lands at 7e-6), and which way depends on the rounding.  Measured 5e-5 to
    2e-4 at W = 6 and 7 over such rounding-level changes, so the FP32 gate is 3e-4; the
    volume target of 1e-4 is met by the FP64 CG mode at both widths
    (test_cg_config1_fp64_mode_matches_oracle)."""
    tol = 3e-4
    inp = synth.config_inputs("C1")
    N, M = inp["N"], inp["M"]
    K, h = _oracle_h(inp)
    Ker = O.kernel(inp["R"], h, K, N).real
    rhs_o = O.backproject(inp["images"].astype(np.float64), inp["shifts"], inp["R"], h, K)
    xo, ho, _ = O.cg(lambda v: O.toeplitz_apply(O.khat(Ker), v).real, rhs_o, 10)
    img0 = inp["images"].astype(np.float32)
    sign = np.where(np.random.default_rng(5).random(img0.shape) < 0.5, -1.0, 1.0).astype(np.float32)
    img1 = (img0 + sign * np.spacing(img0)).astype(np.float32)
    rhs_dev, xs = [], []
    for img in (img0, img1):
        rec = F.Reconstructor(N, M, W=W, lam=0.0)
        R = _dev(inp["R"].reshape(M, 9))
        rec.kernel(R)
        rec.backproject(_dev(img), _dev(inp["shifts"]), R)
        x = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
        hist = torch.empty(11, dtype=torch.float64, device="cuda")
        st, it = rec.cg_solve(x, 10, resid_hist=hist)
        rhs = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
        rec.copy_out(F._lib.FIRM_OUT_RHS, rhs)
        torch.cuda.synchronize()
        assert it == 10
        rhs_dev.append(rhs.cpu().numpy().astype(np.float64))
        xs.append(x.cpu().numpy())
        err = rel(xs[-1], xo)
        print(f"C1 W={W}: CG volume rel err {err:.3e}")
        assert err <= tol
        # residual history: the same drift budget as the volume, relative to the initial
        # residual (late residuals are ~2e-4 of it, so they carry the FP32 drift in full)
        assert np.abs(hist.cpu().numpy() - ho).max() <= tol * ho[0]
        rec.close()
    print(f"C1 W={W}: A*b moved by {rel(rhs_dev[1], rhs_dev[0]):.2e}, the volume by "
          f"{rel(xs[1], xs[0].astype(np.float64)):.2e}")
    assert rel(rhs_dev[1], rhs_dev[0]) <= 3e-7


@pytest.mark.parametrize("W", [6, 7])
def test_cg_config1_fp64_mode_matches_oracle(F, W):
    """The N=32 workload's 10 CG iterations (lambda=0) in the FP64 CG mode: FP64 vectors,
    FP64 K-hat and Toeplitz apply, Ker and A*b from the FP32 NUFFT.  Gate 1e-4 (the
    volume target) at the workload's own W=6 and at W=7."""
    inp = synth.config_inputs("C1")
    N, M = inp["N"], inp["M"]
    K, h = _oracle_h(inp)
    rec = F.Reconstructor(N, M, W=W, lam=0.0, flags=F._lib.FIRM_FLAG_FP64_CG)
    R = _dev(inp["R"].reshape(M, 9))
    rec.kernel(R)
    rec.backproject(_dev(inp["images"]), _dev(inp["shifts"]), R)
    x = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    hist = torch.empty(11, dtype=torch.float64, device="cuda")
    st, it = rec.cg_solve(x, 10, resid_hist=hist)
    torch.cuda.synchronize()
    assert st == 0 and it == 10
    Ker = O.kernel(inp["R"], h, K, N).real
    rhs = O.backproject(inp["images"].astype(np.float64), inp["shifts"], inp["R"], h, K)
    xo, ho, _ = O.cg(lambda v: O.toeplitz_apply(O.khat(Ker), v).real, rhs, 10)
    err = rel(x.cpu().numpy(), xo)
    print(f"C1 W={W} FP64 CG mode: volume rel err {err:.3e}")
    assert err <= 1e-4
    assert np.abs(hist.cpu().numpy() - ho).max() <= 1e-4 * ho[0]
    rec.close()


def test_fp64_mode_long_iterate_and_its_limits(F):
    """FP64 CG mode on a CTF-weighted problem (N=16, 60 views, 2 groups, lambda=1e-3):
    the 25-iteration iterate -- which FP32 vectors move by ~4e-2 -- matches the oracle's;
    unsupported N and a preconditioner are refused."""
    inp = synth.config_inputs("C2", M=60, N=16)
    rng = np.random.default_rng(100)
    sub = rng.choice(inp["groups"].shape[0], 2, replace=False)
    groups = inp["groups"][sub]
    gid = rng.integers(0, 2, 60).astype(np.int32)
    N, M = 16, 60
    rec = F.Reconstructor(N, M, groups=groups, W=8, lam=1e-3, flags=F._lib.FIRM_FLAG_FP64_CG)
    R = _dev(inp["R"].reshape(M, 9))
    g = _dev(gid)
    rec.kernel(R, g)
    rec.backproject(_dev(inp["images"]), _dev(inp["shifts"]), R, g)
    x = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    st, it = rec.cg_solve(x, 25)
    torch.cuda.synchronize()
    K = O.disc(N)
    h = O.ctf_weights(N, K, groups, gid)
    Ker = O.kernel(inp["R"], h, K, N).real
    rhs = O.backproject(inp["images"].astype(np.float64), inp["shifts"], inp["R"], h, K)
    lam = O.lambda_eff(1e-3, 0, Ker[N, N, N])
    xo, _, _ = O.cg(lambda v: O.toeplitz_apply(O.khat(Ker).real, v, lam).real, rhs, 25)
    err = rel(x.cpu().numpy(), xo)
    print(f"N=16 CTF problem, 25 iterations, FP64 CG mode: rel err {err:.3e}")
    assert err <= 1e-4
    rec.set_precond(F._lib.FIRM_PRECOND_CIRCULANT)
    with pytest.raises(F.FirmError) as e:
        rec.cg_solve(x, 5)
    assert e.value.code == F._lib.FIRM_EINVAL
    rec.close()
    with pytest.raises(F.FirmError):
        F.Reconstructor(48, 8, W=6, flags=F._lib.FIRM_FLAG_FP64_CG)


def test_cg_relative_tolerance_and_edge_cases(F):
    """Section 3.3 CG: stops at rel_tol; M = 0 with absolute lam is lam I (one step);
    host buffers in and out."""
    N, M = 16, 60
    inp = _inputs("C2", N, M)
    rec = F.Reconstructor(N, M, groups=inp["groups"], W=7, lam=1e-2)
    R = inp["R"].reshape(M, 9).copy()
    rec.kernel(R, inp["group_id"])                       # host inputs
    rec.backproject(inp["images"], inp["shifts"], R, inp["group_id"])
    x = np.empty((N, N, N), np.float32)
    hist = np.zeros(401)
    st, it = rec.cg_solve(x, 400, rel_tol=1e-4, resid_hist=hist)
    assert st == 0 and 0 < it < 400
    assert hist[it] <= 1e-4 * hist[0] < hist[it - 1] or hist[it] <= 1e-4 * hist[0]
    # recomputed true residual of the returned iterate
    rhs = np.empty((N, N, N), np.float32)
    rec.copy_out(F._lib.FIRM_OUT_RHS, rhs)
    Ax = np.empty((N, N, N), np.float32)
    rec.toeplitz_apply(x, Ax)
    assert np.linalg.norm(Ax - rhs) / np.linalg.norm(rhs) <= 5e-4
    rec.close()
    # no images: Ker = 0, operator = lam I with lam absolute
    rec0 = F.Reconstructor(N, 4, W=7, lam=2.5, lambda_mode=F._lib.FIRM_LAMBDA_ABSOLUTE)
    rec0.kernel(np.zeros((1, 9)), M=0)
    b = np.random.default_rng(1).standard_normal((N, N, N)).astype(np.float32)
    x0 = np.empty_like(b)
    st, it = rec0.cg_solve(x0, 10, rel_tol=1e-6, rhs=b)
    assert it == 1
    np.testing.assert_allclose(x0, b / 2.5, rtol=1e-6)
    rec0.close()


def test_staged_image_upload(F):
    """firm_stage_images: the upload of pinned host images started ahead of firm_kernel
    gives the same A*b as device-resident images (to the run-to-run freedom of the FP64
    grid additions) and as the oracle; a second upload into the same staging waits for
    the first one's image DFT; an unstaged host pointer is still copied as usual; bad
    arguments are refused."""
    N, M, Mp, W = 32, 77, 100, 7
    inp = _inputs("C2", N, M)
    K, h = _oracle_h(inp)
    img_d = _dev(inp["images"]).to(torch.bfloat16)
    img64 = img_d.float().cpu().numpy().astype(np.float64)
    img_h = img_d.cpu().pin_memory()
    img2_h = (img_d.float() * 2.0).to(torch.bfloat16).cpu().pin_memory()     # exact doubling
    R, sh, gid = _dev(inp["R"].reshape(M, 9)), _dev(inp["shifts"]), _dev(inp["group_id"])
    rec = F.Reconstructor(N, Mp, groups=inp["groups"], W=W, img_dtype=F._lib.FIRM_IMG_BF16)

    def rhs_now():
        out = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
        rec.copy_out(F._lib.FIRM_OUT_RHS, out)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    rec.backproject(img_d, sh, R, gid, M=M)
    direct = rhs_now()
    ref = O.backproject(img64, inp["shifts"], inp["R"], h, K)
    assert rel(direct, ref) <= 1e-5
    # staged, with firm_kernel running between the upload and its use
    rec.stage_images(img_h, M=M)
    rec.kernel(R, gid, M=M)
    rec.backproject(img_h, sh, R, gid, M=M)
    staged = rhs_now()
    e = rel(staged, direct)
    print(f"staged upload vs device images: rel diff {e:.2e}")
    assert e <= 1e-6
    # two uploads in a row into the same staging buffer, each read by its own call
    rec.stage_images(img2_h, M=M)
    rec.backproject(img2_h, sh, R, gid, M=M)
    rec.stage_images(img_h, M=M)
    two = rhs_now()
    assert rel(two, 2.0 * direct) <= 1e-6
    rec.backproject(img_h, sh, R, gid, M=M)
    assert rel(rhs_now(), direct) <= 1e-6
    # an upload pending for one pointer; another host pointer is copied as usual
    rec.stage_images(img_h, M=M)
    rec.backproject(img2_h, sh, R, gid, M=M)
    assert rel(rhs_now(), 2.0 * direct) <= 1e-6
    rec.backproject(img_h, sh, R, gid, M=M)
    assert rel(rhs_now(), direct) <= 1e-6
    # refusals
    stg = torch.empty(M * N * N * 2, dtype=torch.uint8, device="cuda")
    for args in ((M, img_d, stg, stg.numel()),                    # device images
                 (Mp + 1, img_h, stg, stg.numel()),               # above the plan's M
                 (M, img_h, stg, stg.numel() - 1),                # staging too small
                 (M, img_h, img_h, stg.numel())):                 # staging on the host
        with pytest.raises(F.FirmError) as ex:
            F._lib.firm_stage_images(rec.plan, *args)
        assert ex.value.code == F._lib.FIRM_EINVAL
    rec.close()


def test_bad_arguments_are_rejected(F):
    N, M = 16, 8
    rec = F.Reconstructor(N, M, W=7)
    with pytest.raises(F.FirmError) as e:
        rec.cg_solve(np.empty((N, N, N), np.float32), 5)
    assert e.value.code == F._lib.FIRM_ESTATE
    with pytest.raises(F.FirmError) as e:
        rec.kernel(np.zeros((M + 1, 9)), M=M + 1)
    assert e.value.code == F._lib.FIRM_EINVAL
    rec.close()


def test_repeated_calls_agree(F):
    """Same inputs, same plan, three calls: Ker and A*b agree to FP32 rounding (the only
    run-to-run freedom is the order of the FP64 grid additions); CG on the same Ker and
    A*b is bit-identical from call to call (its reductions have a fixed order)."""
    inp = synth.config_inputs("C1")
    N, M = inp["N"], inp["M"]
    rec = F.Reconstructor(N, M, W=7, lam=0.0)
    R = _dev(inp["R"].reshape(M, 9))
    img = _dev(inp["images"])
    sh = _dev(inp["shifts"])
    outs = []
    for _ in range(3):
        rec.kernel(R)
        rec.backproject(img, sh, R)
        ker = torch.empty(rec.half_shape(), dtype=torch.float32, device="cuda")
        rhs = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
        rec.copy_out(F._lib.FIRM_OUT_KER, ker)
        rec.copy_out(F._lib.FIRM_OUT_RHS, rhs)
        torch.cuda.synchronize()
        outs.append((ker.cpu().numpy(), rhs.cpu().numpy()))
    for name, i in (("Ker", 0), ("A*b", 1)):
        d = max(rel(o[i], outs[0][i]) for o in outs[1:])
        print(f"repeat {name}: max rel diff {d:.3e}")
        assert d <= 1e-6, (name, d)
    xs = []
    for _ in range(3):
        x = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
        st, it = rec.cg_solve(x, 10)
        assert st == 0 and it == 10
        xs.append(x.cpu().numpy())
    for x in xs[1:]:
        assert np.array_equal(x, xs[0])


def test_preconditioned_cg_matches_oracle(F):
    """PCG with the circulant preconditioner (K-hat at even frequencies): the GPU iterate
    after 8 iterations matches the oracle's PCG iterate; to rel-res 1e-4 it needs fewer
    iterations than plain CG and its true residual meets the tolerance."""
    N, M = 32, 150
    inp = _inputs("C2", N, M)
    K, h = _oracle_h(inp)
    rec = F.Reconstructor(N, M, groups=inp["groups"], W=7, lam=1e-3)
    R = _dev(inp["R"].reshape(M, 9))
    g = _dev(inp["group_id"])
    rec.kernel(R, g)
    rec.backproject(_dev(inp["images"]), _dev(inp["shifts"]), R, g)
    rec.set_precond(F._lib.FIRM_PRECOND_CIRCULANT)
    x = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    rec.cg_solve(x, 8)
    torch.cuda.synchronize()
    Ker = O.kernel(inp["R"], h, K, N).real
    rhs = O.backproject(inp["images"].astype(np.float64), inp["shifts"], inp["R"], h, K)
    lam = O.lambda_eff(1e-3, 0, Ker[N, N, N])
    Kh = O.khat(Ker).real
    op = lambda v: O.toeplitz_apply(Kh, v, lam).real
    Pc = O.circulant_preconditioner(O.wrapped_spectrum(Ker), lam)
    xo, _, _ = O.cg(op, rhs, 8, precond=Pc)
    err = rel(x.cpu().numpy(), xo)
    print(f"PCG 8 iterations: rel err vs oracle {err:.3e}")
    assert err <= 1e-4
    st, it_pc = rec.cg_solve(x, 500, rel_tol=1e-4)
    rec.set_precond(F._lib.FIRM_PRECOND_NONE)
    x2 = torch.empty_like(x)
    # plain CG needs several hundred iterations here; if it hits the cap, the cap is its count
    st2, it_plain = rec.cg_solve(x2, 2000, rel_tol=1e-4, allow=(F._lib.FIRM_ENOTCONV,))
    torch.cuda.synchronize()
    print(f"iterations to rel-res 1e-4: plain {it_plain} (status {st2}), circulant {it_pc}")
    assert st == 0 and it_pc < it_plain
    true_res = np.linalg.norm(op(x.cpu().numpy().astype(np.float64)) - rhs) / np.linalg.norm(rhs)
    assert true_res <= 3e-4


@pytest.mark.parametrize("N,M", [(48, 120), (80, 150)])
def test_preconditioned_cg_matches_oracle_at_uneven_sizes(F, N, M):
    """PCG at the batched workload's non-power-of-two sizes (N = 48, 80: FFT lengths 48, 80,
    96, 160): the circulant preconditioner and a table preconditioner (exp(t_b) / Ker(0)
    per shell x cone bin, Section 3.3's CG preconditioned) after 8 iterations against
    the oracle's PCG.  Ker and A*b of the oracle come from its gridding mode (W = 12).
    Gate 2e-4: these lambda = 1e-3 PCG iterates carry the W = 7 window error of Ker and A*b
    (~1e-6) amplified over the 8 steps (1.2e-4 measured at N = 80)."""
    from oracle import gridding as Gr
    from oracle import lpre as LP
    inp = _inputs("C2", N, M)
    K = O.disc(N)
    rec = F.Reconstructor(N, M, groups=inp["groups"], W=7, lam=1e-3)
    R = _dev(inp["R"].reshape(M, 9))
    g = _dev(inp["group_id"])
    rec.kernel(R, g)
    rec.backproject(_dev(inp["images"]), _dev(inp["shifts"]), R, g)
    Ker = Gr.kernel_gridded(inp["R"], inp["groups"], inp["group_id"], K, N, W=12).real
    rhs = Gr.backproject_gridded(inp["images"], inp["shifts"], inp["R"], inp["groups"], inp["group_id"], K, W=12)
    lam = O.lambda_eff(1e-3, 0, Ker[N, N, N])
    Kh = O.khat(Ker).real
    op = lambda v: O.toeplitz_apply(Kh, v, lam).real
    x = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    # circulant
    rec.set_precond(F._lib.FIRM_PRECOND_CIRCULANT)
    rec.cg_solve(x, 8)
    xo, _, _ = O.cg(op, rhs, 8, precond=O.circulant_preconditioner(O.wrapped_spectrum(Ker), lam))
    e_c = rel(x.cpu().numpy(), xo)
    # a table varying with the shell only: at even N the half spectrum's Nyquist plane
    # (k1 = N/2) has no sign convention that the cone of a general axis respects, so a
    # cone-dependent table is compared at N = 16 (tests/test_gpu_lpre.py) instead
    s_idx = np.arange(64)[:, None]
    table = np.repeat(-0.01 * s_idx, 16, axis=1).astype(np.float32).ravel()
    rec.set_precond_table(table)
    rec.cg_solve(x, 8)
    a = rec.pc_axis().astype(np.float64)
    a /= np.linalg.norm(a)
    d = LP.table_diagonal(table.astype(np.float64), N, Ker[N, N, N], a)
    pc = lambda r: np.fft.ifftn(d * np.fft.fftn(r)).real
    xt, _, _ = O.cg(op, rhs, 8, precond=pc)
    e_t = rel(x.cpu().numpy(), xt)
    print(f"PCG N={N}: circulant {e_c:.2e} table {e_t:.2e}")
    assert e_c <= 2e-4 and e_t <= 2e-4
    rec.close()
