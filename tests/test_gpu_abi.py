"""The C ABI's behaviour on the device: stream order, CG breakdown, the fused channels.

* firm_kernel and firm_backproject with device inputs queue their work on the plan's
  stream and return before the device has finished it (an event recorded right after
  them is still pending); the results equal those of a synchronised run.
* CG breakdown (Section 3.3's recurrences need <p, A p> > 0 and finite scalars) is
  reported as FIRM_EBREAKDOWN, made on the host: a right-hand side holding a NaN, and a
  zero operator (no images, lambda = 0 absolute).
* firm_kernel_backproject (both spreading channels of Section 3.4 steps 2-3 in one pass
  on the 4N grid) against the direct-sum oracle (eq. kernel, eq. backprojection, eq.
  circ1) and against the separate calls, with device, staged and host images.
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


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_kernel_and_backproject_return_before_the_device_finishes(F):
    inp = synth.config_inputs("C2", M=20000, N=128)
    N, M = inp["N"], inp["M"]
    rec = F.Reconstructor(N, M, groups=inp["groups"], W=6, lam=1e-3)
    R, g = _dev(inp["R"].reshape(M, 9)), _dev(inp["group_id"])
    img, sh = _dev(inp["images"]), _dev(inp["shifts"])
    khat = torch.empty(rec.half_shape(), dtype=torch.float32, device="cuda")
    rhs = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    rec.kernel(R, g, khat_out=khat)
    rec.backproject(img, sh, R, g, rhs_out=rhs)
    torch.cuda.synchronize()
    k1, r1 = khat.clone(), rhs.clone()
    khat.zero_()
    rhs.zero_()
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    rec.kernel(R, g, khat_out=khat)
    rec.backproject(img, sh, R, g, rhs_out=rhs)
    ev = torch.cuda.Event()
    ev.record(stream)
    pending = not ev.query()
    torch.cuda.synchronize()
    assert pending, "firm_kernel + firm_backproject waited for the device"
    # the FP64 atomics into the fine grid add in a different order run to run
    assert _rel(khat.cpu().numpy(), k1.double().cpu().numpy()) <= 1e-6
    assert _rel(rhs.cpu().numpy(), r1.double().cpu().numpy()) <= 1e-6
    # the device scalars are read only by a query
    assert rec.lambda_eff() > 0.0
    rec.close()


def test_cg_breakdown_is_reported(F):
    L = F._lib
    N, M = 16, 30
    inp = synth.config_inputs("C2", M=M, N=N)
    rec = F.Reconstructor(N, M, groups=inp["groups"], W=6, lam=1e-3)
    R, g = _dev(inp["R"].reshape(M, 9)), _dev(inp["group_id"])
    rec.kernel(R, g)
    rec.backproject(_dev(inp["images"]), _dev(inp["shifts"]), R, g)
    b = np.random.default_rng(1).standard_normal((N, N, N)).astype(np.float32)
    b[3, 4, 5] = np.nan
    x = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    st, it = rec.cg_solve(x, 10, rhs=_dev(b), allow=(L.FIRM_EBREAKDOWN,))
    assert st == L.FIRM_EBREAKDOWN and it == 0
    # the plan stays usable: a finite right-hand side solves
    st, it = rec.cg_solve(x, 5)
    assert st == L.FIRM_OK and it == 5
    rec.close()
    # zero operator: no images and lambda = 0 (absolute) give <p, A p> = 0
    rec = F.Reconstructor(N, M, W=6, lam=0.0, lambda_mode=L.FIRM_LAMBDA_ABSOLUTE)
    rec.kernel(R, g, M=0)
    b = np.ones((N, N, N), np.float32)
    st, it = rec.cg_solve(x, 10, rhs=_dev(b), allow=(L.FIRM_EBREAKDOWN,))
    assert st == L.FIRM_EBREAKDOWN and it == 0
    rec.close()


@pytest.mark.parametrize("N,M,W", [(16, 40, 6), (16, 33, 7), (32, 90, 6)])
def test_fused_channels_match_oracle_and_separate_calls(F, N, M, W):
    L = F._lib
    inp = synth.config_inputs("C2", M=M, N=N)
    K = O.disc(N)
    h = O.ctf_weights(N, K, inp["groups"], inp["group_id"])
    Ker = O.kernel(inp["R"], h, K, N).real
    rhs_o = O.backproject(inp["images"].astype(np.float64), inp["shifts"], inp["R"], h, K)
    R, g, sh = _dev(inp["R"].reshape(M, 9)), _dev(inp["group_id"]), _dev(inp["shifts"])
    img = _dev(inp["images"])
    rec = F.Reconstructor(N, M, groups=inp["groups"], W=W, lam=1e-3, fused=True)
    khat = torch.empty(rec.half_shape(), dtype=torch.float32, device="cuda")
    rhs = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    ker = torch.empty(rec.half_shape(), dtype=torch.float32, device="cuda")
    rec.kernel_backproject(img, sh, R, g, khat_out=khat, rhs_out=rhs)
    rec.copy_out(L.FIRM_OUT_KER, ker)
    torch.cuda.synchronize()
    e_ker = _rel(ker.cpu().numpy()[:, :, :N], Ker[:, :, N:])
    e_kh = _rel(khat.cpu().numpy(), O.khat_half(Ker))
    e_rhs = _rel(rhs.cpu().numpy(), rhs_o)
    lam_o = O.lambda_eff(1e-3, 0, Ker[N, N, N])
    print(f"fused N={N} M={M} W={W}: Ker {e_ker:.2e} K-hat {e_kh:.2e} A*b {e_rhs:.2e}")
    assert e_ker <= 1e-5 and e_kh <= 1e-5 and e_rhs <= 1e-5
    assert abs(rec.lambda_eff() - lam_o) <= 1e-5 * lam_o
    # the same plan's separate calls give the same Ker up to the fixed-point rounding (the
    # fused pass keeps one more bit), A*b up to the window error of oversampling 2 against 4
    k_sep = torch.empty_like(khat)
    r_sep = torch.empty_like(rhs)
    rec.kernel(R, g, khat_out=k_sep)
    rec.backproject(img, sh, R, g, rhs_out=r_sep)
    torch.cuda.synchronize()
    assert _rel(k_sep.cpu().numpy(), khat.double().cpu().numpy()) <= 5e-6
    assert _rel(r_sep.cpu().numpy(), rhs.double().cpu().numpy()) <= 2e-5
    # CG runs on the fused results
    rec.kernel_backproject(img, sh, R, g)
    x = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    st, it = rec.cg_solve(x, 6)
    assert st == L.FIRM_OK and it == 6
    xo, _, _ = O.cg(lambda v: O.toeplitz_apply(O.khat(Ker), v, lam_o).real, rhs_o, 6)
    assert _rel(x.cpu().numpy(), xo) <= 1e-4
    # host images (copied, then transformed before the binning) and staged images
    rh = np.empty((N, N, N), np.float32)
    rec.kernel_backproject(np.ascontiguousarray(inp["images"]), sh, R, g, rhs_out=rh)
    assert _rel(rh, rhs.double().cpu().numpy()) <= 1e-6
    pinned = torch.from_numpy(np.ascontiguousarray(inp["images"])).pin_memory()
    rec.stage_images(pinned)
    rec.kernel_backproject(pinned, sh, R, g, rhs_out=rhs)
    torch.cuda.synchronize()
    assert _rel(rhs.cpu().numpy(), rh.astype(np.float64)) <= 1e-6
    rec.close()
    # a plan made without the flag refuses the call
    rec = F.Reconstructor(N, M, groups=inp["groups"], W=W, lam=1e-3)
    with pytest.raises(L.FirmError) as e:
        rec.kernel_backproject(img, sh, R, g)
    assert e.value.code == L.FIRM_EINVAL
    rec.close()


def test_image_shards_loaded_into_a_plan_match_the_whole_set(F):
    """Two image shards spread by two plans (two processes' share of the images, run one
    after the other on this one GPU), their Ker half boxes and A*b added, loaded into a
    third plan with firm_load_sums: K-hat, lam_eff, A*b and the CG volume equal those of
    one plan over all the images (Ker and A*b are sums over the images, Section 3.4)."""
    L = F._lib
    N, M = 32, 160
    inp = synth.config_inputs("C2", M=M, N=N)
    R, g, sh, img = (_dev(inp["R"].reshape(M, 9)), _dev(inp["group_id"]), _dev(inp["shifts"]),
                     _dev(inp["images"]))
    whole = F.Reconstructor(N, M, groups=inp["groups"], W=6, lam=1e-3)
    kh_w = torch.empty(whole.half_shape(), dtype=torch.float32, device="cuda")
    rhs_w = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    whole.kernel(R, g, khat_out=kh_w)
    whole.backproject(img, sh, R, g, rhs_out=rhs_w)
    ker_sum = torch.zeros(whole.half_shape(), dtype=torch.float32, device="cuda")
    rhs_sum = torch.zeros((N, N, N), dtype=torch.float32, device="cuda")
    for a, b in ((0, 70), (70, M)):
        part = F.Reconstructor(N, b - a, groups=inp["groups"], W=6, lam=1e-3, fused=(a == 0))
        k = torch.empty_like(ker_sum)
        r = torch.empty_like(rhs_sum)
        if a == 0:
            part.kernel_backproject(img[a:b], sh[a:b], R[a:b], g[a:b])
        else:
            part.kernel(R[a:b], g[a:b])
            part.backproject(img[a:b], sh[a:b], R[a:b], g[a:b])
        part.copy_out(L.FIRM_OUT_KER, k)
        part.copy_out(L.FIRM_OUT_RHS, r)
        torch.cuda.synchronize()
        ker_sum += k
        rhs_sum += r
        part.close()
    loaded = F.Reconstructor(N, M, groups=inp["groups"], W=6, lam=1e-3)
    kh_l = torch.empty_like(kh_w)
    loaded.load_sums(ker_sum, rhs_sum)
    loaded.copy_out(L.FIRM_OUT_KHAT, kh_l)
    torch.cuda.synchronize()
    assert _rel(kh_l.cpu().numpy(), kh_w.double().cpu().numpy()) <= 5e-6
    assert abs(loaded.lambda_eff() - whole.lambda_eff()) <= 5e-6 * whole.lambda_eff()
    x_w = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    x_l = torch.empty_like(x_w)
    whole.cg_solve(x_w, 8)
    loaded.cg_solve(x_l, 8)
    assert _rel(x_l.cpu().numpy(), x_w.double().cpu().numpy()) <= 1e-4
    with pytest.raises(L.FirmError) as e:
        loaded.load_sums(None, None)
    assert e.value.code == L.FIRM_EINVAL
    whole.close()
    loaded.close()


def test_misaligned_images_are_refused(F):
    """Each image is moved into shared memory by one bulk copy, which needs a 16-byte
    aligned source: an image array starting 8 bytes into a buffer is refused with
    FIRM_EINVAL before any GPU work (and an aligned one in the same buffer is taken)."""
    L = F._lib
    N, M = 16, 4
    inp = synth.config_inputs("C2", M=M, N=N)
    rec = F.Reconstructor(N, M, groups=inp["groups"], W=6)
    R, g, sh = _dev(inp["R"].reshape(M, 9)), _dev(inp["group_id"]), _dev(inp["shifts"])
    raw = torch.zeros(M * N * N + 4, dtype=torch.float32, device="cuda")
    bad = raw[2:2 + M * N * N]                           # 8 bytes past a 256-byte boundary
    with pytest.raises(L.FirmError) as e:
        rec.backproject(bad, sh, R, g)
    assert e.value.code == L.FIRM_EINVAL
    good = raw[4:4 + M * N * N]                          # 16 bytes past it
    good.copy_(torch.from_numpy(inp["images"].reshape(-1)).cuda())
    rhs = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    rec.backproject(good, sh, R, g, rhs_out=rhs)
    torch.cuda.synchronize()
    assert torch.isfinite(rhs).all()
    rec.close()
