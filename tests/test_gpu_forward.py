"""The forward projector A (eq. forward-projector, Section 3.1) and the data term of
Section 3.3 on the GPU (firm_forward, firm_data_residual), against the FP64 oracle's
direct sums: A V at every half-disc sample, and sum |b - A V|^2, sum |b|^2 over every
image's whole disc (b = image_dft with the shift phase, eq. measurement).

Tolerances: the type-2 NUFFT uses the same Kaiser-Bessel window as the spreading, so
A V carries the same window error as A*b (about 5e-6 relative at W = 6, 1e-6 at
W = 7) plus FP32 rounding; the gates are those of the A*b parity test."""
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
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


def half_disc(N):
    h = N // 2
    H = [(0, k2) for k2 in range(0, h + 1)]
    H += [(k1, k2) for k1 in range(1, h + 1) for k2 in range(-h, h + 1) if k1 * k1 + k2 * k2 <= h * h]
    return np.array(H)


def _volume(N, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((N, N, N)).astype(np.float32)


@pytest.mark.parametrize("N,M,W", [(16, 30, 6), (16, 25, 7), (32, 20, 6), (32, 12, 8)])
def test_forward_projector_matches_oracle(F, N, M, W):
    inp = synth.config_inputs("C2", M=M, N=N)
    V = _volume(N, 5)
    H = half_disc(N)
    h = O.ctf_weights(N, H, inp["groups"], inp["group_id"])
    ref = O.forward(V.astype(np.float64), inp["R"], h, H)
    rec = F.Reconstructor(N, M, groups=inp["groups"], W=W)
    out = rec.forward(torch.from_numpy(V).cuda(), torch.from_numpy(inp["R"].reshape(M, 9).copy()).cuda(),
                      torch.from_numpy(inp["group_id"]).cuda())
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    got = got[..., 0] + 1j * got[..., 1]
    e = rel(got, ref)
    print(f"A V N={N} M={M} W={W}: rel err {e:.3e}")
    assert e <= 1e-5
    # host arrays in and out through the same entry point
    out_h = np.empty((M, H.shape[0], 2), np.float32)
    F._lib.firm_forward(rec.plan, M, V, inp["R"].reshape(M, 9).copy(), inp["group_id"], out_h)
    assert rel(out_h[..., 0] + 1j * out_h[..., 1], ref) <= 1e-5
    rec.close()


def test_data_residual_matches_oracle(F):
    N, M, W = 16, 40, 6
    inp = synth.config_inputs("C2", M=M, N=N)
    K = O.disc(N)
    h = O.ctf_weights(N, K, inp["groups"], inp["group_id"])
    b = O.image_dft(inp["images"].astype(np.float64), K, inp["shifts"])
    rec = F.Reconstructor(N, M, groups=inp["groups"], W=W, lam=1e-3)
    d = torch.device("cuda")
    R = torch.from_numpy(inp["R"].reshape(M, 9).copy()).to(d)
    gid = torch.from_numpy(inp["group_id"]).to(d)
    img = torch.from_numpy(inp["images"]).to(d)
    sh = torch.from_numpy(inp["shifts"]).to(d)
    # a random volume (no cancellation) and the 10-iteration CG volume (the data term
    # the reconstruction lowers)
    rec.kernel(R, gid)
    rec.backproject(img, sh, R, gid)
    x = torch.empty((N, N, N), dtype=torch.float32, device=d)
    rec.cg_solve(x, 10)
    for name, V, tol in (("random", _volume(N, 7), 1e-5), ("CG", x.cpu().numpy(), 1e-4)):
        res_o = float(np.sum(np.abs(b - O.forward(V.astype(np.float64), inp["R"], h, K)) ** 2))
        b2_o = float(np.sum(np.abs(b) ** 2))
        res, b2 = rec.data_residual(torch.from_numpy(V).to(d), img, sh, R, gid)
        print(f"data term, {name} volume: |b-AV|^2/|b|^2 = {res / b2:.4f}; rel err {abs(res - res_o) / res_o:.2e} "
              f"(|b|^2 {abs(b2 - b2_o) / b2_o:.2e})")
        assert abs(b2 - b2_o) <= 1e-5 * b2_o
        assert abs(res - res_o) <= tol * res_o
        again = rec.data_residual(torch.from_numpy(V).to(d), img, sh, R, gid)
        # FP64 partials per work item; the point order inside the binning may differ
        assert abs(again[0] - res) <= 1e-12 * res and abs(again[1] - b2) <= 1e-12 * b2
    # the CG volume lowers the data term below that of V = 0 (= |b|^2)
    res_cg, b2 = rec.data_residual(x, img, sh, R, gid)
    assert res_cg < b2
    assert rec.data_residual(x, img, sh, R, gid, M=0) == (0.0, 0.0)
    rec.close()


def test_forward_projector_rejects_bad_arguments(F):
    rec = F.Reconstructor(16, 8, W=6)
    V = torch.zeros((16, 16, 16), device="cuda")
    R = torch.zeros((9, 9), dtype=torch.float64, device="cuda")
    with pytest.raises(F.FirmError):
        rec.forward(V, R, M=9)                          # above the plan's M
    with pytest.raises(F.FirmError):
        F._lib.firm_forward(rec.plan, 4, None, R, None, V)
    with pytest.raises(F.FirmError):
        F._lib.firm_data_residual(rec.plan, 4, V, None, None, R)
    rec.close()
