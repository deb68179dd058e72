"""The allocation-free Toeplitz apply (firm_toeplitz_apply_static).

Some callers cannot allocate device memory at all -- a host application whose own
allocator already owns the GPU's memory, or a code path that must keep the device
footprint fixed -- and have no workspace to lend.  This entry point serves them from
a static array inside the library.  The tests call it through the C ABI, twice in a
row for each size (the array keeps the previous call's contents, which must not leak
into the next result), at every size the array is dimensioned for (N = 16, 32, 48 and
64, the last one filling it), against the FP64 oracle's circulant apply and against
the plan-based firm_toeplitz_apply, and check that sizes above its maximum are
refused.
"""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _even_kernel(N, rng):
    """A real kernel over [-N, N)^3 with Ker(-n) = Ker(n): a positive lag-0 peak, a
    smooth decay and random even structure (the lag -N planes are zero)."""
    n = np.arange(-N, N)
    r2 = n[:, None, None] ** 2 + n[None, :, None] ** 2 + n[None, None, :] ** 2
    A = rng.standard_normal((2 * N,) * 3) * np.exp(-r2 / (2.0 * (N / 3.0) ** 2))
    A[0], A[:, 0], A[:, :, 0] = 0.0, 0.0, 0.0
    Ker = A.copy()
    Ker[1:, 1:, 1:] = 0.5 * (A[1:, 1:, 1:] + A[1:, 1:, 1:][::-1, ::-1, ::-1])
    Ker[N, N, N] += 4.0 * np.abs(Ker).sum() ** 0.5
    return Ker


@pytest.mark.parametrize("N", [16, 32, 48, 64])
def test_static_scratch_apply_matches_oracle(N):
    import __graft_entry__ as g
    g.build()
    import paper_1307_5824_gb300 as F
    L = F._lib
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(100 + N)
    Ker = _even_kernel(N, rng)
    khat_full = O.khat(Ker)
    khat = torch.from_numpy(O.khat_half(Ker).astype(np.float32)).cuda()
    lam = 0.03 * float(Ker[N, N, N])
    for call in range(2):
        x64 = rng.standard_normal((N, N, N))
        x = torch.from_numpy(x64.astype(np.float32)).cuda()
        y = torch.full_like(x, float("nan"))
        L.firm_toeplitz_apply_static(N, khat, lam, x, y, stream)
        torch.cuda.synchronize()
        assert torch.isfinite(y).all()
        ref = O.toeplitz_apply(khat_full, x.double().cpu().numpy(), lam).real
        assert _rel(y.cpu().numpy(), ref) <= 1e-5, (N, call)


def test_static_scratch_apply_matches_plan_apply():
    import __graft_entry__ as g
    g.build()
    import paper_1307_5824_gb300 as F
    L = F._lib
    stream = torch.cuda.current_stream().cuda_stream
    for N, M in ((64, 60), (48, 60), (32, 80), (16, 40)):
        inp = synth.config_inputs("C2", M=M, N=N)
        rec = F.Reconstructor(N, M, groups=inp["groups"], W=6, lam=1e-2)
        rec.kernel(torch.from_numpy(inp["R"].reshape(M, 9).copy()).cuda(),
                   torch.from_numpy(inp["group_id"]).cuda())
        khat = torch.empty(rec.half_shape(), dtype=torch.float32, device="cuda")
        rec.copy_out(L.FIRM_OUT_KHAT, khat)
        lam = rec.lambda_eff()
        rng = np.random.default_rng(N)
        for call in range(2):
            x = torch.from_numpy(rng.standard_normal((N, N, N)).astype(np.float32)).cuda()
            y_plan = torch.empty_like(x)
            y_static = torch.full_like(x, float("nan"))
            rec.toeplitz_apply(x, y_plan)
            L.firm_toeplitz_apply_static(N, khat, lam, x, y_static, stream)
            torch.cuda.synchronize()
            assert torch.isfinite(y_static).all()
            assert _rel(y_static.cpu().numpy(), y_plan.cpu().numpy()) <= 1e-5, (N, call)
        rec.close()
    # beyond the static maximum (N = 64) the call is refused before any GPU work
    x = torch.zeros((96, 96, 96), dtype=torch.float32, device="cuda")
    kh = torch.zeros((192, 192, 97), dtype=torch.float32, device="cuda")
    with pytest.raises(L.FirmError) as e:
        L.firm_toeplitz_apply_static(96, kh, 0.0, x, torch.empty_like(x), stream)
    assert e.value.code == L.FIRM_EINVAL
    # host memory is refused as well
    xh = torch.zeros((16, 16, 16), dtype=torch.float32)
    khh = torch.zeros((32, 32, 17), dtype=torch.float32)
    with pytest.raises(L.FirmError) as e:
        L.firm_toeplitz_apply_static(16, khh, 0.0, xh, torch.empty_like(xh), stream)
    assert e.value.code == L.FIRM_EINVAL
