"""The allocation-free Toeplitz apply (firm_toeplitz_apply_static) gives the same result
as the plan-based firm_toeplitz_apply.

Some callers cannot allocate device memory at all -- a host application whose own
allocator already owns the GPU's memory, or a code path that must keep the device
footprint fixed -- and have no workspace to lend.  This entry point serves them from
a static array inside the library.  The test calls it twice in a row through the C ABI
(the array keeps the previous call's contents, which must not leak into the next
result) and checks that sizes above its maximum are refused.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_static_scratch_apply_matches_plan_apply():
    import __graft_entry__ as g
    g.build()
    import paper_1307_5824_gb300 as F
    L = F._lib
    stream = torch.cuda.current_stream().cuda_stream
    for N, M in ((32, 80), (16, 40)):
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
            assert _rel(y_static, y_plan) <= 1e-5, (N, call)
        rec.close()
    # beyond the static maximum (N = 64) the call is refused before any GPU work
    x = torch.zeros((96, 96, 96), dtype=torch.float32, device="cuda")
    kh = torch.zeros((192, 192, 97), dtype=torch.float32, device="cuda")
    with pytest.raises(L.FirmError) as e:
        L.firm_toeplitz_apply_static(96, kh, 0.0, x, torch.empty_like(x), stream)
    assert e.value.code == L.FIRM_EINVAL
