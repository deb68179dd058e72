"""Learned preconditioner on the GPU against the FP64 oracle (oracle/lpre.py).

Features and targets are pinned through the oracle's definitions; the network's
gradient against the FP64 backward pass (itself pinned by finite differences); the BF16
forward pass against the FP32 one; training must lower the loss; the binned and table
preconditioners must run PCG to the tolerance.
"""
import numpy as np
import pytest

import oracle as O
from oracle import lpre as LP
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def F():
    import __graft_entry__ as g
    g.build()
    import paper_1307_5824_gb300 as pkg
    return pkg


def _plan(F, N, M, cfg="C5"):
    inp = synth.config_inputs(cfg, M=M, N=N)
    rec = F.Reconstructor(N, M, groups=inp["groups"], W=7, lam=1e-3)
    rec.kernel(torch.from_numpy(inp["R"].reshape(M, 9).copy()).cuda(), torch.from_numpy(inp["group_id"]).cuda())
    return inp, rec


def test_features_axis_and_target_match_oracle(F):
    N, M = 16, 60
    inp, rec = _plan(F, N, M)
    K = O.disc(N)
    h = O.ctf_weights(N, K, inp["groups"], inp["group_id"])
    a_o = LP.principal_axis(inp["R"])
    a_g = rec.pc_axis().astype(np.float64)
    assert abs(abs(a_g @ a_o) - 1.0) < 1e-5
    f = np.empty(1024, np.float32)
    rec.pc_features(f)
    f_o = LP.features(inp["R"], h, K, N, a_g / np.linalg.norm(a_g))
    print(f"features: L1 diff {np.abs(f - f_o).sum():.3e}")
    assert np.abs(f - f_o).sum() <= 2e-3            # points within rounding of a bin edge may move
    t = np.empty(1024, np.float32)
    rec.pc_target(t)
    Ker = O.kernel(inp["R"], h, K, N).real
    lam = O.lambda_eff(1e-3, 0, Ker[N, N, N])
    t_o = LP.target(O.wrapped_spectrum(Ker), lam, Ker[N, N, N], a_g / np.linalg.norm(a_g))
    d = np.abs(t - t_o)
    print(f"target: median {np.median(d):.3e} max {d.max():.3e}")
    assert np.median(d) <= 1e-4 and np.mean(d) <= 1e-2
    rec.close()


def test_bin_volumes_and_baseline_match_oracle(F):
    N, M = 16, 60
    inp, rec = _plan(F, N, M)
    a_g = rec.pc_axis().astype(np.float64)
    a_g /= np.linalg.norm(a_g)
    v = np.empty(1024, np.float32)
    rec.pc_bin_volumes(v)
    v_o = LP.bin_volumes(N, a_g)
    assert abs(v.sum() - 1.0) <= 1e-6
    assert np.abs(v - v_o).sum() <= 2e-3            # frequencies on a cone edge may move
    f = np.empty(1024, np.float32)
    rec.pc_features(f)
    b = np.empty(1024, np.float32)
    rec.pc_baseline(b)
    b_o = LP.baseline(f.astype(np.float64), v.astype(np.float64), 1e-3)
    assert np.abs(b - b_o).max() <= 1e-4
    rec.close()


def test_mlp_gradient_and_bf16_forward_match_oracle(F):
    L = F._lib
    rng = np.random.default_rng(60)
    params_np = []
    w = LP.WIDTHS
    for i in range(3):
        params_np.append(rng.standard_normal((w[i + 1], w[i])) / np.sqrt(w[i]))
        params_np.append(0.1 * rng.standard_normal(w[i + 1]))
    flat = np.concatenate([p.ravel() for p in params_np]).astype(np.float32)
    B = 5
    x = rng.standard_normal((B, 1024)).astype(np.float32)
    t = rng.standard_normal((B, 1024)).astype(np.float32)
    dev = torch.device("cuda")
    P = torch.from_numpy(flat).to(dev)
    g = torch.empty_like(P)
    work = torch.empty(L.firm_mlp_work_floats(B), dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    L.firm_mlp_grad(P, B, torch.from_numpy(x).to(dev), torch.from_numpy(t).to(dev), g, work, loss)
    torch.cuda.synchronize()
    p32 = [p.astype(np.float32).astype(np.float64) for p in params_np]
    lo, go = LP.mlp_loss_grad(p32, x.astype(np.float64), t.astype(np.float64))
    assert abs(float(loss.item()) - lo) <= 1e-5 * lo
    gg = g.cpu().numpy()
    off = 0
    for ref in go:
        got = gg[off:off + ref.size].reshape(ref.shape)
        off += ref.size
        assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref)
    y32 = np.empty((B, 1024), np.float32)
    yb = np.empty((B, 1024), np.float32)
    xd = torch.from_numpy(x).to(dev)
    yd = torch.empty((B, 1024), device=dev)
    L.firm_mlp_forward(P, B, xd, yd, work)
    y32 = yd.cpu().numpy()
    yo, _ = LP.mlp_forward(p32, x.astype(np.float64))
    assert np.linalg.norm(y32 - yo) <= 1e-5 * np.linalg.norm(yo)
    pb = torch.empty(P.numel(), dtype=torch.bfloat16, device=dev)
    L.firm_mlp_to_bf16(P, pb)
    L.firm_mlp_forward_bf16(pb, P, B, xd, yd, work)
    yb = yd.cpu().numpy()
    e = np.linalg.norm(yb - y32) / np.linalg.norm(y32)
    print(f"bf16 forward rel err {e:.2e}")
    assert e <= 2e-2


def test_training_lowers_loss_and_preconditioners_converge(F):
    from paper_1307_5824_gb300 import learned
    X, T = learned.generate(24, N=16, seed=61, m_range=(40, 120))
    params, hist = learned.train(X, T, steps=300, batch=16, lr=1e-3, log_every=100)
    print("loss history", hist)
    assert hist[-1][1] < 0.5 * hist[0][1]
    N, M = 16, 100
    inp, rec = _plan(F, N, M)
    g = torch.from_numpy(inp["group_id"]).cuda()
    R = torch.from_numpy(inp["R"].reshape(M, 9).copy()).cuda()
    rec.backproject(torch.from_numpy(inp["images"]).cuda(), torch.from_numpy(inp["shifts"]).cuda(), R, g)
    x = torch.empty((N, N, N), device="cuda")
    its = {}
    for name, mode in (("none", F._lib.FIRM_PRECOND_NONE), ("binned", F._lib.FIRM_PRECOND_BINNED),
                       ("circulant", F._lib.FIRM_PRECOND_CIRCULANT)):
        rec.set_precond(mode)
        st, its[name] = rec.cg_solve(x, 800, rel_tol=1e-4)
        assert st == 0
    learned.apply_learned(rec, params)
    st, its["learned"] = rec.cg_solve(x, 800, rel_tol=1e-4)
    assert st == 0
    print("iterations", its)
    # what the trained network gains over the method without it (plain CG)
    assert its["learned"] <= 0.8 * its["none"]
    rec.close()
