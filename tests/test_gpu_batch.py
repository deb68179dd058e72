"""Batched reconstructions (firm_batch_*): every volume of a batch equals what the
single-plan calls give for that plan (firm_kernel, firm_backproject, firm_cg_solve with
a fixed iteration count, Section 3.4), in every execution form (worker streams only,
persistent spreading, CUDA graph, tuned), and the N=16 member matches the FP64
oracle's CG after the same count.  That oracle comparison uses 10 iterations: on this
CTF-weighted problem the 25-iteration iterate moves by > 1e-3 under 1e-9 operator
noise even in FP64 (test_cg_trajectory_horizon_under_tiny_operator_noise)."""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ITERS = 25


@pytest.fixture(scope="module")
def F():
    import __graft_entry__ as g
    g.build()
    import paper_1307_5824_gb300 as pkg
    return pkg


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


# (N, M, groups used) -- uneven sizes, N = 80 included
SPECS = [(16, 60, 2), (48, 300, 1), (32, 150, 4), (80, 120, 3), (64, 200, 2), (16, 0, 1)]


def _problem(k, N, M, ng):
    inp = synth.config_inputs("C2", M=max(M, 1), N=N)
    rng = np.random.default_rng(100 + k)
    sub = rng.choice(inp["groups"].shape[0], ng, replace=False)
    groups = inp["groups"][sub]
    gid = rng.integers(0, ng, max(M, 1)).astype(np.int32)
    return dict(N=N, M=M, R=inp["R"][:max(M, 1)], shifts=inp["shifts"][:max(M, 1)],
                images=inp["images"][:max(M, 1)], groups=groups, gid=gid)


@pytest.fixture(scope="module")
def problems():
    return [_problem(k, *s) for k, s in enumerate(SPECS)]


def _dev_item(p, x):
    d = torch.device("cuda")
    M = p["M"]
    return dict(M=M, R=torch.from_numpy(p["R"].reshape(-1, 9).copy()).to(d),
                group=torch.from_numpy(p["gid"]).to(d), images=torch.from_numpy(p["images"]).to(d),
                shifts=torch.from_numpy(p["shifts"]).to(d), x=x)


def _single(F, p):
    """The single-plan path for one problem."""
    N, M = p["N"], p["M"]
    rec = F.Reconstructor(N, max(M, 1), groups=p["groups"], W=6, lam=1e-3)
    it = _dev_item(p, None)
    rec.kernel(it["R"], it["group"], M=M)
    rec.backproject(it["images"], it["shifts"], it["R"], it["group"], M=M)
    x = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    st, n = rec.cg_solve(x, ITERS)
    assert st == 0 and n == (ITERS if M > 0 else n)
    torch.cuda.synchronize()
    out = x.cpu().numpy()
    rec.close()
    return out


def test_batch_matches_single_plans_and_oracle(F, problems):
    refs = [_single(F, p) for p in problems]
    recs = [F.Reconstructor(p["N"], max(p["M"], 1), groups=p["groups"], W=6, lam=1e-3) for p in problems]
    xs = [torch.zeros((p["N"],) * 3, dtype=torch.float32, device="cuda") for p in problems]
    items = [_dev_item(p, x) for p, x in zip(problems, xs)]
    B = F.BatchReconstructor(recs, n_streams=4)
    B.set_items(items)
    results = {}
    for name, graph, persistent in (("streams", False, False), ("persistent", False, True),
                                    ("graph", True, False), ("graph+persistent", True, True),
                                    ("replay", True, True)):
        for x in xs:
            x.zero_()
        B.run(ITERS, graph=graph, persistent=persistent)
        st, sts, its = B.wait()
        assert st == 0 and (sts == 0).all()
        assert all(int(i) == ITERS for i, p in zip(its, problems) if p["M"] > 0)
        got = [x.cpu().numpy() for x in xs]
        errs = [rel(g, r) if np.linalg.norm(r) > 0 else float(np.abs(g).max()) for g, r in zip(got, refs)]
        print(name, ["%.1e" % e for e in errs], "launches", B.launch_count())
        assert max(errs) <= 2e-5, (name, errs)
        results[name] = got
    assert B.launch_count() > 0
    # the tuner picks a configuration; results stay the same under it
    cfg = B.tune(ITERS)
    print("tuned", cfg)
    B.run(ITERS)
    B.wait()
    for x, r in zip(xs, refs):
        if np.linalg.norm(r) > 0:
            assert rel(x.cpu().numpy(), r) <= 2e-5
    # plans are usable on their own after the batch (lam_eff, A*b)
    lam = recs[0].lambda_eff()
    assert lam > 0
    # the N = 16 member against the oracle's CG (10 iterations, lam_eff = 1e-3 Ker(0))
    B.run(10)
    B.wait()
    x10 = xs[0].cpu().numpy()
    p = problems[0]
    N = p["N"]
    K = O.disc(N)
    h = O.ctf_weights(N, K, p["groups"], p["gid"])
    Ker = O.kernel(p["R"], h, K, N).real
    rhs = O.backproject(p["images"].astype(np.float64), p["shifts"], p["R"], h, K)
    lam_o = O.lambda_eff(1e-3, 0, Ker[N, N, N])
    assert abs(lam - lam_o) <= 1e-5 * lam_o
    Kh = O.khat(Ker).real
    xo, _, _ = O.cg(lambda v: O.toeplitz_apply(Kh, v, lam_o).real, rhs, 10)
    e = rel(x10, xo)
    print(f"batch N=16 vs oracle after 10 iterations: {e:.2e}")
    assert e <= 1e-4
    # the empty member: no images, x = 0
    assert float(np.abs(results["graph+persistent"][-1]).max()) == 0.0
    B.close()
    for r in recs:
        r.close()


def test_batch_rejects_bad_arguments(F):
    recs = [F.Reconstructor(16, 8, W=6), F.Reconstructor(16, 8, W=7)]
    with pytest.raises(F.FirmError):
        F.BatchReconstructor(recs)                       # mixed W
    B = F.BatchReconstructor(recs[:1])
    with pytest.raises(F.FirmError):
        B.set_config(0, 4096)
    with pytest.raises(F.FirmError):
        B.set_config(1, 1000)
    x = torch.zeros((16, 16, 16), device="cuda")
    B.set_items([dict(M=9, R=torch.zeros((9, 9), dtype=torch.float64, device="cuda"),
                      images=torch.zeros((9, 16, 16), device="cuda"), x=x)])
    with pytest.raises(F.FirmError):
        B.run(5)                                          # M above the plan's M
    B.close()
    for r in recs:
        r.close()


def _true_res(L, rec, x):
    """||A*b - (A*A + lam_eff) x|| / ||A*b|| of a plan's volume (one Toeplitz apply)."""
    y = torch.empty_like(x)
    b = torch.empty_like(x)
    rec.toeplitz_apply(x, y)
    rec.copy_out(L.FIRM_OUT_RHS, b)
    torch.cuda.synchronize()
    bn = b.double().cpu().numpy()
    return float(np.linalg.norm(bn - y.double().cpu().numpy()) / np.linalg.norm(bn))


def _single_solve(F, p, max_iter, rel_tol, mode=None, infer=None):
    """The single-plan path to a tolerance: firm_cg_solve with the plan's preconditioner."""
    N, M = p["N"], p["M"]
    rec = F.Reconstructor(N, max(M, 1), groups=p["groups"], W=6, lam=1e-3)
    it = _dev_item(p, None)
    rec.kernel(it["R"], it["group"], M=M)
    rec.backproject(it["images"], it["shifts"], it["R"], it["group"], M=M)
    if infer is not None:
        infer.apply(rec)
    elif mode is not None:
        rec.set_precond(mode)
    x = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    st, n = rec.cg_solve(x, max_iter, rel_tol=rel_tol, allow=(F._lib.FIRM_ENOTCONV,))
    torch.cuda.synchronize()
    out = x.cpu().numpy()
    rec.close()
    return out, n


def test_batch_solve_to_tolerance_with_each_preconditioner(F, problems):
    """firm_batch_solve: every plan of the batch to rel-res 1e-3 with plain CG, with its own
    circulant preconditioner and with the batch's learned network (one forward pass for
    all plans), in chunked CG with and without a CUDA graph.  Every volume meets the
    tolerance (its true residual, recomputed) and needs the iterations the single-plan
    firm_cg_solve needs, within a few (a long CG run's stopping iteration moves with the
    last bits of Ker, whose FP64 atomics add in a different order run to run); the
    circulant preconditioner needs fewer iterations in total than plain CG; a
    circulant-preconditioned member after 8 iterations matches the oracle's PCG
    (Section 3.3's CG with a preconditioner)."""
    from paper_1307_5824_gb300 import learned
    L = F._lib
    tol = 1e-3
    X, T = learned.generate(64, N=32, seed=61, m_range=(60, 300))
    net, _ = learned.train(X, T, steps=800, batch=16, lr=1e-3, log_every=200)
    infer = learned.DeviceInference(net)
    recs = [F.Reconstructor(p["N"], max(p["M"], 1), groups=p["groups"], W=6, lam=1e-3) for p in problems]
    xs = [torch.zeros((p["N"],) * 3, dtype=torch.float32, device="cuda") for p in problems]
    items = [_dev_item(p, x) for p, x in zip(problems, xs)]
    B = F.BatchReconstructor(recs, n_streams=4)
    B.set_items(items)
    B.set_network(net)
    totals = {}
    for name, mode in (("plain", L.FIRM_PRECOND_NONE), ("circulant", L.FIRM_PRECOND_CIRCULANT),
                       ("learned", None)):
        for r in recs:
            r.set_precond(mode if mode is not None else L.FIRM_PRECOND_NONE)
        for graph in (False, True):
            for x in xs:
                x.zero_()
            B.solve(1000, tol, graph=graph, learned=mode is None)
            st, sts, its = B.wait(allow=(L.FIRM_ENOTCONV,))
            assert (sts == 0).all() or mode is None, (name, sts)
            for k, (p, x) in enumerate(zip(problems, xs)):
                if p["M"] == 0:
                    assert float(x.abs().max()) == 0.0
                    continue
                ref, n_ref = _single_solve(F, p, 1000, tol, mode=mode, infer=infer if mode is None else None)
                tr = _true_res(L, recs[k], x)
                e = rel(x.cpu().numpy(), ref)
                print(name, graph, k, "iterations", int(its[k]), n_ref, "true res %.2e" % tr, "vs single %.1e" % e)
                assert abs(int(its[k]) - n_ref) <= max(3, 0.05 * n_ref), (name, graph, k, int(its[k]), n_ref)
                if sts[k] == 0:
                    assert tr <= 2 * tol and e <= 20 * tol, (name, graph, k, tr, e)
                else:                                   # the single-plan solve stops at max_iter too
                    assert n_ref == 1000 and e <= 1e-2, (name, graph, k, n_ref, e)
        totals[name] = int(its.sum())
    print("batched iterations to rel-res 1e-3:", totals)
    # (the network's gain over plain CG is asserted with a proper training set in
    # tests/test_gpu_lpre.py and measured on the batched workload by the benchmark; this
    # small network is only there to drive the batched path)
    assert totals["circulant"] < totals["plain"]
    # a preconditioned member after a fixed count against the oracle's PCG
    for r in recs:
        r.set_precond(L.FIRM_PRECOND_CIRCULANT)
    B.solve(8, 0.0)
    B.wait()
    p = problems[2]                                      # N = 32, 150 images, 4 groups
    N = p["N"]
    K = O.disc(N)
    # the oracle's Ker and A*b with the batch's own NUFFT (Kaiser-Bessel W = 6) in FP64:
    # this lambda = 1e-3 PCG iterate amplifies the window's ~5e-6 error to ~1e-4, which is
    # the method's approximation, not the FP32 path's
    from oracle import gridding as Gr
    Ker = Gr.kernel_gridded(p["R"], p["groups"], p["gid"], K, N, W=6, window="kb").real
    rhs = Gr.backproject_gridded(p["images"], p["shifts"], p["R"], p["groups"], p["gid"], K, W=6, window="kb")
    lam = O.lambda_eff(1e-3, 0, Ker[N, N, N])
    Kh = O.khat(Ker).real
    Pc = O.circulant_preconditioner(O.wrapped_spectrum(Ker), lam)
    xo, _, _ = O.cg(lambda v: O.toeplitz_apply(Kh, v, lam).real, rhs, 8, precond=Pc)
    e = rel(xs[2].cpu().numpy(), xo)
    print(f"batched PCG member vs oracle after 8 iterations: {e:.2e}")
    assert e <= 1e-4
    # learned without a network is refused
    B.set_network(net)
    L.firm_batch_set_network(B.batch, None, None)
    with pytest.raises(F.FirmError) as ex:
        B.solve(10, tol, learned=True)
    assert ex.value.code == L.FIRM_ESTATE
    B.close()
    for r in recs:
        r.close()
