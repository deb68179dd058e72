"""Full-size parity on sampled outputs: Ker and A*b of the whole workloads (N=64 with
5,000 images; N=128 with 50,000 BF16 images, the configuration the benchmark times:
W=6, sigma=2), each compared at a few voxels with the oracle's direct sums
(eq. kernel, eq. backprojection), which it can evaluate one voxel at a time.

Bounds: a type-1 NUFFT's error at any output is at most a small multiple of the l1
norm of its weights (sum h^2 for Ker, sum |h b| for A*b), and over the sampled voxels
the relative L2 error stays at the window's ~5e-6 (W=6).
"""
import multiprocessing as mp
import os

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


def _oracle_sums(inp, images, nvox_ker, nvox_rhs):
    """Oracle sums over all images, split across host cores (spawned workers)."""
    N, M = inp["N"], inp["M"]
    K = O.disc(N)
    hg = O.ctf_weights(N, K, inp["groups"], np.arange(max(1, inp["groups"].shape[0]), dtype=np.int32)) \
        if inp["groups"].shape[0] else np.ones((1, K.shape[0]))
    nw = max(1, min(16, os.cpu_count() or 1))
    cuts = np.linspace(0, M, nw + 1).astype(int)
    vox = np.concatenate([nvox_ker, nvox_rhs])
    jobs = [(inp["R"][a:b], inp["group_id"][a:b], hg, images[a:b], inp["shifts"][a:b], K, N, vox)
            for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
    old = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in old:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(len(jobs)) as pool:
            parts = pool.starmap(O.sums_at_voxels, jobs)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    ker = sum(p[0] for p in parts)
    rhs = sum(p[1] for p in parts)
    l1k = sum(p[2] for p in parts)
    l1r = sum(p[3] for p in parts)
    nk = len(nvox_ker)
    return ker[:nk], rhs[nk:], l1k, l1r


@pytest.mark.parametrize("cfg,bf16", [("C2", False), ("C3", True)])
def test_fullsize_kernel_and_rhs_at_sampled_voxels(F, cfg, bf16):
    inp = synth.config_inputs(cfg)
    N, M = inp["N"], inp["M"]
    dev = torch.device("cuda")
    img = torch.from_numpy(inp["images"]).to(dev)
    if bf16:
        img = img.to(torch.bfloat16)
    images_used = img.float().cpu().numpy()          # the pixels the GPU reads (BF16-rounded)
    del inp["images"]
    rec = F.Reconstructor(N, M, groups=inp["groups"], W=6, lam=1e-3,
                          img_dtype=F._lib.FIRM_IMG_BF16 if bf16 else F._lib.FIRM_IMG_F32)
    R = torch.from_numpy(inp["R"].reshape(M, 9).copy()).to(dev)
    g = torch.from_numpy(inp["group_id"]).to(dev)
    rec.kernel(R, g)
    rec.backproject(img, torch.from_numpy(inp["shifts"]).to(dev), R, g)
    ker = torch.empty(rec.half_shape(), dtype=torch.float32, device=dev)
    rhs = torch.empty((N, N, N), dtype=torch.float32, device=dev)
    rec.copy_out(F._lib.FIRM_OUT_KER, ker)
    rec.copy_out(F._lib.FIRM_OUT_RHS, rhs)
    torch.cuda.synchronize()
    ker, rhs = ker.cpu().numpy(), rhs.cpu().numpy()
    rec.close()
    del img

    rng = np.random.default_rng(7)
    # lags (n1, n2, n3): n1 in [0, N), n2, n3 in [-N, N); plus lag 0 and a few small lags
    lk = np.stack([rng.integers(0, N, 10), rng.integers(-N, N, 10), rng.integers(-N, N, 10)], 1)
    lk = np.concatenate([[[0, 0, 0], [1, 0, 0], [0, 2, -1]], lk])
    vr = rng.integers(-N // 2, N // 2, (13, 3))
    ko, ro, l1k, l1r = _oracle_sums(inp, images_used, lk, vr)
    kg = ker[lk[:, 2] + N, lk[:, 1] + N, lk[:, 0]]
    rg = rhs[vr[:, 2] + N // 2, vr[:, 1] + N // 2, vr[:, 0] + N // 2]
    ek = np.abs(kg - ko.real)
    er = np.abs(rg - ro.real)
    rel_k = np.linalg.norm(kg - ko.real) / np.linalg.norm(ko.real)
    rel_r = np.linalg.norm(rg - ro.real) / np.linalg.norm(ro.real)
    print(f"{cfg}: Ker max|err|/l1 {ek.max() / l1k:.2e} rel-L2 {rel_k:.2e}; "
          f"A*b max|err|/l1 {er.max() / l1r:.2e} rel-L2 {rel_r:.2e}")
    assert ek.max() <= 1e-5 * l1k and er.max() <= 1e-5 * l1r
    assert rel_k <= 1.5e-5 and rel_r <= 3e-5
