"""Full-size parity at the workloads the benchmark and the configurations name: N=64 with
5,000 FP32 images (4 defocus groups, 30 CG iterations in its configuration) and N=128
with 50,000 BF16 images (20 defocus groups; the benchmark's workload), both at W=6,
sigma=2, lambda=1e-3 relative, in the launch configuration the benchmark uses.

The whole arrays are compared with the oracle's gridding mode (oracle/gridding.py: an
FP64 type-1 NUFFT with an exponential-of-semicircle window, pinned against the direct
sums in tests/test_oracle.py: ~1e-11 at W=12, ~1e-7 at W=8):

  * Ker (eq. kernel) on its stored half box, K-hat (eq. circ1) on its half spectrum and
    A*b (eq. backprojection): relative L2 <= 1e-5;
  * the volume after 10 plain CG iterations (Section 3.3) from the same seeded inputs:
    relative L2 <= 1e-4 against the oracle's FP64 CG run on the oracle's Ker and A*b.

The oracle itself is cross-checked at full size against its direct sums at a few
voxels (eq. kernel, eq. backprojection one voxel at a time), and so is the GPU.
BF16 images: the oracle takes the same BF16-rounded pixels.
"""
import multiprocessing as mp
import os
import time

import numpy as np
import pytest

import oracle as O
import synth
from oracle import gridding as Gr

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


def _oracle_voxel_sums(inp, images, vox):
    """Direct sums at the voxels vox over all images, split across host cores (spawned
    workers, so no CUDA state is inherited)."""
    N, M = inp["N"], inp["M"]
    K = O.disc(N)
    hg = O.ctf_weights(N, K, inp["groups"], np.arange(max(1, inp["groups"].shape[0]), dtype=np.int32)) \
        if inp["groups"].shape[0] else np.ones((1, K.shape[0]))
    nw = max(1, min(16, os.cpu_count() or 1))
    cuts = np.linspace(0, M, nw + 1).astype(int)
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
    return (sum(p[0] for p in parts), sum(p[1] for p in parts), sum(p[2] for p in parts),
            sum(p[3] for p in parts))


@pytest.mark.parametrize("cfg,bf16,w_oracle", [("C2", False, 12), ("C3", True, 8)])
def test_fullsize_whole_arrays_and_cg_volume_match_the_oracle(F, cfg, bf16, w_oracle):
    t0 = time.time()
    inp = synth.config_inputs(cfg)
    N, M = inp["N"], inp["M"]
    iters = 10
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
    khat = torch.empty(rec.half_shape(), dtype=torch.float32, device=dev)
    rhs = torch.empty((N, N, N), dtype=torch.float32, device=dev)
    rec.copy_out(F._lib.FIRM_OUT_KER, ker)
    rec.copy_out(F._lib.FIRM_OUT_KHAT, khat)
    rec.copy_out(F._lib.FIRM_OUT_RHS, rhs)
    x = torch.empty((N, N, N), dtype=torch.float32, device=dev)
    st, it = rec.cg_solve(x, iters)
    torch.cuda.synchronize()
    assert it == iters
    lam_gpu = rec.lambda_eff()
    ker, khat, rhs, x = (t.cpu().numpy() for t in (ker, khat, rhs, x))
    rec.close()
    del img, R, g
    torch.cuda.empty_cache()
    t_gpu = time.time() - t0

    # oracle: gridding NUFFT in FP64
    K = O.disc(N)
    Ker_o = Gr.kernel_gridded(inp["R"], inp["groups"], inp["group_id"], K, N, W=w_oracle).real
    rhs_o = Gr.backproject_gridded(images_used, inp["shifts"], inp["R"], inp["groups"], inp["group_id"], K,
                                   W=w_oracle)
    t_grid = time.time() - t0 - t_gpu
    e_ker = _rel(ker[:, :, :N], Ker_o[:, :, N:])
    Kh_o = O.khat(Ker_o)
    e_kh = _rel(khat, Kh_o.real[:, :, :N + 1])
    e_rhs = _rel(rhs, rhs_o)
    lam_o = O.lambda_eff(1e-3, 0, Ker_o[N, N, N])
    xo, _, _ = O.cg(lambda v: O.toeplitz_apply(Kh_o, v, lam_o).real, rhs_o, iters)
    e_x = _rel(x, xo)

    # the oracle's gridding and the GPU at a few voxels against the direct sums
    rng = np.random.default_rng(7)
    lk = np.stack([rng.integers(0, N, 6), rng.integers(-N, N, 6), rng.integers(-N, N, 6)], 1)
    lk = np.concatenate([[[0, 0, 0], [1, 0, 0]], lk])
    vr = rng.integers(-N // 2, N // 2, (8, 3))
    vox = np.concatenate([lk, vr])
    kd, rd, l1k, l1r = _oracle_voxel_sums(inp, images_used, vox)
    kd, rd = kd[:len(lk)].real, rd[len(lk):].real
    kg_o = Ker_o[lk[:, 2] + N, lk[:, 1] + N, lk[:, 0] + N]
    rg_o = rhs_o[vr[:, 2] + N // 2, vr[:, 1] + N // 2, vr[:, 0] + N // 2]
    kg = ker[lk[:, 2] + N, lk[:, 1] + N, lk[:, 0]]
    rg = rhs[vr[:, 2] + N // 2, vr[:, 1] + N // 2, vr[:, 0] + N // 2]
    print(f"{cfg}: Ker {e_ker:.2e}  K-hat {e_kh:.2e}  A*b {e_rhs:.2e}  CG volume ({iters} it) {e_x:.2e}  "
          f"lam_eff {abs(lam_gpu - lam_o) / lam_o:.1e}; oracle vs direct sums at voxels: Ker "
          f"{np.abs(kg_o - kd).max() / l1k:.1e}, A*b {np.abs(rg_o - rd).max() / l1r:.1e} (of l1); "
          f"GPU {t_gpu:.0f}s, oracle gridding {t_grid:.0f}s, total {time.time() - t0:.0f}s")
    # the oracle's own accuracy at this size (its window error is ~1e-7 or better)
    assert np.abs(kg_o - kd).max() <= 1e-8 * l1k
    assert np.abs(rg_o - rd).max() <= 1e-8 * l1r
    assert np.abs(kg - kd).max() <= 1e-5 * l1k and np.abs(rg - rd).max() <= 1e-5 * l1r
    # the gates
    assert abs(lam_gpu - lam_o) <= 1e-5 * lam_o
    assert e_ker <= 1e-5 and e_kh <= 1e-5 and e_rhs <= 1e-5
    assert e_x <= 1e-4
