"""The FP64 oracle's whole FIRM reconstruction at large N -- test infrastructure only.

Only the tests, the smoke check and the benchmark's CPU-baseline / reference legs may
use this module.  It chains the oracle's own steps in the order of Section 3.4:
  1-2. image DFTs on the disc with the shift phase and the CTF, spread and transformed
       to A*b (eq. measurement, eq. backprojection) by the gridding NUFFT of
       oracle/gridding.py;
  3.   Ker (eq. kernel) by the same NUFFT, its circulant embedding and K-hat
       (eq. embedding_circulant, eq. circ1);
  4.   textbook CG (Section 3.3) on (A*A + lam_eff I) V = A*b from V = 0.
Each part is timed, so that a bounded sample of the images can stand for the whole
set: the spreading work is linear in the images, the transforms and the CG are not.
"""
from __future__ import annotations

import time

import numpy as np

from . import firm as _F
from . import gridding as _G

__all__ = ["reconstruct"]


def reconstruct(inp, *, iters=None, rel_tol=0.0, W=6, window="kb", threads=None, images=None,
                sample_images=None, cg_iters_timed=None):
    """FIRM steps 1-4 on the workload `inp` (synth.config_inputs) in FP64.

    images: the pixels to use (default inp["images"]).  sample_images: spread only the
    first that many images and scale the spreading time to all M (the returned volume
    is then not the workload's).  cg_iters_timed: run that many CG iterations and scale
    their time to `iters`.  Returns (volume or None, seconds per reconstruction,
    timing parts, CG iterations)."""
    N, M = inp["N"], inp["M"]
    images = inp["images"] if images is None else images
    Ms = M if sample_images is None else min(M, int(sample_images))
    K = _F.disc(N)
    sub = dict(R=inp["R"][:Ms], group_id=inp["group_id"][:Ms])
    tk, tb = {}, {}
    Ker = _G.kernel_gridded(sub["R"], inp["groups"], sub["group_id"], K, N, W=W, window=window,
                            threads=threads, timing=tk).real
    rhs = _G.backproject_gridded(images[:Ms], inp["shifts"][:Ms], sub["R"], inp["groups"], sub["group_id"], K,
                                 W=W, window=window, threads=threads, timing=tb)
    t0 = time.perf_counter()
    Kh = _F.khat(Ker)
    t_khat = time.perf_counter() - t0
    lam = _F.lambda_eff(float(inp["cfg"]["lam"]), 0, Ker[N, N, N])      # the workload's lambda (reading 6)
    n_run = iters if cg_iters_timed is None else min(int(cg_iters_timed), int(iters))
    t0 = time.perf_counter()
    x, hist, it = _F.cg(lambda v: _F.toeplitz_apply(Kh, v, lam).real, rhs, n_run if n_run is not None else 100000,
                        rel_tol=rel_tol)
    t_cg = time.perf_counter() - t0
    n_total = it if cg_iters_timed is None else int(iters)
    scale = M / Ms
    parts = {"spread_ker_s": tk["spread_s"] * scale, "spread_rhs_s": tb["spread_s"] * scale,
             "transform_ker_s": tk["transform_s"], "transform_rhs_s": tb["transform_s"], "khat_s": t_khat,
             "cg_s": t_cg / max(it, 1) * n_total, "cg_s_per_iter": t_cg / max(it, 1), "images_spread": Ms}
    total = sum(v for k, v in parts.items() if k.endswith("_s") and k != "cg_s_per_iter")
    return (x if Ms == M else None), total, parts, n_total
