"""Image-sharded FIRM across processes (torch.distributed; argument marshalling only).

Ker and A*b are sums over the images (eq. kernel, eq. backprojection; Section 3.4), so
one reconstruction can be split by images: every process spreads its own images with
its own plan, the partial Ker half boxes and A*b are summed by all-reduce (the one
exchange step), and every process loads the sums into its plan (firm_load_sums), which
forms K-hat and lam_eff from them; CG then runs on each process (it is cheap next to
the spreading).  The arithmetic stays in libfirm.so and in the collective.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import _lib as L


def allreduce_sums(ker_half: torch.Tensor, rhs: torch.Tensor, group=None):
    """Sums the partial Ker half box and A*b of every process in place (two all-reduces)."""
    dist.all_reduce(ker_half, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(rhs, op=dist.ReduceOp.SUM, group=group)


def sharded_kernel_backproject(rec, images, shifts, R, group_ids=None, M=None, pg=None):
    """FIRM steps 1-3 for this process's images, then the sums over all processes loaded
    into `rec` (a Reconstructor): afterwards rec.cg_solve solves the whole problem.
    Returns the summed (Ker half box, A*b) tensors on rec's device."""
    if rec.params.flags & L.FIRM_FLAG_FUSED:
        rec.kernel_backproject(images, shifts, R, group_ids, M=M)
    else:
        rec.kernel(R, group_ids, M=M)
        rec.backproject(images, shifts, R, group_ids, M=M)
    ker = torch.empty(rec.half_shape(), dtype=torch.float32, device=rec.device)
    rhs = torch.empty((rec.N,) * 3, dtype=torch.float32, device=rec.device)
    rec.copy_out(L.FIRM_OUT_KER, ker)
    rec.copy_out(L.FIRM_OUT_RHS, rhs)
    torch.cuda.current_stream(rec.device).synchronize()      # the collective runs on its own stream
    allreduce_sums(ker, rhs, pg)
    rec.load_sums(ker, rhs)
    return ker, rhs
