"""A FIRM plan whose workspace is a torch CUDA tensor (argument marshalling only)."""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as L


class Reconstructor:
    """Owns one firm_plan: workspace from torch's caching allocator, stream = torch's
    current stream on `device`.  Methods forward to the C ABI of the same name."""

    def __init__(self, N: int, M: int, groups=None, W: int = 6, lam: float = 0.0,
                 lambda_mode: int = L.FIRM_LAMBDA_RELATIVE, img_dtype: int = L.FIRM_IMG_F32,
                 device="cuda:0", stream=None, flags: int = 0, fused: bool = False):
        if not torch.cuda.is_available():
            raise RuntimeError("the FIRM CUDA path needs a CUDA device")
        self.device = torch.device(device)
        table = np.zeros((0, 6)) if groups is None else np.asarray(groups, float).reshape(-1, 6)
        if fused:
            flags |= L.FIRM_FLAG_FUSED
        self.params = L.make_params(N, M, table.shape[0], W, 2.0, lam, lambda_mode, 0, img_dtype, flags)
        self._groups = L.make_groups(table)
        self.ws_bytes = L.firm_workspace_size(self.params)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            base = self.workspace.data_ptr()
            self._base = (base + 255) // 256 * 256
            self.plan = L.firm_plan(self.params, self._groups, self._base, self.ws_bytes, self.stream.cuda_stream)
        self.N, self.M = N, M

    # -- FIRM steps --------------------------------------------------------------
    def kernel(self, R, group=None, khat_out=None, M=None):
        L.firm_kernel(self.plan, self.M if M is None else M, R, group, khat_out)

    def backproject(self, images, shifts, R, group=None, rhs_out=None, M=None):
        L.firm_backproject(self.plan, self.M if M is None else M, images, shifts, R, group, rhs_out)

    def kernel_backproject(self, images, shifts, R, group=None, khat_out=None, rhs_out=None, M=None):
        """Steps 1-3 with both spreading channels in one pass (plans made with fused=True)."""
        L.firm_kernel_backproject(self.plan, self.M if M is None else M, images, shifts, R, group, khat_out, rhs_out)

    def load_sums(self, ker_half=None, rhs=None):
        """Ker half box and / or A*b summed elsewhere (image shards) -> K-hat, lam_eff."""
        L.firm_load_sums(self.plan, ker_half, rhs)

    def stage_images(self, images, M=None):
        """Starts the upload of host `images` (pinned, M x N x N) into a device buffer
        held by this object; the next backproject with the same tensor reads it."""
        M = self.M if M is None else M
        if getattr(self, "_staging", None) is None:     # sized once for the plan's M
            nbytes = max(self.M, 1) * self.N * self.N * images.element_size()
            self._staging = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        L.firm_stage_images(self.plan, M, images, self._staging, self._staging.numel())

    def forward(self, V, R, group=None, out=None, M=None):
        """(A V) on every image's half disc, M x |K|/2 complex64 (out: a device or host
        float32 array of shape (M, |K|/2, 2), allocated on the device when None)."""
        M = self.M if M is None else M
        if out is None:
            nH = (L.disc_size(self.N) + 1) // 2
            out = torch.empty((M, nH, 2), dtype=torch.float32, device=self.device)
        L.firm_forward(self.plan, M, V, R, group, out)
        return out

    def data_residual(self, V, images, shifts, R, group=None, M=None):
        """(sum |b - A V|^2, sum |b|^2) over every image's whole disc, FP64."""
        return L.firm_data_residual(self.plan, self.M if M is None else M, V, images, shifts, R, group)

    def cg_solve(self, x, max_iter, rel_tol=0.0, rhs=None, resid_hist=None, allow=()):
        return L.firm_cg_solve(self.plan, rhs, x, max_iter, rel_tol, resid_hist, allow)

    def toeplitz_apply(self, x, y):
        L.firm_toeplitz_apply(self.plan, x, y)

    def solve_nonneg(self, x, max_iter, rel_tol, allow=()):
        """V >= 0 minimiser of the data term (projected CG); returns (status, applies)."""
        return L.firm_solve_nonneg(self.plan, x, max_iter, rel_tol, allow)

    def set_damping(self, mu: float):
        """mu of the first-difference penalty mu ||D V||^2, from the next kernel() on."""
        L.firm_set_damping(self.plan, mu)

    def set_precond(self, mode: int):
        L.firm_set_precond(self.plan, mode)

    def set_precond_table(self, table_log):
        L.firm_set_precond_table(self.plan, table_log)

    def pc_features(self, out):
        L.firm_pc_features(self.plan, out)

    def pc_net_input(self, out):
        """The learned network's input, log(1024 f + 1e-3) of the features (on the device)."""
        L.firm_pc_net_input(self.plan, out)

    def pc_target(self, out):
        L.firm_pc_target(self.plan, out)

    def pc_residual_target(self, out):
        L.firm_pc_residual_target(self.plan, out)

    def set_precond_residual(self, delta):
        L.firm_set_precond_residual(self.plan, delta)

    def pc_baseline(self, out):
        L.firm_pc_baseline(self.plan, out)

    def pc_bin_volumes(self, out):
        L.firm_pc_bin_volumes(self.plan, out)

    def pc_axis(self):
        return L.firm_pc_axis(self.plan)

    def lambda_eff(self) -> float:
        return L.firm_lambda_eff(self.plan)

    def copy_out(self, which, dst):
        L.firm_copy_out(self.plan, which, dst)

    def set_timing(self, on=True):
        L.firm_set_timing(self.plan, on)

    def stage_times(self):
        return L.firm_stage_times(self.plan)

    def launch_count(self) -> int:
        return L.firm_launch_count(self.plan)

    # -- buffers ---------------------------------------------------------------------
    def half_shape(self):
        return (2 * self.N, 2 * self.N, self.N + 1)

    def close(self):
        if getattr(self, "plan", None):
            L.firm_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
