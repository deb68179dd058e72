"""Learned Fourier-domain CG preconditioner: training data from the method itself, training
and inference through the C ABI (firm_pc_features, firm_pc_target, firm_mlp_*).

Training set: kernels the method generates at N = 64 from random orientation mixtures
(Haar, von Mises--Fisher about 1-3 axes, polar caps), 500-3000 images, 1-4 of 8 defocus
groups; each sample is the per-bin density feature vector and the per-bin least-squares
target of the circulant preconditioner.  The network (1024 -> 256 -> 256 -> 1024) maps
log-density to the log table; the plan then uses exp(table) / Ker(0) as the Fourier
diagonal (FIRM_PRECOND_TABLE).  Python only marshals arguments and draws the seeded
random numbers (initial weights, mini-batch indices, orientations); every arithmetic
step runs in libfirm.so.
"""
from __future__ import annotations

import numpy as np
import torch

import synth

from . import _lib as L
from .recon import Reconstructor

NBINS = 1024
DEFOCUS_UM = np.linspace(1.0, 3.5, 8)


def random_rotations(M: int, rng: np.random.Generator) -> np.ndarray:
    """A random mixture of Haar, von Mises--Fisher and polar-cap view distributions."""
    kinds = rng.dirichlet(np.ones(3))
    n = (kinds * M).astype(int)
    n[0] += M - n.sum()
    parts = [synth.haar_rotations(n[0], rng)]
    if n[1] > 0:
        parts.append(synth.mixed_rotations(n[1], rng, frac_vmf=1.0, kappa=float(rng.uniform(5, 60)),
                                           n_axes=int(rng.integers(1, 4))))
    if n[2] > 0:
        pole = rng.standard_normal(3)
        parts.append(synth.cap_rotations(n[2], float(rng.uniform(10, 40)), pole, rng))
    R = np.concatenate(parts)
    return R[rng.permutation(M)]


def generate(n_kernels: int = 2000, N: int = 64, seed: int = 51, m_range=(500, 3000), device="cuda:0",
             defocus_um=DEFOCUS_UM, max_groups: int = 4, residual: bool = False):
    """(X, T): network inputs and targets of n_kernels method-generated kernels; each
    kernel uses 1..max_groups of the defocus values.  With residual, T is the target
    minus the density-per-volume baseline (firm_pc_baseline), for a network that learns
    only the correction (an option: the baseline is extreme in bins with few grid
    frequencies, and the raw table trains better)."""
    rng = np.random.default_rng(seed)
    defocus_um = np.asarray(defocus_um, float)
    groups = synth.ctf_group_table(defocus_um)
    rec = Reconstructor(N, m_range[1], groups=groups, W=6, lam=1e-3, device=device)
    X = np.empty((n_kernels, NBINS), np.float32)
    T = np.empty((n_kernels, NBINS), np.float32)
    t = np.empty(NBINS, np.float32)
    for i in range(n_kernels):
        M = int(rng.integers(m_range[0], m_range[1] + 1))
        R = random_rotations(M, rng)
        sub = rng.choice(len(defocus_um), int(rng.integers(1, min(max_groups, len(defocus_um)) + 1)), replace=False)
        gid = sub[rng.integers(0, len(sub), M)].astype(np.int32)
        rec.kernel(np.ascontiguousarray(R.reshape(M, 9)), gid, M=M)
        rec.pc_net_input(X[i])
        if residual:
            rec.pc_residual_target(t)
        else:
            rec.pc_target(t)
        T[i] = t
    rec.close()
    return X, T


def init_params(seed: int = 52) -> np.ndarray:
    """He-normal weights, zero biases, in the firm_mlp parameter layout."""
    rng = np.random.default_rng(seed)
    w = (NBINS, 256, 256, NBINS)
    out = []
    for i in range(3):
        out.append((rng.standard_normal((w[i + 1], w[i])) * np.sqrt(2.0 / w[i])).astype(np.float32).ravel())
        out.append(np.zeros(w[i + 1], np.float32))
    p = np.concatenate(out)
    assert p.size == L.firm_mlp_param_count()
    return p


def train(X: np.ndarray, T: np.ndarray, steps: int = 3000, batch: int = 64, lr: float = 1e-3, seed: int = 53,
          device="cuda:0", log_every: int = 500, lr_final: float | None = None):
    """Adam on the mean squared error, the step size decayed from lr to lr_final on a
    half cosine (constant when lr_final is None); returns (params on the device, loss
    history)."""
    dev = torch.device(device)
    rng = np.random.default_rng(seed)
    params = torch.from_numpy(init_params(seed - 1)).to(dev)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    g = torch.empty_like(params)
    Xd = torch.from_numpy(X).to(dev)
    Td = torch.from_numpy(T).to(dev)
    work = torch.empty(L.firm_mlp_work_floats(batch), dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    s = torch.cuda.current_stream(dev).cuda_stream
    hist = []
    for step in range(1, steps + 1):
        idx = torch.from_numpy(rng.integers(0, X.shape[0], batch)).to(dev)
        xb = Xd.index_select(0, idx).contiguous()
        tb = Td.index_select(0, idx).contiguous()
        L.firm_mlp_grad(params, batch, xb, tb, g, work, loss, s)
        lr_t = lr if lr_final is None else lr_final + (lr - lr_final) * 0.5 * (1.0 + np.cos(np.pi * (step - 1) / steps))
        L.firm_mlp_adam(params, g, m, v, step, lr_t, s)
        if step % log_every == 0 or step == 1:
            hist.append((step, float(loss.item())))
    return params, hist


def evaluate(params: torch.Tensor, X: np.ndarray, T: np.ndarray, bf16: bool = False) -> float:
    """Mean squared error of the network on (X, T)."""
    y = predict(params, X, bf16=bf16)
    return float(((y - T) ** 2).mean())


def predict(params: torch.Tensor, X: np.ndarray, bf16: bool = True) -> np.ndarray:
    """Network output (log tables) for rows of X; BF16 weights by default (inference)."""
    dev = params.device
    n = X.shape[0]
    x = torch.from_numpy(np.ascontiguousarray(X, np.float32)).to(dev)
    y = torch.empty((n, NBINS), dtype=torch.float32, device=dev)
    work = torch.empty(L.firm_mlp_work_floats(n), dtype=torch.float32, device=dev)
    s = torch.cuda.current_stream(dev).cuda_stream
    if bf16:
        pb = torch.empty(params.numel(), dtype=torch.bfloat16, device=dev)
        L.firm_mlp_to_bf16(params, pb, s)
        L.firm_mlp_forward_bf16(pb, params, n, x, y, work, s)
    else:
        L.firm_mlp_forward(params, n, x, y, work, s)
    torch.cuda.synchronize(dev)
    return y.cpu().numpy()


def apply_learned(rec: Reconstructor, params: torch.Tensor, bf16: bool = True, residual: bool = False) -> np.ndarray:
    """Features of the plan's last kernel -> network (+ the density baseline when the
    network was trained on residuals) -> FIRM_PRECOND_TABLE.  Returns the table."""
    x = np.empty(NBINS, np.float32)
    rec.pc_net_input(x)
    out = predict(params, x[None], bf16=bf16)[0]
    if residual:
        rec.set_precond_residual(np.ascontiguousarray(out))
    else:
        rec.set_precond_table(np.ascontiguousarray(out))
    return out


class DeviceInference:
    """The trained network applied to a plan without leaving the device: the features'
    network input (firm_pc_net_input), the BF16 forward pass (firm_mlp_forward_bf16) and
    the table (firm_set_precond_table) all read and write device buffers on the plan's
    stream, so a reconstruction step never waits for the host."""

    def __init__(self, params: torch.Tensor):
        dev = params.device
        self.params = params
        self.pb = torch.empty(params.numel(), dtype=torch.bfloat16, device=dev)
        self.x = torch.empty((1, NBINS), dtype=torch.float32, device=dev)
        self.y = torch.empty((1, NBINS), dtype=torch.float32, device=dev)
        self.work = torch.empty(L.firm_mlp_work_floats(1), dtype=torch.float32, device=dev)
        L.firm_mlp_to_bf16(params, self.pb, torch.cuda.current_stream(dev).cuda_stream)

    def apply(self, rec: Reconstructor):
        s = rec.stream.cuda_stream
        rec.pc_net_input(self.x)
        L.firm_mlp_forward_bf16(self.pb, self.params, 1, self.x, self.y, self.work, s)
        rec.set_precond_table(self.y)

