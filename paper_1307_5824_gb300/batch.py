"""Batched FIRM: many independent reconstructions as one unit of work (argument
marshalling only; the execution plan -- worker streams, the persistent spreading
launch, graph capture and the tuner -- lives in libfirm.so, firm_batch_*)."""
from __future__ import annotations

import json
import os

import torch

from . import _lib as L
from .recon import Reconstructor


class BatchReconstructor:
    """A batch over existing Reconstructors (one plan each, same W, same device)."""

    def __init__(self, recs: list[Reconstructor], n_streams: int = 8, device="cuda:0", stream=None):
        self.recs = list(recs)
        self.device = torch.device(device)
        n = len(self.recs)
        self.ws_bytes = L.firm_batch_workspace_size(n)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
            base = (self.workspace.data_ptr() + 255) // 256 * 256
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.batch = L.firm_batch_create([r.plan for r in self.recs], n_streams, base, self.ws_bytes,
                                             self.stream.cuda_stream)
        self._items = None
        self._keep = None

    def set_items(self, items: list[dict]):
        """items[i]: dict(M, R, images, x, group=None, shifts=None) of device tensors for
        recs[i].  The tensors must stay alive (and at the same addresses) while used."""
        self._keep = items
        self._items = L.make_batch_items(items)

    def run(self, iters: int, graph: bool = True, persistent: bool = True):
        flags = (L.FIRM_BATCH_GRAPH if graph else 0) | (L.FIRM_BATCH_PERSISTENT if persistent else 0)
        L.firm_batch_run(self.batch, self._items, iters, flags)

    def solve(self, max_iter: int, rel_tol: float, graph: bool = True, persistent: bool = True,
              learned: bool = False):
        """Every reconstruction to rel_tol (or max_iter) with its plan's preconditioner, or
        with the batch's network (set_network) when learned; returns when all are done."""
        flags = ((L.FIRM_BATCH_GRAPH if graph else 0) | (L.FIRM_BATCH_PERSISTENT if persistent else 0) |
                 (L.FIRM_BATCH_LEARNED if learned else 0))
        L.firm_batch_solve(self.batch, self._items, max_iter, rel_tol, flags)

    def set_network(self, params: torch.Tensor):
        """The learned preconditioner's network (FP32 parameters on the device) for
        solve(learned=True); its BF16 copy is made here, on the batch's stream."""
        self._net = params
        self._net_bf16 = torch.empty(params.numel(), dtype=torch.bfloat16, device=params.device)
        L.firm_mlp_to_bf16(params, self._net_bf16, self.stream.cuda_stream)
        L.firm_batch_set_network(self.batch, self._net_bf16, self._net)

    def wait(self, allow=()):
        return L.firm_batch_wait(self.batch, len(self.recs), allow)

    def tune(self, iters: int, graph: bool = True, persistent: bool = True, cache_path: str | None = None) -> dict:
        """Chooses the worker-stream count and the spreading work-item size by timing the
        candidates on the current items; with cache_path, a previous choice for the same
        device and the same (N, M) list is reused instead."""
        flags = (L.FIRM_BATCH_GRAPH if graph else 0) | (L.FIRM_BATCH_PERSISTENT if persistent else 0)
        key = "%s|%s|%d|%d" % (torch.cuda.get_device_name(self.device),
                               ",".join("%dx%d" % (r.N, it["M"]) for r, it in zip(self.recs, self._keep)),
                               iters, flags)
        cache = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
        if key in cache:
            c = cache[key]
            L.firm_batch_set_config(self.batch, c["n_streams"], c["chunk"])
            return dict(c, cached=True)
        ms = L.firm_batch_tune(self.batch, self._items, iters, flags)
        ns, ch = L.firm_batch_get_config(self.batch)
        c = {"n_streams": ns, "chunk": ch, "ms": ms}
        if cache_path:
            cache[key] = c
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        return dict(c, cached=False)

    def config(self):
        return L.firm_batch_get_config(self.batch)

    def set_config(self, n_streams: int, chunk: int):
        L.firm_batch_set_config(self.batch, n_streams, chunk)

    def launch_count(self) -> int:
        return L.firm_batch_launch_count(self.batch)

    def close(self):
        if getattr(self, "batch", None):
            L.firm_batch_destroy(self.batch)
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
