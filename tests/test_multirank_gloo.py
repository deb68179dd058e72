"""Two CPU ranks (gloo): Ker and A*b are sums over images (eq. kernel, eq. backprojection,
Section 3.4), so splitting the images across ranks and adding the ranks' partial sums
with one all-reduce gives the single-process result.  The all-reduce is the product's
own exchange step (paper_1307_5824_gb300.shard.allreduce_sums) applied to the oracle's
per-rank sums; tests/test_gpu_abi.py loads such sums into a plan (firm_load_sums).  The
benchmark's multi-GPU mode runs replicas and reduces only its timings, which the test
also checks (max over ranks)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp

import oracle as O
import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        inp = synth.config_inputs("C2", M=24, N=8)
        N, M = inp["N"], inp["M"]
        K = O.disc(N)
        h = O.ctf_weights(N, K, inp["groups"], inp["group_id"])
        a, b = rank * M // world, (rank + 1) * M // world
        ker = O.kernel(inp["R"][a:b], h[a:b], K, N).real
        rhs = O.backproject(inp["images"][a:b].astype(np.float64), inp["shifts"][a:b], inp["R"][a:b], h[a:b], K)
        # the product's exchange step (paper_1307_5824_gb300.shard), on CPU tensors
        from paper_1307_5824_gb300 import shard
        kt, rt = torch.from_numpy(ker.copy()), torch.from_numpy(rhs.copy())
        shard.allreduce_sums(kt, rt)
        t = torch.cat([kt.reshape(-1), rt.reshape(-1)])
        # timing reduction of the benchmark: max over ranks, whole job = world reconstructions
        import bench
        slow, per_recon = bench.job_time([10.0 + rank, 30.0 - rank], world, "cpu")
        if rank == 0:
            np.savez(out_path, sums=t.numpy(), ms=np.array(slow), per=np.array(per_recon))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_image_shards_add_up_over_gloo_ranks(tmp_path, world):
    out = str(tmp_path / "sums.npz")
    tmp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    got = np.load(out)
    inp = synth.config_inputs("C2", M=24, N=8)
    N = inp["N"]
    K = O.disc(N)
    h = O.ctf_weights(N, K, inp["groups"], inp["group_id"])
    ker = O.kernel(inp["R"], h, K, N).real
    rhs = O.backproject(inp["images"].astype(np.float64), inp["shifts"], inp["R"], h, K)
    ref = np.concatenate([ker.ravel(), rhs.ravel()])
    assert np.linalg.norm(got["sums"] - ref) <= 1e-12 * np.linalg.norm(ref)
    assert list(got["ms"]) == [10.0 + world - 1, 30.0]
    assert list(got["per"]) == [(10.0 + world - 1) / world, 30.0 / world]
