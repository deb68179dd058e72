"""Benchmark of the FIRM hot path on GB300.

One step = one whole reconstruction of the N=128, 50,000-image workload (FIRM steps
1-4: image DFTs, spreading into A*b and the Toeplitz kernel, fine-grid transforms,
circulant K-hat, CG to relative residual 1e-4) with the inputs already resident in
HBM.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl firm|reference]

Under torchrun (N > 1) every rank reconstructs its own copy of the workload
(replicas only: FIRM's per-image sums would need one all-reduce of Ker and A*b to
shard a single reconstruction, and no call here uses more than one GPU); the
timed region is bracketed by barriers, and `value` is the slowest rank's step time
divided by the number of ranks (whole-job seconds per reconstruction).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spread Gpts/s + s/recon (N=128, 50k imgs) vs plain CG on GB300 at rel-res 1e-4"
WORKLOAD = "C3"
REL_TOL = 1e-4
MAX_ITER = 5000


def job_time(local, world: int, dev):
    """Max over ranks of each per-rank time in `local`, and the same divided by world:
    every rank reconstructs once per step, so the whole job makes world
    reconstructions in the slowest rank's time (replicas, weak scaling)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(v) for v in local], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        local = [float(v) for v in t.tolist()]
    return list(local), [float(v) / world for v in local]


# Training set of the learned preconditioner per workload: (kernels, volume edge, most
# images per kernel).  All are kernels the method generates from random orientation
# mixtures, never the workload's own.  The 15-degree-cap workload trains at N=64 as its
# configuration states; for the N=128 Haar workload, N=96 kernels with up to 10,000
# images gave the table closest to its least-squares target (96 PCG iterations against
# 130 with the N=64 set, 103-107 with N=128 sets).
TRAIN_DEFAULTS = {"C3": (3000, 96, 10000), "C5": (2000, 64, 3000), "RCT": (3000, 96, 10000)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="firm", choices=["firm", "reference"])
    ap.add_argument("--images", type=int, default=None, help="override image count (smaller runs)")
    ap.add_argument("--N", type=int, default=None, help="override volume edge (profiling of smaller cases)")
    ap.add_argument("--max-iter", type=int, default=MAX_ITER, help="CG iteration cap (profiling)")
    ap.add_argument("--W", type=int, default=6)
    ap.add_argument("--precond", default="learned", choices=["none", "circulant", "binned", "learned", "physics"],
                    help="physics: the density-per-volume table alone (the learned network's baseline)")
    ap.add_argument("--residual", action="store_true",
                    help="learned: train on the target minus the density baseline (default: the raw table)")
    ap.add_argument("--no-compare", action="store_true", help="skip the plain-CG comparison run")
    ap.add_argument("--train-kernels", type=int, default=None,
                    help="kernels the learned preconditioner trains on (default per workload, see TRAIN_DEFAULTS)")
    ap.add_argument("--train-steps", type=int, default=3000, help="Adam steps of the learned preconditioner")
    ap.add_argument("--train-m-max", type=int, default=None, help="largest image count of a training kernel")
    ap.add_argument("--train-N", type=int, default=None, help="volume edge of the training kernels")
    ap.add_argument("--train-groups", type=int, default=4,
                    help="training kernels use 1..this many of the defocus values (max 20)")
    ap.add_argument("--train-defocus", type=int, default=8, help="defocus values (1.0-3.5 um) training draws from")
    ap.add_argument("--train-lr-final", type=float, default=None, help="final Adam step size (cosine decay from 1e-3)")
    ap.add_argument("--workload", default="C3", choices=["C3", "C5", "C4", "RCT"],
                    help="C3: 50k Haar views, 20 groups; C5: 40k views 85%% in a 15 degree cap, 8 groups; "
                         "C4: 64 independent reconstructions, N in {48,64,80,96}, 1k-8k images, 25 CG iterations; "
                         "RCT: random conical tilt (60 degrees), N=96, 10k images, SNR 1, with the FCR of the "
                         "solution inside and outside the missing cone")
    ap.add_argument("--batch", type=int, default=None, help="C4: reconstructions per batch (default 64)")
    ap.add_argument("--channels", default="fused", choices=["fused", "separate"],
                    help="separate: firm_kernel then firm_backproject (the image upload of the end-to-end step "
                         "hides behind the whole kernel channel); fused: one binning and one spreading pass for Ker "
                         "and A*b (firm_kernel_backproject; only the binning can hide the upload).  The other form "
                         "is timed beside it either way")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-c4", action="store_true", help="skip the batched (64-reconstruction) leg")
    ap.add_argument("--oracle-single", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--spread-only", action="store_true",
                    help="profiling: the separate channels (firm_kernel + firm_backproject) twice, then the fused "
                         "call twice, stage times printed; no benchmark line")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def workload(M_override=None, N_override=None, name=WORKLOAD):
    import synth
    inp = synth.config_inputs(name, M=M_override, N=N_override)
    return inp


def workload_name(inp, W, precond, name):
    """The workload as a sentence, from its configuration."""
    c, N, M = inp["cfg"], inp["N"], inp["M"]
    views = {"haar": "Haar views", "cap": "views 85% in a 15-degree cap", "mixed": "vMF/Haar views",
             "rct": "random conical tilt %g deg" % c.get("tilt_deg", 0.0)}[c["views"]]
    groups = "%d defocus groups" % len(c["defocus_um"]) if c["defocus_um"] else "no CTF"
    return ("N=%d volume, %d BF16 %dx%d images (%d-blob phantom, %s, %s, SNR %g), KB W=%d sigma=2, "
            "lambda=1e-3 x Ker(0), %s-preconditioned CG to rel-res 1e-4"
            % (N, M, N, N, c["n_blobs"], views, groups, c["snr"], W, precond))


def run_config(inp, args):
    """The `config` object of the benchmark line: the same for this arm and the
    reference arm (the oracle), which reconstructs the same workload."""
    N, M = inp["N"], inp["M"]
    fused = args.channels == "fused"
    return {"workload": workload_name(inp, args.W, args.precond, args.workload), "N": N, "M": M, "W": args.W,
            "precond": args.precond, "channels": args.channels,
            "l2": "inputs larger than L2: %.2f GB BF16 images read and %.2f GB of FP64 fine grids written every "
                  "step" % (M * N * N * 2 / 1e9, (3 if fused else 1) * (4 * N) ** 3 * 8 / 1e9)}


def disc_size(N):
    h = N // 2
    k = np.arange(-h, h + 1)
    return int(((k[:, None] ** 2 + k[None, :] ** 2) <= h * h).sum())


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample, scaled to one reconstruction)
# ---------------------------------------------------------------------------
ORACLE_SAMPLE_IMAGES = 2000     # images spread per sample (4% of the N=128 workload)
ORACLE_CG_TIMED = 2             # CG iterations run per sample (scaled to the count)


def oracle_cg_iterations(workload_name: str):
    """The oracle's own plain-CG iteration count to rel-res 1e-4 on this workload
    (oracle/cg_iterations.json, written by oracle/cg_iterations.py), or None."""
    try:
        return int(json.load(open(os.path.join(ROOT, "oracle", "cg_iterations.json")))[workload_name]["cg_iters"])
    except Exception:
        return None


def oracle_sample(inp, cg_iters: int, sample_images: int = ORACLE_SAMPLE_IMAGES, threads=None,
                  cg_timed: int = ORACLE_CG_TIMED):
    """The FP64 oracle as it stands (oracle/recon.py: gridding NUFFT with the workload's
    Kaiser-Bessel W=6, numpy/scipy transforms, textbook CG) on a bounded sample of the
    workload: the spreading of `sample_images` images, scaled to all M (it is linear in
    the images), the whole fine-grid transforms and K-hat, and `cg_timed` CG iterations
    scaled to `cg_iters`.  Returns (seconds per reconstruction, sample sentence, parts)."""
    from oracle import recon
    _, secs, parts, n_it = recon.reconstruct(inp, iters=max(int(cg_iters), 1), W=6, window="kb", threads=threads,
                                             sample_images=sample_images, cg_iters_timed=cg_timed)
    Ms = parts["images_spread"]
    sample = (f"FP64 oracle (gridding NUFFT, Kaiser-Bessel W=6, scipy FFTs, plain CG): spreading of {Ms} of "
              f"{inp['M']} images scaled to all, full fine-grid transforms and K-hat, {cg_timed} CG iterations "
              f"scaled to {n_it}")
    return secs, sample, {k: round(v, 4) for k, v in parts.items()}


def _oracle_single_core(name: str):
    """Child process: the oracle pinned to one host core on a small workload (the paper's
    own timings are single-core, Section 4): C1 in full, C2 with its spreading sampled."""
    os.sched_setaffinity(0, {sorted(os.sched_getaffinity(0))[0]})
    import synth
    from oracle import firm as OF
    OF.FFT_WORKERS = 1
    inp = synth.config_inputs(name)
    it = int(inp["cfg"]["iters"])
    sample = None if name == "C1" else 1000
    secs, text, parts = oracle_sample(inp, it, sample_images=sample or inp["M"], threads=1,
                                      cg_timed=it if name == "C1" else 3)
    print(json.dumps({"workload": name, "s_per_recon": secs, "sample": text, "parts": parts}))


def oracle_single_core_times():
    """C1 and C2 single-core oracle times, each in a child process pinned to one core."""
    out = {}
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    for name in ("C1", "C2"):
        try:
            r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-single", name],
                               capture_output=True, text=True, env=env, timeout=300)
            out[name] = json.loads(r.stdout.strip().splitlines()[-1])
        except Exception as ex:                     # reported, never fatal to the benchmark
            out[name] = {"error": str(ex)[:200]}
    return out


def host_cpu_model():
    try:
        for line in subprocess.run(["lscpu"], capture_output=True, text=True).stdout.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def cufft_comparison(rec, N, dev, stream, ours_apply_us, ours_fft_ker_ms):
    """cuFFT (through torch.fft, FP32), timed only as a comparison with the hand-written
    transforms: (a) the Toeplitz apply y = crop(IFFT(K-hat FFT(pad x))) + lam_eff x on
    the plan's K-hat, (b) a real-to-complex 3-D FFT of a (4N)^3 FP32 grid, the size of
    the kernel channel's fine grid (the hand-written pass reads the FP64 grid and prunes
    its output to the modes kept).  CUDA events on the current stream."""
    import torch
    from paper_1307_5824_gb300 import _lib as L
    L2 = 2 * N
    kh = torch.empty((L2, L2, N + 1), dtype=torch.float32, device=dev)
    rec.copy_out(L.FIRM_OUT_KHAT, kh)
    lam = rec.lambda_eff()
    x = torch.randn((N, N, N), device=dev)
    pad = torch.zeros((L2, L2, L2), device=dev)

    def apply():
        pad[:N, :N, :N] = x
        return torch.fft.irfftn(torch.fft.rfftn(pad) * kh, s=(L2, L2, L2))[:N, :N, :N] + lam * x

    y_ours = torch.empty_like(x)
    rec.toeplitz_apply(x, y_ours)
    y = apply()
    torch.cuda.synchronize(dev)
    agree = float(torch.linalg.vector_norm(y - y_ours) / torch.linalg.vector_norm(y_ours))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        apply()
    e0.record(stream)
    for _ in range(20):
        apply()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_apply = e0.elapsed_time(e1) / 20 * 1e3
    del pad, y
    g = torch.randn((4 * N,) * 3, device=dev)
    for _ in range(2):
        torch.fft.rfftn(g)
    e0.record(stream)
    for _ in range(5):
        torch.fft.rfftn(g)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_fine = e0.elapsed_time(e1) / 5
    del g
    torch.cuda.empty_cache()
    return {"library": "cuFFT via torch.fft (FP32)",
            "toeplitz_apply_us": t_apply, "hand_written_toeplitz_apply_us": ours_apply_us,
            "toeplitz_rel_diff_vs_hand_written": agree,
            "fine_grid_r2c_%d_cubed_ms" % (4 * N): t_fine, "hand_written_fine_grid_ms": ours_fft_ker_ms}


def cores_used():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


# ---------------------------------------------------------------------------
# reference arm: the oracle, timed step by step on bounded samples
# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    name = args.workload if args.workload != "C4" else "C3"
    inp = workload(args.images, args.N, name)
    iters = oracle_cg_iterations(name) or 272
    src = "the oracle's own count (oracle/cg_iterations.json)" if oracle_cg_iterations(name) else "assumed"
    # warm-up: the fixed parts (fine-grid transforms, K-hat, CG iterations) once; every
    # timed step then spreads a fresh slice of images (linear in the images)
    Ms = 500
    _, _, fixed = oracle_sample(inp, iters, sample_images=Ms, cg_timed=1)
    from oracle import gridding as Gr
    from oracle import firm as OF
    K = OF.disc(inp["N"])
    table_g = inp["groups"]
    vals = []
    t_all = None
    n_warm = max(0, args.warmup - 1)
    for step in range(n_warm + max(1, args.steps)):
        if step == n_warm:
            vals, t_all = [], time.perf_counter()
        a = (step * Ms) % max(1, inp["M"] - Ms)
        sub = dict(R=inp["R"][a:a + Ms], gid=inp["group_id"][a:a + Ms])
        tk, tb = {}, {}
        Gr.kernel_gridded(sub["R"], table_g, sub["gid"], K, inp["N"], W=6, window="kb", spread_only=True, timing=tk)
        Gr.backproject_gridded(inp["images"][a:a + Ms], inp["shifts"][a:a + Ms], sub["R"], table_g, sub["gid"], K,
                               W=6, window="kb", spread_only=True, timing=tb)
        per_image = (tk["spread_s"] + tb["spread_s"]) / Ms
        est = per_image * inp["M"] + fixed["transform_ker_s"] + fixed["transform_rhs_s"] + fixed["khat_s"] + \
            fixed["cg_s_per_iter"] * iters
        vals.append(est)
    wall = time.perf_counter() - t_all
    v = float(np.mean(vals))
    sample = (f"FP64 oracle (gridding NUFFT, Kaiser-Bessel W=6, scipy FFTs, plain CG): per step the spreading of "
              f"{Ms} of {inp['M']} images (both channels, a different slice each step) scaled to all; fine-grid "
              f"transforms, K-hat and one CG iteration timed once in the warm-up; {iters} CG iterations ({src})")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s/recon", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / max(1, args.steps) * 1e3,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           # the workload this arm reconstructs is the GPU arm's (its line carries the same
           # config); how the oracle reconstructs it (plain CG, FP64) is in cpu_baseline.sample
           "config": run_config(inp, args),
           "cpu_baseline": {"value": v, "unit": "s/recon", "cores": cores_used(), "kind": "oracle",
                            "sample": sample, "cpu_model": host_cpu_model(), "parts_fixed": fixed},
           "e2e": {"value": v, "unit": "s/recon", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ---------------------------------------------------------------------------
# the batched form (64 reconstructions per step)
# ---------------------------------------------------------------------------
def run_batched(args):
    out = batched_result(args)
    if out is not None:
        print(json.dumps(out))


def batched_result(args):
    """The batched form (64 reconstructions of uneven size): its JSON record on rank 0,
    None on the other ranks."""
    import multiprocessing as mp

    import synth
    n = args.batch or synth.BATCH["n"]
    iters = synth.BATCH["iters"]
    t_syn = time.perf_counter()
    with mp.get_context("spawn").Pool(max(1, min(16, cores_used()))) as pool:
        probs = pool.map(synth.batch_inputs, range(n))
    t_syn = time.perf_counter() - t_syn
    import torch

    from paper_1307_5824_gb300 import BatchReconstructor, Reconstructor
    from paper_1307_5824_gb300 import _lib as L
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch.distributed as dist
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    recs, items, host = [], [], []
    for p in probs:
        recs.append(Reconstructor(p["N"], p["M"], groups=p["groups"], W=args.W, lam=synth.BATCH["lam"], device=dev))
        h = dict(R=torch.from_numpy(p["R"].reshape(p["M"], 9).copy()).pin_memory(),
                 group=torch.from_numpy(p["group_id"].copy()).pin_memory(),
                 images=torch.from_numpy(p["images"]).pin_memory(),
                 shifts=torch.from_numpy(p["shifts"].copy()).pin_memory(),
                 x=torch.empty((p["N"],) * 3, dtype=torch.float32).pin_memory())
        host.append(h)
        items.append(dict(M=p["M"], R=h["R"].to(dev), group=h["group"].to(dev), images=h["images"].to(dev),
                          shifts=h["shifts"].to(dev), x=torch.empty((p["N"],) * 3, dtype=torch.float32, device=dev)))
    for p in probs:
        del p["images"]
    B = BatchReconstructor(recs, n_streams=16, device=dev)
    B.set_items(items)
    tuned = B.tune(iters)
    for _ in range(max(3, args.warmup)):
        B.run(iters)
    B.wait()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            B.run(iters)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    st, sts, its = B.wait()
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    # the same batch without the graph, and as 64 single-plan reconstructions in a row
    B.run(iters, graph=False)
    B.wait()
    torch.cuda.synchronize(dev)
    e0.record(stream)
    B.run(iters, graph=False)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_nograph = e0.elapsed_time(e1)

    def sequential():
        for r, it in zip(recs, items):
            r.kernel(it["R"], it["group"], M=it["M"])
            r.backproject(it["images"], it["shifts"], it["R"], it["group"], M=it["M"])
            r.cg_solve(it["x"], iters)
    sequential()
    torch.cuda.synchronize(dev)
    e0.record(stream)
    sequential()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_seq = e0.elapsed_time(e1)
    # end to end: pinned host inputs in, volumes out, inside the timed region
    h2d = sum(h["R"].numel() * 8 + h["group"].numel() * 4 + h["images"].numel() * 4 + h["shifts"].numel() * 8
              for h in host)
    d2h = sum(h["x"].numel() * 4 for h in host)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for h, it in zip(host, items):
            for k in ("R", "group", "images", "shifts"):
                it[k].copy_(h[k], non_blocking=True)
        B.run(iters)
        for h, it in zip(host, items):
            h["x"].copy_(it["x"], non_blocking=True)
        torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t0) / args.steps
    # to relative residual 1e-4 (the learned preconditioner's target): the batch with the
    # network (one forward pass over all plans), the batch with plain CG, and plain FIRM
    # one reconstruction after another through the single-plan calls
    from paper_1307_5824_gb300 import learned
    t0 = time.perf_counter()
    X, T = learned.generate(1000, N=64, m_range=(500, 3000), device=dev)
    net, _ = learned.train(X, T, steps=2000, device=dev)
    t_train = time.perf_counter() - t0
    B.set_network(net)
    tol_runs = {}
    for name, is_learned in (("learned", True), ("plain", False)):
        for r in recs:
            r.set_precond(L.FIRM_PRECOND_NONE)
        B.solve(MAX_ITER, REL_TOL, learned=is_learned)
        B.wait(allow=(L.FIRM_ENOTCONV, L.FIRM_EBREAKDOWN))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        B.solve(MAX_ITER, REL_TOL, learned=is_learned)
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        st_b, sts_b, its_b = B.wait(allow=(L.FIRM_ENOTCONV, L.FIRM_EBREAKDOWN))
        bad = [(int(r.N), int(it["M"]), int(s_), int(i_)) for r, it, s_, i_ in zip(recs, items, sts_b, its_b) if s_ != 0]
        tol_runs[name] = {"s_per_batch": dt, "recon_per_s": n / dt, "cg_iters_total": int(its_b.sum()),
                          "cg_iters_median": int(np.median(its_b)), "all_converged": not bad,
                          "not_converged (N, M, status, iterations)": bad[:8]}

    def sequential_plain():
        its_ = []
        for r, it in zip(recs, items):
            r.set_precond(L.FIRM_PRECOND_NONE)
            r.kernel(it["R"], it["group"], M=it["M"])
            r.backproject(it["images"], it["shifts"], it["R"], it["group"], M=it["M"])
            its_.append(r.cg_solve(it["x"], MAX_ITER, rel_tol=REL_TOL, allow=(L.FIRM_ENOTCONV,))[1])
        return its_
    sequential_plain()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    its_seq = sequential_plain()
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    tol_runs["plain_single_plan_sequential"] = {"s_per_batch": dt, "recon_per_s": n / dt,
                                                "cg_iters_total": int(np.sum(its_seq))}
    tol_runs["learned_vs_plain_sequential_speedup"] = dt / tol_runs["learned"]["s_per_batch"]
    tol_runs["learned_vs_plain_batched_speedup"] = tol_runs["plain"]["s_per_batch"] / tol_runs["learned"]["s_per_batch"]
    tol_runs["network"] = {"kernels": 1000, "N": 64, "steps": 2000, "train_s": round(t_train, 1)}
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return None
    pts = sum(it["M"] * disc_size(r.N) for r, it in zip(recs, items))
    out = {"metric": "batched FIRM reconstructions/s (64 recon, N in {48,64,80,96}, 1k-8k images, 25 CG iterations)",
           "value": n * world / (ms / 1e3), "unit": "recon/s", "n_gpus": world, "steps": args.steps,
           "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "%d independent reconstructions: N uniform over {48,64,80,96}, M uniform in "
                                  "[1000,8000] float32 images, own 30-blob phantom each, views as the N=64 workload, "
                                  "1-4 defocus groups, SNR 0.1, lambda=1e-3 x Ker(0), 25 CG iterations; one CUDA "
                                  "graph per step, persistent spreading over all plans" % n,
                      "images_total": int(sum(it["M"] for it in items)), "points_total": int(pts), "W": args.W,
                      "l2": "inputs larger than L2 (%.1f GB of images read per step)" %
                            (sum(it["images"].numel() * 4 for it in items) / 1e9)},
           "tuned": tuned, "ms_no_graph": ms_nograph, "ms_sequential_single_plan": ms_seq,
           "speedup_vs_sequential": ms_seq / ms, "cg_status_ok": bool(st == 0),
           "to_rel_res_1e-4": tol_runs,
           "gpu_launches": int(B.launch_count() * args.steps),
           "e2e": {"value": n / e2e_s, "unit": "recon/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
           "clocks": clk.summary(), "synth_s": round(t_syn, 1)}
    B.close()
    for r in recs:
        r.close()
    if world > 1:
        dist.destroy_process_group()
    return out


# ---------------------------------------------------------------------------
# profiling driver: the spreading stages alone
# ---------------------------------------------------------------------------
def run_spread_only(args):
    import torch

    from paper_1307_5824_gb300 import Reconstructor
    from paper_1307_5824_gb300 import _lib as L
    inp = workload(args.images, args.N, args.workload)
    N, M = inp["N"], inp["M"]
    dev = torch.device("cuda")
    img = torch.from_numpy(inp["images"]).to(dev).to(torch.bfloat16)
    R = torch.from_numpy(inp["R"].reshape(M, 9).copy()).to(dev)
    g = torch.from_numpy(inp["group_id"]).to(dev)
    sh = torch.from_numpy(inp["shifts"]).to(dev)
    rec = Reconstructor(N, M, groups=inp["groups"], W=args.W, lam=1e-3, img_dtype=L.FIRM_IMG_BF16, fused=True)
    rec.set_timing(True)
    for form in ("separate", "separate", "fused", "fused"):
        if form == "fused":
            rec.kernel_backproject(img, sh, R, g)
        else:
            rec.kernel(R, g)
            rec.backproject(img, sh, R, g)
        torch.cuda.synchronize()
        print(form, {k: round(v, 3) for k, v in rec.stage_times().items() if k not in ("cg", "cg_iters")})
    rec.close()


# ---------------------------------------------------------------------------
# the CUDA arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    if args.oracle_single:
        return _oracle_single_core(args.oracle_single)
    tk, tn, tm = TRAIN_DEFAULTS.get(args.workload, (2000, 64, 3000))
    args.train_kernels = tk if args.train_kernels is None else args.train_kernels
    args.train_N = tn if args.train_N is None else args.train_N
    args.train_m_max = tm if args.train_m_max is None else args.train_m_max
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "C4":
        return run_batched(args)
    if args.spread_only:
        return run_spread_only(args)
    import torch
    import torch.distributed as dist

    from paper_1307_5824_gb300 import Reconstructor
    from paper_1307_5824_gb300 import _lib as L

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    t_syn = time.perf_counter()
    inp = workload(args.images, args.N, args.workload)
    t_syn = time.perf_counter() - t_syn
    N, M = inp["N"], inp["M"]
    nK = disc_size(N)

    R_h = torch.from_numpy(inp["R"].reshape(M, 9).copy()).pin_memory()
    g_h = torch.from_numpy(inp["group_id"].copy()).pin_memory()
    s_h = torch.from_numpy(inp["shifts"].copy()).pin_memory()
    img_h = torch.from_numpy(inp["images"]).to(torch.bfloat16).pin_memory()
    R = R_h.to(dev)
    gid = g_h.to(dev)
    sh = s_h.to(dev)
    img = img_h.to(dev)
    inp["images"] = inp["images"][:5000].copy()     # the CPU-baseline sample keeps a few

    fused = args.channels == "fused"
    rec = Reconstructor(N, M, groups=inp["groups"], W=args.W, lam=1e-3, img_dtype=L.FIRM_IMG_BF16, device=dev,
                        fused=True)
    pc_modes = {"none": L.FIRM_PRECOND_NONE, "circulant": L.FIRM_PRECOND_CIRCULANT,
                "binned": L.FIRM_PRECOND_BINNED, "learned": L.FIRM_PRECOND_TABLE}
    infer = None
    train_info = None
    if args.precond == "learned":
        from paper_1307_5824_gb300 import learned
        t0 = time.perf_counter()
        X, T = learned.generate(args.train_kernels, N=args.train_N, m_range=(500, args.train_m_max), device=dev,
                                defocus_um=np.linspace(1.0, 3.5, args.train_defocus), max_groups=args.train_groups,
                                residual=args.residual)
        t_gen = time.perf_counter() - t0
        net, hist = learned.train(X[: int(0.9 * len(X))], T[: int(0.9 * len(X))], steps=args.train_steps,
                                  lr_final=args.train_lr_final, device=dev)
        train_info = {"kernels": int(len(X)), "N": args.train_N, "m_max": args.train_m_max,
                      "steps": args.train_steps, "gen_s": round(t_gen, 1), "loss": hist,
                      "val_mse_bf16": learned.evaluate(net, X[int(0.9 * len(X)):], T[int(0.9 * len(X)):], bf16=True)}
        if not args.residual:
            infer = learned.DeviceInference(net)
    elif args.precond != "physics":
        rec.set_precond(pc_modes[args.precond])
    x = torch.empty((N, N, N), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    base_tab = np.empty(1024, np.float32)
    per_step_pc = {"on": True}          # the comparison run switches the per-step tables off
    mode = {"fused": fused}

    def step(R_, g_, s_, im_, x_):
        if mode["fused"]:
            rec.kernel_backproject(im_, s_, R_, g_)
        else:
            rec.kernel(R_, g_)
        if per_step_pc["on"] and infer is not None:
            infer.apply(rec)                           # on the device: no host round trip
        elif per_step_pc["on"] and args.precond == "learned":
            learned.apply_learned(rec, net, residual=True)
        elif per_step_pc["on"] and args.precond == "physics":
            rec.pc_baseline(base_tab)
            rec.set_precond_table(base_tab)
        if not mode["fused"]:
            rec.backproject(im_, s_, R_, g_)
        st, it = rec.cg_solve(x_, args.max_iter, rel_tol=REL_TOL, allow=(L.FIRM_ENOTCONV,))
        return st, it

    for _ in range(max(3, args.warmup)):
        st, iters = step(R, gid, sh, img, x)
    torch.cuda.synchronize(dev)
    if args.precond == "learned":
        # how far the network's table is from its own target for this workload's kernel
        xin = np.empty(1024, np.float32)
        rec.pc_net_input(xin)
        tab = learned.predict(net, xin[None], bf16=True)[0]
        tgt = np.empty(1024, np.float32)
        if args.residual:
            rec.pc_residual_target(tgt)
        else:
            rec.pc_target(tgt)
        train_info["table_vs_target_mse"] = float(((tab - tgt) ** 2).mean())

    def timed(n_steps, label="firm_step"):
        """n_steps steps between CUDA events on the plan's stream, stage events recorded
        (no extra host synchronisation); returns (ms per step, stage ms, iterations,
        launches, clocks)."""
        rec.set_timing(True)
        l0 = rec.launch_count()
        acc, its = {}, []
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(torch.cuda.current_device()) as clk:
            e0.record(stream)
            for _ in range(n_steps):
                torch.cuda.nvtx.range_push(label)          # lets a profiler select the timed steps
                _, it_ = step(R, gid, sh, img, x)
                torch.cuda.nvtx.range_pop()
                its.append(it_)
                for k, v in rec.stage_times().items():
                    acc[k] = acc.get(k, 0.0) + v
            e1.record(stream)
            torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        rec.set_timing(False)
        return (e0.elapsed_time(e1) / n_steps, {k: v / n_steps for k, v in acc.items()}, its,
                rec.launch_count() - l0, clk.summary())

    # timed region: device-resident inputs
    ms_total, stages, iters_list, launches, clocks = timed(args.steps)
    (ms_step,), (ms_per_recon,) = job_time([ms_total], world, dev)
    # the other channel form, same preconditioner, for comparison
    mode["fused"] = not fused
    for _ in range(2):
        step(R, gid, sh, img, x)
    ms_other, stages_other, _, _, _ = timed(max(2, min(args.steps, 5)), "firm_step_other_form")
    mode["fused"] = fused
    step(R, gid, sh, img, x)
    torch.cuda.synchronize(dev)

    # the true relative residual of the returned volume, ||A*b - (A*A + lam_eff) x|| / ||A*b||,
    # recomputed with one Toeplitz apply (the solve stops on the recurrence residual)
    y_true = torch.empty_like(x)
    rhs_true = torch.empty_like(x)
    rec.toeplitz_apply(x, y_true)
    rec.copy_out(L.FIRM_OUT_RHS, rhs_true)
    torch.cuda.synchronize(dev)
    rh = rhs_true.cpu().numpy().astype(np.float64)
    true_rel_res = float(np.linalg.norm(rh - y_true.cpu().numpy().astype(np.float64)) / np.linalg.norm(rh))

    # end-to-end through the C ABI with host (pinned) buffers, copies inside the region
    e2e = None
    if not args.no_e2e:
        x_h = torch.empty((N, N, N), dtype=torch.float32).pin_memory()

        # both channel forms, each with the upload staged ahead and in stream order,
        # alternating step by step (the same drift for all four); the staged upload
        # overlaps the binning (fused) or the whole kernel channel (separate)
        n_e2e = max(args.steps, 5)
        variants = [(f, staged) for f in (fused, not fused) for staged in (False, True)]
        res = {v: 0.0 for v in variants}
        for f, staged in variants:               # one untimed step of each
            mode["fused"] = f
            if staged:
                rec.stage_images(img_h)
            step(R_h, g_h, s_h, img_h, x_h)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        for _ in range(n_e2e):
            for f, staged in variants:
                mode["fused"] = f
                t0 = time.perf_counter()
                if staged:
                    rec.stage_images(img_h)
                step(R_h, g_h, s_h, img_h, x_h)
                torch.cuda.synchronize(dev)
                res[(f, staged)] += time.perf_counter() - t0
        mode["fused"] = fused
        _, times = job_time([res[v] / n_e2e for v in variants], world, dev)
        res = dict(zip(variants, times))
        h2d = R_h.numel() * 8 + g_h.numel() * 4 + s_h.numel() * 8 + img_h.numel() * 2
        # the user's call for host-resident inputs is the faster form with the upload staged
        best = min((fused, not fused), key=lambda f: res[(f, True)])
        name = lambda f: "fused" if f else "separate"
        e2e = {"value": res[(best, True)], "unit": "s/recon", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(x_h.numel() * 4), "form": name(best) + " channels",
               "upload": "staged ahead (firm_stage_images), overlapped with the binning" if best else
                         "staged ahead (firm_stage_images), overlapped with the kernel channel",
               "value_serial_upload": res[(best, False)],
               "by_form": {name(f) + ("_staged" if st else "_serial"): res[(f, st)] for f, st in variants}}

    # the same reconstruction with plain CG (the comparison the metric names)
    plain = None
    if not args.no_compare and args.precond != "none":
        per_step_pc["on"] = False
        rec.set_precond(L.FIRM_PRECOND_NONE)
        for _ in range(2):
            step(R, gid, sh, img, x)
        ms_plain, st_plain, it_plain, _, _ = timed(args.steps)
        plain = {"s_per_recon": ms_plain / 1e3, "cg_iters": int(np.median(it_plain)), "cg_ms": st_plain["cg"]}
        per_step_pc["on"] = True

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    iters = int(np.median(iters_list))
    pts = M * nK
    W = args.W
    nH = (nK + 1) // 2
    # Spreading time of this form (the fused pass is stage 1; the separate channels are
    # stages 1 and 6) and the roofline of the dominant kernel, the spreading pass.  Work
    # unit: one shared-memory atomic add: W^3 per half-disc point for the kernel channel,
    # 2 W^3 for A*b, 3 W^3 for the fused pass.  Peak: 152 SMs x 32 lanes x 2.07 GHz (one
    # warp-wide shared atomic per clock per SM) = 10.07e12 / s.
    spread_ms = stages["spread_ker"] + stages["spread_rhs"] + stages.get("gather_fused", 0.0)

    def roofline_of(st, is_fused):
        """Shared-atomic rate of the dominant spreading kernel of one channel form, with
        its DRAM bytes per launch from an ncu capture of this workload (committed with
        the hash of the spreading source it was taken on; null once that source changed)."""
        if is_fused:
            dom, atoms, kname = "spread_ker", M * nH * W ** 3 * 3, f"k_spread_fused<{W}>"
        else:
            dom = "spread_rhs" if st["spread_rhs"] >= st["spread_ker"] else "spread_ker"
            atoms = M * nH * W ** 3 * (2 if dom == "spread_rhs" else 1)
            kname = f"k_spread<{W},{'complex' if dom == 'spread_rhs' else 'real'}>"
        peak = 152 * 32 * 2.07e9
        achieved = atoms / (st[dom] * 1e-3)
        traffic = None
        prof = os.path.join(ROOT, "profiles", "spread_traffic.json")
        if os.path.exists(prof) and (N, M, W) == (128, 50000, 6):   # the figure is for this workload
            try:
                import hashlib
                rec_t = json.load(open(prof)).get(kname) or {}
                src = open(os.path.join(ROOT, "paper_1307_5824_gb300", "csrc", "spread.cu"), "rb").read()
                if rec_t.get("source_sha256") == hashlib.sha256(src).hexdigest():
                    traffic = rec_t.get("dram_bytes")
            except Exception:
                traffic = None
        return {"kernel": kname, "bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                "unit": "Tatomic/s", "frac": achieved / peak, "traffic": traffic,
                "peak_source": "derived: 152 SMs x 32 shared-atomic lanes/clk x 2.07 GHz"}

    roofline = roofline_of(stages, fused)
    roofline_other = roofline_of(stages_other, not fused)
    # the spreading pass against HBM (not its binding bound): algorithmic bytes = point ids
    # and weights read + the FP64 fine grids written once
    Gk, Gr = 4 * N, 2 * N
    if fused:   # the weight gather (ids, weights by id, weights in payload order) + the pass
        spread_bytes = M * nH * (4 + 8 + 8) + M * nH * (4 + 8) + 3 * Gk ** 3 * 8
    else:
        spread_bytes = M * nH * 4 + Gk ** 3 * 8 + M * nH * (4 + 8 + 2) + Gr ** 3 * 16
    hbm_peak = None
    try:
        hbm_peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
        hbm_src = "measured (MEASURED_PEAKS.json)"
    except Exception:
        hbm_peak, hbm_src = 6800.0, "fallback"
    # a7 alone: Toeplitz applies on device buffers, CUDA events on the plan's stream.
    # Algorithmic bytes of one apply (three passes; the x/y intermediate of each plane
    # stays on chip): x in + t2 out, t2 + K-hat -> t2 (z), t2 + x in -> y out, with
    # t2 = N x 2N x (N+1) complex64.
    T2 = N * 2 * N * (N + 1) * 8
    toep_bytes = (N ** 3 * 4 + T2) + (2 * T2 + 2 * N * 2 * N * (N + 1) * 4) + (T2 + 2 * N ** 3 * 4)
    xa = torch.randn((N, N, N), device=dev)
    ya = torch.empty_like(xa)
    for _ in range(3):
        rec.toeplitz_apply(xa, ya)
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_app = 50
    torch.cuda.synchronize(dev)
    t0e.record(stream)
    for _ in range(n_app):
        rec.toeplitz_apply(xa, ya)
    t1e.record(stream)
    torch.cuda.synchronize(dev)
    toep_s = t0e.elapsed_time(t1e) / 1e3 / n_app
    toeplitz = {"applies_per_s": 1.0 / toep_s, "us_per_apply": toep_s * 1e6, "algorithmic_bytes": toep_bytes,
                "achieved_gbs": toep_bytes / toep_s / 1e9, "hbm_peak_gbs": hbm_peak,
                "hbm_frac": toep_bytes / toep_s / 1e9 / hbm_peak, "peak_source": hbm_src}
    del xa, ya
    cufft = cufft_comparison(rec, N, dev, stream, toep_s * 1e6, stages.get("fft_ker", 0.0))
    spread_hbm = {"algorithmic_bytes": int(spread_bytes), "achieved_gbs": spread_bytes / (spread_ms * 1e-3) / 1e9,
                  "hbm_frac": spread_bytes / (spread_ms * 1e-3) / 1e9 / hbm_peak, "peak_source": hbm_src,
                  "note": "not the binding bound: the spreading is bound by shared-memory atomic issue"}

    # the forward projector A of the solution (type-2 NUFFT at every half-disc sample)
    # and the data term |b - A x|^2 / |b|^2, device buffers, CUDA events
    fwd_out = torch.empty((M, (nK + 1) // 2, 2), dtype=torch.float32, device=dev)
    rec.forward(x, R, gid, fwd_out)
    torch.cuda.synchronize(dev)
    t0e.record(stream)
    rec.forward(x, R, gid, fwd_out)
    t1e.record(stream)
    torch.cuda.synchronize(dev)
    fwd_s = t0e.elapsed_time(t1e) / 1e3
    t0r = time.perf_counter()
    res2, b2 = rec.data_residual(x, img, sh, R, gid)
    res_s = time.perf_counter() - t0r
    del fwd_out
    forward = {"ms": fwd_s * 1e3, "points": M * ((nK + 1) // 2), "gpts_per_s": M * ((nK + 1) // 2) / fwd_s / 1e9,
               "data_residual_ms": res_s * 1e3, "data_term_rel": res2 / b2}

    # the positivity-constrained solve (projected CG), capped at 200 applies: its rate
    # with the host's two scalar reads per step (A*b and K-hat of the last step)
    rec.backproject(img, sh, R, gid)
    xn = torch.empty_like(x)
    torch.cuda.synchronize(dev)
    t0n = time.perf_counter()
    st_n, its_n = rec.solve_nonneg(xn, 200, 1e-4, allow=(L.FIRM_ENOTCONV,))
    nn_s = time.perf_counter() - t0n
    nonneg = {"applies": its_n, "ms": nn_s * 1e3, "us_per_apply": nn_s / max(its_n, 1) * 1e6,
              "held_at_zero_frac": float((xn == 0).float().mean()), "converged": st_n == L.FIRM_OK}

    # random conical tilt: resolution of the solution against the phantom inside and
    # outside the missing cone (Section 4's modified FCR)
    fcr = None
    if args.workload == "RCT":
        import synth
        from paper_1307_5824_gb300 import metrics as Mt
        truth = synth.blob_volume(inp["blobs"], N)
        sol = x.cpu().numpy()
        cone = Mt.cone_mask(N, (0, 0, 1), 90.0 - inp["cfg"]["tilt_deg"])
        f_out, f_in = Mt.fsc(sol, truth, ~cone), Mt.fsc(sol, truth, cone)
        below = np.flatnonzero(f_out < 0.5)
        fcr = {"cone_half_angle_deg": 90.0 - inp["cfg"]["tilt_deg"],
               "outside": [round(float(v), 4) for v in f_out], "inside": [round(float(v), 4) for v in f_in],
               "first_shell_outside_below_0.5": int(below[0]) + 1 if below.size else None}

    cpu = None
    if not args.no_cpu and world == 1:                 # the oracle baseline: rank 0 at N=1 only
        it_o = oracle_cg_iterations(args.workload) or (plain["cg_iters"] if plain else iters)
        est, sample, parts = oracle_sample(inp, it_o)
        cpu = {"value": est, "unit": "s/recon", "cores": cores_used(), "kind": "oracle", "sample": sample,
               "parts": parts, "cpu_model": host_cpu_model(), "threads": "gridding: OpenMP over all cores; "
               "FFTs: scipy workers over all cores",
               "single_core": oracle_single_core_times()}

    out = {
        "metric": METRIC, "value": ms_per_recon / 1e3, "unit": "s/recon", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": run_config(inp, args),
        "channels": args.channels,
        "spread_gpts_per_s": pts / (spread_ms * 1e-3) / 1e9,
        "spread_points": pts,
        "spread_hbm": spread_hbm,
        ("s_per_recon_separate_channels" if fused else "s_per_recon_fused_channels"): ms_other / 1e3,
        ("stage_ms_separate_channels" if fused else "stage_ms_fused_channels"):
            {k: round(v, 4) for k, v in stages_other.items() if k != "cg_iters"},
        "cufft_comparison": cufft,
        "toeplitz_applies_per_s": toeplitz["applies_per_s"],
        "toeplitz": toeplitz,
        "forward_projector": forward,
        "nonneg_solve": nonneg,
        "fcr": fcr,
        "cg_iters_per_s": (iters / (stages["cg"] * 1e-3)) if stages.get("cg") else None,
        "cg_iters": iters,
        "true_rel_residual": true_rel_res,
        # with separate channels the kernel channel (binning and spreading of Ker, its
        # transform, K-hat) depends on the poses only: a one-time precompute for a fixed
        # pose set
        "s_per_recon_without_precompute": ((ms_other if fused else ms_per_recon) - sum(
            (stages_other if fused else stages).get(k, 0.0) for k in ("bin_ker", "spread_ker", "fft_ker", "khat")))
        / 1e3,
        "stage_ms": {k: round(v, 4) for k, v in stages.items() if k != "cg_iters"},
        "roofline": roofline,
        ("roofline_separate_channels" if fused else "roofline_fused_channels"): roofline_other,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "synth_s": round(t_syn, 1),
        "precond": args.precond,
        "learned_training": train_info,
        "plain_cg": plain,
    }
    # the batched form (64 reconstructions of uneven N and image count, one graph launch
    # per step; to rel-res 1e-4 with the batch's network) on the same GPU, after this
    # workload's buffers are released
    if world == 1 and args.workload == WORKLOAD and args.images is None and not (args.no_c4 or args.no_compare):
        rec.close()
        del img, img_h, R, R_h, x
        torch.cuda.synchronize(dev)
        torch.cuda.empty_cache()
        try:
            c4_args = argparse.Namespace(**vars(args))
            c4_args.steps, c4_args.warmup, c4_args.batch = 3, 3, None
            c4 = batched_result(c4_args)
            out["batched_c4"] = {k: c4[k] for k in ("metric", "value", "unit", "ms_per_step", "tuned", "ms_no_graph",
                                                    "ms_sequential_single_plan", "speedup_vs_sequential",
                                                    "cg_status_ok", "to_rel_res_1e-4", "e2e", "gpu_launches",
                                                    "clocks", "config")}
        except Exception as exc:                     # reported, never fatal to the main line
            out["batched_c4"] = {"error": f"{type(exc).__name__}: {exc}"}
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
