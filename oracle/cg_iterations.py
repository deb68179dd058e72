"""Writes oracle/cg_iterations.json: the FP64 oracle's own plain-CG iteration count to
relative residual 1e-4 (Section 3.3; reading 8, the recurrence residual) on the N=128,
50,000-image workload, with the workload's Kaiser-Bessel W=6 NUFFT (oracle/recon.py).

Test infrastructure: the benchmark's reference arm reads the count, so that its bounded
samples scale to the number of iterations the oracle itself needs (running them costs
minutes).  Calls only oracle/ and the seeded input generator.

    python oracle/cg_iterations.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    import numpy as np

    import synth
    from oracle import recon

    out = {}
    for name in ("C3",):
        inp = synth.config_inputs(name)
        # the images as the GPU path reads them: BF16-rounded (round to nearest even)
        u = inp["images"].astype(np.float32).view(np.uint32)
        u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
        images = u.view(np.float32)
        t0 = time.perf_counter()
        _, secs, parts, it = recon.reconstruct(inp, rel_tol=1e-4, images=images)
        out[name] = {"cg_iters": int(it), "rel_tol": 1e-4, "W": 6, "window": "kb", "seconds": round(secs, 1),
                     "wall_s": round(time.perf_counter() - t0, 1),
                     "parts": {k: round(v, 3) for k, v in parts.items()}}
        print(name, out[name], flush=True)
    path = os.path.join(ROOT, "oracle", "cg_iterations.json")
    json.dump(out, open(path, "w"), indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
