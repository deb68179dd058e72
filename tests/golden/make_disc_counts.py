"""Write disc_counts.txt: |{k in Z^2 : |k| <= N/2}| counted row by row.

Each row k1 in [-h, h] of the disc holds 2*floor(sqrt(h^2 - k1^2)) + 1 lattice
points; the count uses integer square roots only, independent of the oracle."""
import math
import os

here = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(here, "disc_counts.txt"), "w") as f:
    f.write("# N  |K|  (eq. truncation, symmetric disc |k| <= N/2)\n")
    for N in (8, 16, 32, 48, 64, 80, 96, 128):
        h = N // 2
        cnt = sum(2 * math.isqrt(h * h - k1 * k1) + 1 for k1 in range(-h, h + 1))
        f.write(f"{N} {cnt}\n")
