"""Reader for the hand-derived tiling goldens (tiling_golden.txt)."""
import os
from collections import defaultdict

HERE = os.path.dirname(os.path.abspath(__file__))


def tiling_goldens():
    """{(W, H, N): [(row, y, h, n_C, [widths])...]}"""
    out = defaultdict(list)
    with open(os.path.join(HERE, "tiling_golden.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            a, b, c = line.split("|")
            W, H, N = map(int, a.split())
            row, y, h, nc = map(int, b.split())
            out[(W, H, N)].append((row, y, h, nc, list(map(int, c.split()))))
    return dict(out)
