"""Write the oracle's semi-axis history of the oscillating elliptical drop
(Section 5.2; [-2,2]^2, g = 0, k0 = 2.25e9, CFL 0.9) to a text fixture.

The stored values are the FP64 oracle's alone: this script calls only
`oracle/` (and the input generator `cases.drop`), never the CUDA library.

    python tests/golden/make_drop_history.py N STEPS EVERY OUT

writes, every EVERY steps, the step, the simulated time t and the semi-axes
a (x) and b (y) from the alpha = 0.5 crossings on the positive axes (linear
interpolation between the two cells next to the axis), plus the wall time.
"""
from __future__ import annotations

import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import oracle  # noqa: E402
from paper_1806_04960_gb300 import cases  # noqa: E402


def semi_axes(c, q):
    """Semi-axes (a, b) from the alpha = 0.5 crossings on the positive x and y
    axes of the n x n drop grid (n even: the axes run between two cells)."""
    n = c.nx
    col = 0.5 * (q[3][:, n // 2 - 1] + q[3][:, n // 2])
    row = 0.5 * (q[3][n // 2 - 1, :] + q[3][n // 2, :])
    y, x = c.yc(), c.xc()
    up = np.flatnonzero((y[:-1] > 0) & (col[:-1] >= 0.5) & (col[1:] < 0.5))[0]
    rt = np.flatnonzero((x[:-1] > 0) & (row[:-1] >= 0.5) & (row[1:] < 0.5))[0]
    a = x[rt] + (row[rt] - 0.5) / (row[rt] - row[rt + 1]) * c.dx
    b = y[up] + (col[up] - 0.5) / (col[up] - col[up + 1]) * c.dy
    return float(a), float(b)


def main(argv):
    n, steps, every, out = int(argv[1]), int(argv[2]), int(argv[3]), argv[4]
    c = cases.drop(n)
    q, t = c.q, 0.0
    t0 = time.perf_counter()
    rows = []
    for k in range(steps // every):
        q, tt, _, _ = oracle.run(c, every, q=q)
        t += tt
        a, b = semi_axes(c, q)
        rows.append(((k + 1) * every, t, a, b))
        print(rows[-1], f"{time.perf_counter() - t0:.0f} s", flush=True)
    with open(out, "w") as f:
        f.write("# Oscillating elliptical drop (Section 5.2), FP64 oracle, written by\n")
        f.write(f"# tests/golden/make_drop_history.py {n} {steps} {every} <out>\n")
        f.write(f"# grid {n} x {n} on [-2,2]^2, g = 0, k0 = 2.25e9, CFL {c.cfl}; "
                f"{oracle.max_threads()} threads, {time.perf_counter() - t0:.0f} s\n")
        f.write("# columns: step  t  a  b  (alpha = 0.5 crossings on the positive axes)\n")
        for s, tt, a, b in rows:
            f.write(f"{s} {tt!r} {a!r} {b!r}\n")


if __name__ == "__main__":
    main(sys.argv)
