"""Writes tests/golden/star_pyramid80_extended.txt: the FP64 march of the
80-triangle star-based pyramid (Section VI-A, third scatterer: stand-in
geometry of paper_2510_07989_gb300.inputs.meshes.star_pyramid, m = 2;
eps_r = 5, c dt = 0.2, one plane wave with w = 30 c dt, t0 = 60 dt, r_obj = 1)
evaluated by the oracle in extended precision (oracle.extended), sampled.

On this mesh the march magnifies operator-level rounding: FP64 evaluations of
the same definition differ from one machine's linear algebra to another's by
up to ~2e-7 of the peak, so the stored extended-precision values are the
reference. Calls only oracle/ and the seeded input generators.

    python tests/golden/make_star_pyramid80.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import extended as X  # noqa: E402
from paper_2510_07989_gb300.inputs import meshes as MS  # noqa: E402
from paper_2510_07989_gb300.inputs.assemble import assemble  # noqa: E402

N_STEPS = 120
STEPS = list(range(30, N_STEPS + 1, 3))     # sampled steps (1-based)
UNKNOWNS = list(range(0, 240, 6))          # sampled unknowns of [u; v] (2 N_e = 240)


def compute():
    ops = assemble(MS.star_pyramid(5, m=2), 5.0, 1.0, 0.2)
    exc = MS.single_wave(ops.dt, 30, 60, r_obj=1.0)
    W = X.ExtendedSystem(ops).march(exc, N_STEPS)
    return ops, W


def main():
    ops, W = compute()
    assert 2 * ops.ne == 240
    peak = float(np.abs(W).max())
    lines = [
        "# FP64 march of the 80-triangle star-based pyramid (Section VI-A, third",
        "# scatterer; stand-in geometry star_pyramid(5, m=2), eps_r = 5, c dt = 0.2,",
        "# one plane wave p = x, k = z, w = 30 c dt, t0 = 60 dt, r_obj = 1), evaluated",
        "# by oracle.extended (long double), written by tests/golden/make_star_pyramid80.py.",
        "# peak: the largest |w| over the whole run (steps 1..%d)." % N_STEPS,
        "# rows: step (1-based), unknown index of [u; v], value.",
        "peak %.17e" % peak,
    ]
    for i in STEPS:
        for j in UNKNOWNS:
            lines.append("w %d %d %.17e" % (i, j, float(W[i - 1, j])))
    with open(os.path.join(HERE, "star_pyramid80_extended.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
