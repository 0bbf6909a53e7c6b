"""Writes effective_friction_L16.txt: the oracle's g (Eq. (aeffcorr)) of the
settling test of Sec. 4.6 for phi_2, phi_3, phi_4 at five grid positions,
L = 16, 1500 steps, F = 1e-4, a0 = 1 (oracle.effective_friction defaults).
Calls only the oracle.  Run from the repository root:
    python tests/golden/make_effective_friction.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as ora  # noqa: E402

OFFSETS = [(0.0, 0.0, 0.0), (0.5, 0.0, 0.0), (0.5, 0.5, 0.0), (0.5, 0.5, 0.5), (0.2, 0.3, 0.4)]


def main():
    lines = ["# settling test of Sec. 4.6 by the FP64 oracle: L=16, 1500 steps, F=1e-4, a0=1, eta=1/6",
             "# kernel ox oy oz u0 g"]
    for k in (2, 3, 4):
        for off in OFFSETS:
            r = ora.effective_friction(k, off, L=16, steps=1500)
            lines.append("%d %.1f %.1f %.1f %.17g %.17g" % (k, off[0], off[1], off[2], r["u0"], r["g"]))
    with open(os.path.join(HERE, "effective_friction_L16.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
