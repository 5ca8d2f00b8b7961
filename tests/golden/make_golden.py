"""Writes the stored expected values under tests/golden/ by calling only the oracle.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from workloads import sphere_32  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    g, (s,) = sphere_32()
    I, A = oracle.forward(s, g)
    I = I.reshape(g.det_ny, g.det_nx)
    rows = {
        "workload": "sphere r=12 in 32^3, delta=1e-3, beta=1e-4, wavelength 8, flat 64x64 detector to 30 deg",
        "writer": "tests/golden/make_golden.py (oracle only)",
        "central_row_v32": [float(x) for x in I[32]],
        "diagonal": [float(I[k, k]) for k in range(g.det_nx)],
        "total": float(I.sum()),
    }
    with open(os.path.join(HERE, "sphere_32_oracle.json"), "w") as f:
        json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
