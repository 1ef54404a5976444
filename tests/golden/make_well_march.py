"""Writes well_march_10x40.json: the FP64 oracle's time march of a reduced
horizontal-well instance (paper Sec. 5 example, geometry of the
multi-stage configuration scaled down): 10 parallel fractures at 20 m
spacing, half-length 100 m, 40 constant elements each; RATE system (rows
sigma_s and sigma_n + p, the fluid source prescribed by the injection of
0.01 m^3/s per fracture over a 100 m fracture height, split uniformly
along the fracture); Table 2 stresses and initial pore
pressure; 100 time steps of 60 s, the history of all previous steps
subtracted at every step (oracle.march: dense matrices, direct solves).

Calls only oracle/ and the seeded input generators.  Run from the
repository root:  python tests/golden/make_well_march.py   (about 10 min on
8 cores)."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1812_05087_gb300 import inputs  # noqa: E402

N_FRAC, ELEMS, STEPS = 10, 40, 100
KEEP_D = (1, 10, 100)
KEEP_K = (1, 2, 5, 10, 20, 30, 40, 50, 60, 70, 80, 90, 100)


def main():
    mat = inputs.material_tuple()
    xy, segs = inputs.parallel_fractures(n_frac=N_FRAC, spacing=20.0, half_length=100.0, elems=ELEMS)
    N = xy.shape[1]
    tips = inputs.tips_of(segs)
    b = oracle.rhs(xy, system="rate", **inputs.WELL_LOADS)
    dq = np.full(N, inputs.well_source(100.0))
    times = inputs.WELL_DT * np.arange(STEPS + 1)
    sols = oracle.march(mat, xy, times, [b] * STEPS, system="rate", Dq_steps=[dq] * STEPS)
    out = {
        "source": "oracle.march (FP64 dense, direct solves) of the reduced horizontal-well instance; "
                  "paper Sec. 5 example, Table 2 loads; written by tests/golden/make_well_march.py",
        "n_frac": N_FRAC, "elems": ELEMS, "spacing": 20.0, "half_length": 100.0, "dt": inputs.WELL_DT,
        "steps": STEPS, "loads": inputs.WELL_LOADS, "injection": inputs.WELL_INJECTION,
        "height": inputs.WELL_HEIGHT,
        "tips": tips.tolist(),
        "D": {str(h): [float("%.13e" % v) for v in sols[h - 1][:2 * N]] for h in KEEP_D},
        "KI": {}, "KII": {},
    }
    for h in KEEP_K:
        KI, KII = oracle.sif(mat, xy, sols[h - 1], tips)
        out["KI"][str(h)] = [float("%.13e" % v) for v in KI]
        out["KII"][str(h)] = [float("%.13e" % v) for v in KII]
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "well_march_10x40.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
