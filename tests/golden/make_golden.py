"""Writes the stored expected values under tests/golden/ by calling only the
FP64 oracle (never the CUDA path).

* rand2d_6x6_d16_sidewise.json -- the 6 x 6 depth-16 reduction of the 8 x 8 random
  circuit workload (same generation rules, seed 0), one amplitude of a
  seed-random bitstring, by the oracle's side-wise (left-to-right) FP64
  contraction (the naive-order scheme of the paper's Thm. 2 discussion).
  Takes tens of minutes and ~30 GB of host memory.

Usage: python tests/golden/make_golden.py [rand2d_6x6_d16]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import circuits as C  # noqa: E402
import oracle as O  # noqa: E402


def rand2d_6x6_d16(seed: int = 0):
    gl, info = C.workload("rand2d_8x8_d16", seed, reduced=True)
    t0 = time.time()
    a = O.sidewise_amplitudes(gl, info["bits"], order="columns")
    dt = time.time() - t0
    out = {
        "description": "6x6 depth-16 random circuit (Haar 1q, CZ on brick patterns ABCD), seed %d; amplitude "
                       "<x|C|0> of the seed-random bitstring x by the oracle's side-wise FP64 contraction" % seed,
        "generator": "circuits.workload('rand2d_8x8_d16', %d, reduced=True)" % seed,
        "bits": info["bits"][0].tolist(),
        "amplitude": [float(a[0, 0].real), float(a[0, 0].imag)],
        "oracle_seconds": round(dt, 1),
    }
    with open(os.path.join(HERE, "rand2d_6x6_d16_sidewise.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    which = sys.argv[1:] or ["rand2d_6x6_d16"]
    if "rand2d_6x6_d16" in which:
        rand2d_6x6_d16()
