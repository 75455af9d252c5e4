"""Writes the regression fixtures in this folder.  Calls only the FP64 oracle
and the seeded generators; never the CUDA library.

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402


def main():
    f = synth.make_frame(6, 8, 42)
    out = oracle.denoise(f, synth.make_weights(seed=42))
    np.savetxt(os.path.join(HERE, "tiny_denoise_8x6_seed42.txt"), out.reshape(-1), fmt="%.17e",
               header="oracle.denoise of synth.make_frame(6, 8, 42) with synth.make_weights(seed=42); "
                      "[3, 6, 8] flattened, float64")


if __name__ == "__main__":
    main()
