"""Writes the stored expected values under tests/golden/.

It calls only the CPU oracle (``oracle/``) on seeded synthetic inputs
(``synth``); no stored value comes from the CUDA path.

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
    img = synth.uniform_2d_256()
    for mode in (oracle.VERTEX, oracle.TOPCELL):
        ecc = oracle.ecc(img, 0, 255, mode)
        path = os.path.join(HERE, f"uniform_256x256_seed0_{mode}.txt")
        np.savetxt(path, ecc, fmt="%d",
                   header=f"ECC[g] = chi(K_<=g), g=0..255, {mode} complex; 256x256 uint8 "
                          "iid uniform numpy default_rng(0); written by make_golden.py (oracle only)")
        print("wrote", path)


if __name__ == "__main__":
    main()
