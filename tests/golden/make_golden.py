"""Writes the stored expected values under tests/golden/ by calling only oracle/.

    python tests/golden/make_golden.py

mlp_forward_8_16_16_4.txt: the oracle MLP forward pass on fixed, formula-given
weights (W[i, j] = 0.3 sin(1 + i + 2 j) style, see _weights) and inputs, a
regression pin of the oracle network (GELU with erf, Hendrycks and Gimpel 2016).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import mlp  # noqa: E402


def _weights(D=8, H=16, r=4):
    def mat(n, m, a):
        i = np.arange(n)[:, None]
        j = np.arange(m)[None, :]
        return 0.3 * np.sin(a + i + 2.0 * j) / np.sqrt(m)
    return {"W1": mat(H, D, 1.0), "b1": 0.1 * np.cos(np.arange(H)),
            "W2": mat(H, H, 2.0), "b2": 0.05 * np.sin(np.arange(H)),
            "W3": mat(r, H, 3.0), "b3": 0.2 * np.cos(0.5 * np.arange(r))}


def _inputs(B=5, D=8):
    i = np.arange(B)[:, None]
    j = np.arange(D)[None, :]
    return np.cos(0.7 * i + 0.3 * j) * 1.5


def main():
    Y, _ = mlp.forward(_weights(), _inputs())
    path = os.path.join(HERE, "mlp_forward_8_16_16_4.txt")
    with open(path, "w") as f:
        f.write("# oracle MLP forward (8->16->16->4, exact GELU) on the weights/inputs of make_golden.py\n")
        for row in Y:
            f.write(" ".join("%.17e" % v for v in row) + "\n")


if __name__ == "__main__":
    main()
