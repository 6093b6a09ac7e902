"""Writes the stored expected values under tests/golden/ (calls only oracle/).

single_L16_exact.txt: exact discrete-dtau G(tau_k) and D of the single-grid
workload (Bethe bath, U = 4, beta = 8, dtau = 0.5, Lambda = 16) by enumeration
of all 2^16 HS fields; the Monte Carlo of both the oracle and the GPU path
must land on these within error bars.

Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_0801_1222_gb300 import inputs  # noqa: E402


def main():
    beta, U, L = 8.0, 4.0, 16
    g0 = inputs.bethe_G0_tau(beta, L)
    g, D, Z = oracle.brute_force(oracle.bath_matrix(g0), oracle.lam(beta / L, U))
    G = np.concatenate([-g, [-1.0 + g[0]]])
    with open(os.path.join(HERE, "single_L16_exact.txt"), "w") as f:
        f.write("# exact G(tau_k), k=0..16 (k=16 is beta-), then D; Bethe W=4, U=4, beta=8, L=16\n")
        f.write("# written by tests/golden/make_golden.py from oracle.brute_force (2^16 fields)\n")
        for v in G:
            f.write(f"{v:.17e}\n")
        f.write(f"{D:.17e}\n")


if __name__ == "__main__":
    main()
