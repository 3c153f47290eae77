"""Writes c2_ionic_20x20_adam3000.txt: the FP64 oracle's Adam run on the 20x20 ionic workload.

Workload (Sec. III lattice and temperature; Eq. 1 and Eq. 2): L = 20, t = 1, U = 6, Delta = 0.5,
T = 0.1, mu = 0, 256 positive Matsubara frequencies x 2 spins, start field the SplitMix64 field
of seed 0, Adam lr = 0.01, betas (0.9, 0.999), eps = 1e-8, 3000 updates without a gate.  The
run uses oracle.adam_run_spectral (the eigenvalue route, pinned against the LU route in
tests/test_oracle_pins.py), which takes about two minutes on one CPU.

Usage: python tests/golden/make_c2_reference.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2311_04435_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "c2_ionic_20x20_adam3000.txt")


def main():
    L, n_omega, U, delta, T = 20, 256, 6.0, 0.5, 0.1
    p = oracle.make_params(L, n_omega, U=U, T=T, delta=delta)
    phi0 = inputs.seed_phi(0, L * L)
    rows = []
    phi = phi0
    done = 0
    for target in (1000, 2000, 3000):
        # adam_run_spectral restarts the moments, so each checkpoint is one run from phi0
        phi, k, om, gm = oracle.adam_run_spectral(p, phi0, lr=0.01, max_steps=target)
        stag, mean = oracle.staggered_order(phi, L)
        rows.append((k, om, gm, stag, mean))
        done = k
    with open(OUT, "w") as f:
        f.write("# FP64 oracle (oracle.adam_run_spectral): 20x20 ionic Hubbard, t=1, U=6, Delta=0.5,\n")
        f.write("# T=0.1, mu=0, 256 Matsubara frequencies, seed-0 SplitMix64 start, Adam lr=0.01\n")
        f.write("# betas (0.9, 0.999), eps 1e-8, no gate.  Written by make_c2_reference.py.\n")
        f.write("# steps omega max|g| stag|phi| mean|phi|  (Omega and max|g| at the field after the steps)\n")
        for k, om, gm, stag, mean in rows:
            f.write(f"{k} {float(om)!r} {float(gm)!r} {float(stag)!r} {float(mean)!r}\n")
        f.write(f"# phi after {done} steps, site order i = x*L + y\n")
        for v in phi:
            f.write(f"{float(v)!r}\n")


if __name__ == "__main__":
    main()
