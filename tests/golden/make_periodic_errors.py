"""Writes periodic_primal_errors.txt: the steady-state errors of the periodic primal
scheme against the manufactured solution (Section 4.2.2), N_x = 32, 64, 128, 256.

Calls only the oracle (its exact per-wavevector fixed point) and the closed-form inputs;
run from the repository root:  python tests/golden/make_periodic_errors.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import fourier  # noqa: E402
from paper_2609_31347_b300 import inputs as I  # noqa: E402

NXS = (32, 64, 128, 256)


def errors(nx):
    """Relative errors (e^d L2, e^d Linf, e^sigma L2, e^sigma Linf) of the steady state
    (Eqs. L2_norm, Linf_norm; stress as Frobenius rows)."""
    m = I.periodic_manufactured(nx)
    fS = fourier.periodic_fixed_point(nx, I.PAPER_E, I.PAPER_NU, m["Fstar"])
    d = fourier.displacement(fS, m["Fstar"], m["dx"])
    s = fourier.stress(fS, m["Fstar"], m["dx"], I.PAPER_E, I.PAPER_NU)
    fro = oracle.stress_frobenius_rows
    return (oracle.norm_L2(d - m["dstar"], m["dx"]) / oracle.norm_L2(m["dstar"], m["dx"]),
            oracle.norm_Linf(d - m["dstar"]) / oracle.norm_Linf(m["dstar"]),
            oracle.norm_L2(fro(s - m["sigma"]), m["dx"]) / oracle.norm_L2(fro(m["sigma"]), m["dx"]),
            oracle.norm_Linf(s - m["sigma"]) / oracle.norm_Linf(m["sigma"]))


def main():
    rows = np.array([errors(nx) for nx in NXS])
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "periodic_primal_errors.txt")
    with open(out, "w") as fh:
        fh.write("# Steady periodic primal errors, Section 4.2.2 setup (delta = (9e-4, 7e-4),\n")
        fh.write("# E = 0.11, nu = 0.8, g = dx^2 F, sigma = -mbar_2 / dx), relative discrete\n")
        fh.write("# L2 / Linf norms of Section 4.1.  Written by make_periodic_errors.py from the\n")
        fh.write("# oracle's exact fixed point; the paper prints only their EOCs.\n")
        fh.write("nx " + " ".join(str(n) for n in NXS) + "\n")
        for j, key in enumerate(["e_d_L2", "e_d_Linf", "e_sigma_L2", "e_sigma_Linf"]):
            fh.write(key + " " + " ".join("%.12e" % v for v in rows[:, j]) + "\n")
    print(out)


if __name__ == "__main__":
    main()
