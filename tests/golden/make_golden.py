"""Writes the stored oracle values of tests/golden/ (calls only oracle/ and the seeded input
generator).  Run from the repository root: python tests/golden/make_golden.py"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import epwi_oracle as O  # noqa: E402
from paper_2306_16493_gb300 import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def tiny_6():
    """Tiny system (seed 1) on a 6^3 grid, T = 300 K, mu at the band centre, eta = 50 meV,
    all states: the SERTA rates (Sec. II C, Eq. 10) and the transport tensors (Eqs. 12-14)."""
    s = synth.tiny_system(1)
    gr = O.Grids(s, (6, 6, 6))
    mu = gr.band_centre()
    T, eta = 300.0, 0.05
    r = O.serta(gr, T, mu, eta, -np.inf, np.inf)
    v = gr.velocities(r["ik"], r["n"])
    sig, S, kap = O.transport_coefficients(s.volume, gr.nk, v, r["inv_tau"], gr.eps[r["ik"], r["n"]], mu, T)
    path = os.path.join(HERE, "tiny_6_serta.txt")
    with open(path, "w") as f:
        f.write("# tiny system (seed 1), 6^3 grid, T = 300 K, mu = band centre, eta = 0.05 eV, all states\n")
        f.write("# Sec. II C Eq. 10 (1/tau, s^-1) and Eqs. 12-14 (sigma S/m, S V/K, kappa_e W/(m K))\n")
        f.write(f"mu {float(mu)!r}\n")
        f.write(f"n_pairs {r['n_pairs']}\n")
        for name, t in (("sigma", sig), ("seebeck", S), ("kappa_e", kap)):
            f.write(name + " " + " ".join(repr(float(x)) for x in t.ravel()) + "\n")
        f.write("# ik n inv_tau\n")
        for ik, n, x in zip(r["ik"], r["n"], r["inv_tau"]):
            f.write(f"{int(ik)} {int(n)} {float(x)!r}\n")
    return path


if __name__ == "__main__":
    print(tiny_6())
