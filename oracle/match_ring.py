"""Match the 72-cell ring's quadrupole gradients to bare tunes (22.40, 20.75).

Writes nothing; prints the two gradients that paper_2010_11540_gb300/synth.py
stores as C2_K1F / C2_K1D.  Uses only the oracle (one-turn matrix of the
push at psigma = 0, cos mu = Tr/2) and Newton iteration on the tunes.
Run: python -m oracle.match_ring
"""
import numpy as np

import oracle
from paper_2010_11540_gb300 import synth

TARGET = np.array([22.40, 20.75])


def cell_tunes(k):
    b = synth.beam(circumference=24.0)
    cell = synth.table(synth.ring_c2_cell(k1f=k[0], k1d=k[1]))
    M = oracle.one_turn_matrix(cell, b)
    mux = oracle.twiss_from_matrix(M[:2, :2])[0]
    muy = oracle.twiss_from_matrix(M[2:, 2:])[0]
    return 72 * np.array([mux, muy]) / (2 * np.pi)


def main():
    k = np.array([0.16, -0.15])
    for _ in range(30):
        f = cell_tunes(k) - TARGET
        J = np.zeros((2, 2))
        for c in range(2):
            dk = np.zeros(2)
            dk[c] = 1e-7
            J[:, c] = (cell_tunes(k + dk) - cell_tunes(k - dk)) / 2e-7
        k = k - np.linalg.solve(J, f)
        if np.max(np.abs(f)) < 1e-12:
            break
    print(repr(float(k[0])), repr(float(k[1])), cell_tunes(k))


if __name__ == "__main__":
    main()
