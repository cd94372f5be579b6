"""Match the 72-cell ring's quadrupole gradients to bare tunes (22.40, 20.75).

Writes nothing; prints the two gradients that paper_2010_11540_gb300/synth.py
stores as C2_K1F / C2_K1D.  Uses only the oracle (one-turn matrix of the
push at psigma = 0, cos mu = Tr/2) and Newton iteration on the tunes.
Run: python -m oracle.match_ring
With --scan: the 8 x 8 working points (22.40, 20.75) + (dqx, dqy), dqx and
dqy in 8 equal steps over [-0.1, 0.1], one line per point (k1F, k1D, Qx, Qy),
the table synth.py stores as C4_WORKING_POINTS.
"""
import sys

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


def match(target, k0=(0.16, -0.15)):
    k = np.array(k0, dtype=float)
    for _ in range(30):
        f = cell_tunes(k) - target
        J = np.zeros((2, 2))
        for c in range(2):
            dk = np.zeros(2)
            dk[c] = 1e-7
            J[:, c] = (cell_tunes(k + dk) - cell_tunes(k - dk)) / 2e-7
        k = k - np.linalg.solve(J, f)
        if np.max(np.abs(f)) < 1e-12:
            break
    return k


def main():
    if "--scan" in sys.argv:
        k = np.array([0.16, -0.15])
        for dqx in np.linspace(-0.1, 0.1, 8):
            for dqy in np.linspace(-0.1, 0.1, 8):
                k = match(TARGET + np.array([dqx, dqy]), k)
                q = cell_tunes(k)
                print(f"    ({float(k[0])!r}, {float(k[1])!r}),  # ({q[0]:.4f}, {q[1]:.4f})")
        return
    k = match(TARGET)
    print(repr(float(k[0])), repr(float(k[1])), cell_tunes(k))


if __name__ == "__main__":
    main()
