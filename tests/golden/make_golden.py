"""Writes oracle_two_species.json beside this script: a small seeded
two-species trajectory (the stored inputs) and the FP64 oracle's spectra on it,
incoherent and coherent, for every window and direction.

The expected values come from the oracle alone (``oracle.spectra``: the
discretised far-field integral of Sec. 2.2 with the Lienard-Wiechert integrand
of Jackson eq. 14.67, the rectangle rule over the leapfrog samples, and the
1/(4 pi^2 c) prefactor); the inputs come from the seeded generator
(``trajgen``, Boris push of two counter-streaming beams in a frozen periodic
field).  The inputs are stored too, so the fixture does not depend on the
generator's random streams.  Regenerate with

    python tests/golden/make_golden.py

only when a change to the oracle's arithmetic has been justified from the
paper; the stored file is the record that such a change shows up against.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle    # noqa: E402
import trajgen   # noqa: E402

OUT = os.path.join(HERE, "oracle_two_species.json")


def workload():
    """3 electrons (gamma 3) + 2 ions (m = 16, q = +1), 25 calls, 3 directions,
    a 20-point log grid and a 7-point linear grid, three windows (one per
    species and one for both)."""
    return trajgen.Workload(
        "golden-two-species", [(3, -1.0, 1.0, 3.0), (2, 1.0, 16.0, 3.0)], 25, 0.05,
        np.array([[0.0, 1.0, 0.0], [1.0, 0.0, 0.0], [0.6, 0.0, 0.8]]),
        [trajgen.log_grid(0.1, 100.0, 20), np.linspace(0.5, 9.5, 7)],
        [(0, 24, 3, 0), (5, 17, 1, 1), (3, 11, 2, 0)], b_rms=0.3, field_seed=5,
        particle_seed=9)


def main():
    w = workload()
    X, U = w.trajectory_numpy()
    species = [(s[0], s[1]) for s in w.species]
    data = {
        "what": "FP64 oracle spectra (oracle.spectra) on stored inputs",
        "citation": "Sec. 2.2 discretised P_omega integral; Jackson eq. 14.67 integrand; "
                    "S = 1/(4 pi^2) sum_j |A_j|^2 (incoherent) or |sum_j A_j|^2 (coherent)",
        "writer": "tests/golden/make_golden.py (calls only oracle/ for expected values)",
        "dt": w.dt, "box_L": w.L,
        "species": [[int(s[0]), float(s[1]), float(s[2])] for s in w.species],
        "dirs": w.dirs.tolist(),
        "grids": [np.asarray(g).tolist() for g in w.grids],
        "windows": [list(map(int, win)) for win in w.windows],
        "x": X.tolist(), "u": U.tolist(),
    }
    for coh in (False, True):
        S = oracle.spectra(X, U, w.dt, w.dirs, w.grids, w.windows, species, coherent=coh,
                           box_L=w.L)
        data["coherent" if coh else "incoherent"] = [np.asarray(s).tolist() for s in S]
    with open(OUT, "w") as f:
        json.dump(data, f, separators=(",", ":"))
        f.write("\n")
    print(f"wrote {OUT}: {os.path.getsize(OUT)} bytes")


if __name__ == "__main__":
    main()
