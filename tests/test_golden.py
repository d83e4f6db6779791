"""The oracle against its stored record: tests/golden/oracle_two_species.json
holds a small seeded two-species trajectory and the FP64 oracle's spectra on it
(written by tests/golden/make_golden.py, which takes its expected values from
oracle/ alone).  Any later change to the oracle's arithmetic shows up here and
has to be justified from the paper (Sec. 2.2) before the record is rewritten."""
import json
import os

import numpy as np

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_reproduces_its_golden_record():
    with open(os.path.join(HERE, "golden", "oracle_two_species.json")) as f:
        d = json.load(f)
    X, U = np.array(d["x"]), np.array(d["u"])
    assert X.shape == U.shape == (25, 3, 5)
    dirs = np.array(d["dirs"])
    grids = [np.array(g) for g in d["grids"]]
    windows = [tuple(w) for w in d["windows"]]
    species = [(s[0], s[1]) for s in d["species"]]
    for key, coh in (("incoherent", False), ("coherent", True)):
        got = oracle.spectra(X, U, d["dt"], dirs, grids, windows, species, coherent=coh,
                             box_L=d["box_L"])
        assert len(got) == len(d[key]) == 3
        for g, e in zip(got, d[key]):
            e = np.array(e)
            assert g.shape == e.shape
            assert np.all(e >= 0.0) and e.max() > 0.0
            # libm sin/cos may differ by an ulp between machines: 1e-12, not bitwise
            for k in range(e.shape[0]):
                assert np.linalg.norm(g[k] - e[k]) <= 1e-12 * np.linalg.norm(e[k]), (key, k)
