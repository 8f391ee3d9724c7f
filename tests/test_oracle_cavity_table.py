"""The oracle's long cavity runs against the paper's Table vort (Sec. 4.4.1).

tests/golden/cavity100_long_oracle.txt holds the oracle's own 2e5-step runs of
the 100 x 100 cavity as the paper sets it up (boundary nodes on the walls with
bounce-back and a constant lid, density 2.7, lid 0.1, polynomial f*, median
filter delta = 1e-3 and 1e-4), written by tests/golden/make_cavity_long_runs.py.
The paper's vortex centres (tests/golden/table_vort_polynomial.txt, rows (b) and
(c)) must be within one cell (1/99) of the oracle's, mass must be conserved, and
unregularised LBGK (row (a)) must blow up at Re = 7500.
"""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
CELL = 1.0 / 99.0
NAMES = ("primary", "lower_left", "lower_right", "top_left")


def read_table():
    rows = {}
    for line in open(os.path.join(HERE, "golden", "table_vort_polynomial.txt")):
        if line.startswith("#") or not line.strip():
            continue
        p = line.split()
        rows[(int(p[0]), p[1])] = np.array([float(x) for x in p[2:10]]).reshape(4, 2)
    return rows


def read_oracle_runs():
    runs = {}
    for line in open(os.path.join(HERE, "golden", "cavity100_long_oracle.txt")):
        if line.startswith("#") or not line.strip():
            continue
        p = line.split()
        key = (int(p[0]), p[1], float(p[2]))
        runs[key] = {"steps": int(p[3]), "centres": np.array([float(x) for x in p[4:12]]).reshape(4, 2),
                     "drift": float(p[12])}
    return runs


def test_oracle_long_runs_reproduce_table_vort_within_one_cell():
    table, runs = read_table(), read_oracle_runs()
    for re in (5000, 7500):
        for delta, row in ((1e-3, "b"), (1e-4, "c")):
            run = runs[(re, "median", delta)]
            assert run["steps"] == 200000
            assert abs(run["drift"]) < 1e-10, (re, delta, run["drift"])
            want = table[(re, row)]
            for v, name in enumerate(NAMES):
                got = run["centres"][v]
                assert np.all(np.abs(got - want[v]) <= CELL + 1e-4), (re, row, name, got, want[v])


def test_unregularised_lbgk_blows_up_at_re_7500():
    run = read_oracle_runs()[(7500, "none", 0.0)]
    assert run["steps"] < 200000 and np.isnan(run["centres"]).all()
