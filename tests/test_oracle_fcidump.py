"""Pins for the FCIDUMP reader/writer (oracle).

A hand-written file (tests/golden/fcidump_2orb.txt) against its hand
expansion by the format's symmetry rules; write/read round trips of
synthetic integrals are exact; the Hamiltonian of read integrals has the
original's Hartree-Fock energy.
"""

import os

import numpy as np

import synth
from oracle import fcidump
from test_oracle_hamiltonian import hf_energy_closed_form

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def expected_2orb():
    h = np.full((2, 2), np.nan)
    g = np.full((2, 2, 2, 2), np.nan)
    meta = {}
    for line in open(os.path.join(GOLD, "fcidump_2orb_expected.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] == "h":
            h[int(f[1]), int(f[2])] = float(f[3])
        elif f[0] == "g":
            g[tuple(int(x) for x in f[1:5])] = float(f[5])
        elif f[0] == "e":
            meta["e"] = float(f[1])
        else:
            meta[f[0]] = int(f[1])
    assert not np.isnan(h).any() and not np.isnan(g).any()
    return h, g, meta


def test_hand_written_file():
    h, g, meta = expected_2orb()
    rh, rg, e, n, ne, ms2 = fcidump.read(os.path.join(GOLD, "fcidump_2orb.txt"))
    assert np.array_equal(rh, h) and np.array_equal(rg, g)
    assert e == meta["e"] and n == meta["norb"] and ne == meta["nelec"] and ms2 == meta["ms2"]


def test_round_trip_is_exact(tmp_path):
    for n, seed in [(3, 6), (4, 0), (6, 1)]:
        ints = synth.integrals(n, seed)
        path = str(tmp_path / f"f{n}.txt")
        fcidump.write(path, ints.h, ints.g, 1.25, 2 * (n // 2))
        h, g, e, nn, ne, ms2 = fcidump.read(path)
        assert nn == n and ne == 2 * (n // 2) and ms2 == 0 and e == 1.25
        assert np.array_equal(h, ints.h) and np.array_equal(g, ints.g)


def test_read_integrals_give_the_same_hf_energy(tmp_path):
    ints = synth.integrals(4, 3)
    path = str(tmp_path / "f.txt")
    fcidump.write(path, ints.h, ints.g, 0.0, 4)
    h, g, *_ = fcidump.read(path)
    assert hf_energy_closed_form(h, g, 4) == hf_energy_closed_form(ints.h, ints.g, 4)
