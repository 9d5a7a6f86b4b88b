"""The test helpers that sample the full-size workloads: binned candidates and
per-centre oracle rows equal the oracle's list over every atom."""
import numpy as np

import synth
from oracle import mtp as O
from tests.helpers import BinnedCandidates, oracle_rows


def test_binned_candidates_give_the_full_rows():
    st = synth.crystal("bcc", (8, 8, 8), 3.16, 0.08, 3, 2)
    r_cut = 5.0
    i, j, n = O.neighbor_list(st.x, st.cell, st.pbc, r_cut)
    cands = BinnedCandidates(st, r_cut + 0.5)
    for c in synth.rng(2, 91).choice(st.n, 12, replace=False):
        oj, on = oracle_rows(st, r_cut, c, cands(c))
        sel = i == c
        assert np.array_equal(oj, j[sel])
        assert np.array_equal(on, n[sel])
