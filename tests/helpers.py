"""Shared test helpers: potentials, workloads, oracle sampling at full size."""
import json
import os

import numpy as np

import synth
from oracle import mtp as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def pot_dict(name):
    with open(os.path.join(ROOT, "potentials", name + ".json")) as fh:
        return json.load(fh)


def oracle_model(name):
    return O.load_model(pot_dict(name))


def structure(kind, cells, a, sigma, species, stream, sub=0):
    if kind == "gas":
        return synth.random_gas(cells, 0.085, 1.9, species, synth.rng(stream, 200 + sub))
    return synth.crystal(kind, cells, a, sigma, species, stream, sub)


def min_image_candidates(st, centres, radius):
    """Atoms within ``radius`` of any centre under the minimum image (valid when
    every cell height exceeds twice the radius)."""
    inv = np.linalg.inv(st.cell)
    h = 1.0 / np.linalg.norm(inv, axis=0)
    assert np.all(h > 2 * radius)
    frac = st.x @ inv
    keep = np.zeros(st.n, dtype=bool)
    for c in np.atleast_1d(centres):
        d = frac - frac[c]
        d -= np.round(d)
        r = np.linalg.norm(d @ st.cell, axis=1)
        keep |= r < radius
    return np.nonzero(keep)[0]


def oracle_sampled(model, st, r_cut, centres, force_atoms=()):
    """Oracle site energies of ``centres`` and forces on ``force_atoms`` of a
    large periodic structure, from neighbour lists of the atoms involved only."""
    res = {}
    centres = np.asarray(centres)
    cand = min_image_candidates(st, centres, r_cut + 0.5)
    nl = O.neighbor_list(st.x, st.cell, st.pbc, r_cut, query=centres, candidates=cand)
    out = O.evaluate(model, st.x, st.z, st.cell, nl, want=("e",), atoms=centres)
    res["e_atom"] = out["e_atom"]
    res["nbr_count"] = np.bincount(np.searchsorted(centres, nl[0]), minlength=len(centres)) if len(centres) else []
    forces = []
    for k in force_atoms:
        cand_k = min_image_candidates(st, [k], 2 * r_cut + 0.5)
        nl_k = O.neighbor_list(st.x, st.cell, st.pbc, r_cut, query=[k], candidates=cand_k)
        involved = np.unique(np.concatenate([[k], nl_k[1]]))
        nl_i = O.neighbor_list(st.x, st.cell, st.pbc, r_cut, query=involved, candidates=cand_k)
        out = O.evaluate(model, st.x, st.z, st.cell, nl_i, want=("e", "f"), atoms=involved)
        forces.append(out["f"][k])
    res["forces"] = np.array(forces)
    return res


class BinnedCandidates:
    """Candidate atoms near a centre from a grid of fractional bins at least
    ``radius`` high (valid when every cell height exceeds three bins): the
    atoms of the 27 bins around the centre's bin, periodic in every axis."""

    def __init__(self, st, radius):
        inv = np.linalg.inv(st.cell)
        h = 1.0 / np.linalg.norm(inv, axis=0)
        self.nb = np.maximum(1, np.floor(h / radius).astype(int))
        assert np.all(self.nb >= 3)
        frac = (st.x @ inv) % 1.0
        self.bin = np.minimum((frac * self.nb).astype(int), self.nb - 1)
        key = (self.bin[:, 0] * self.nb[1] + self.bin[:, 1]) * self.nb[2] + self.bin[:, 2]
        self.order = np.argsort(key, kind="stable")
        self.start = np.searchsorted(key[self.order], np.arange(int(np.prod(self.nb)) + 1))

    def __call__(self, c):
        b = self.bin[c]
        out = []
        for d0 in (-1, 0, 1):
            for d1 in (-1, 0, 1):
                for d2 in (-1, 0, 1):
                    q = (b + (d0, d1, d2)) % self.nb
                    k = (q[0] * self.nb[1] + q[1]) * self.nb[2] + q[2]
                    out.append(self.order[self.start[k]:self.start[k + 1]])
        return np.unique(np.concatenate(out))


def oracle_rows(st, r_cut, centre, cand):
    """The oracle's neighbour rows (j, n) of one centre, computed on the
    sub-array of its candidates (the same coordinates, so the same arithmetic)
    and mapped back to the full structure's atom indices."""
    sub = np.union1d(cand, [centre])
    loc = int(np.searchsorted(sub, centre))
    _, j, n = O.neighbor_list(st.x[sub], st.cell, st.pbc, r_cut, query=[loc])
    return sub[j], n
