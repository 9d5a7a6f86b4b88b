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
