"""Writes the synthetic potentials (and grade active sets) under ``potentials/``.

TEST INFRASTRUCTURE: runs the oracle once, offline; the files it writes are
data, the way a fitted MLIP potential file is data.  Run from the repo root:

    python -m oracle.make_potentials            # all workloads
    python -m oracle.make_potentials bcc-l8-s1  # one
    python -m oracle.make_potentials active     # grade active sets (after the potentials)

Normalisation (a reading: the paper's workloads use trained potentials, which
are not available).  Raw coefficients are drawn by ``synth.raw_potential``:
c ~ N(0, 0.1^2), s ~ N(0, 1), xi_raw ~ N(0, 0.1^2).  Products of up to eight
moments then give site energies of 1e4 to 1e9 eV, far outside any physical
range, so each linear coefficient is rescaled to xi_alpha = xi_raw_alpha /
rms_alpha, with rms_alpha the root mean square of B_alpha over the atoms of a
small seeded reference structure drawn from the same recipe as the workload
(same lattice, displacement, species mix; a different seed).  Every term
xi_alpha B_alpha is then O(0.1) eV.

The basis is the oracle's own: enumeration plus FP64 greedy pruning on random
neighbourhoods (``oracle.mtp.make_basis``); the file stores it in canonical
form so a consumer can check its own basis against it.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

import synth
from oracle import mtp as O

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(os.path.dirname(HERE), "potentials")

# name: (level, species, n_q, r_cut, reference-structure recipe, stream)
SPECS = {
    "bcc-l8-s1": dict(level=8, species=1, n_q=8, r_cut=5.0, ref=("bcc", (4, 4, 4), 3.16, 0.05), stream=1),
    "bcc-l16-s3": dict(level=16, species=3, n_q=8, r_cut=5.0, ref=("bcc", (4, 4, 4), 3.16, 0.08), stream=2),
    "bcc-l16-s3-rc5.6": dict(level=16, species=3, n_q=8, r_cut=5.6, ref=("bcc", (4, 4, 4), 3.16, 0.08), stream=2),
    "fcc-l20-s4": dict(level=20, species=4, n_q=10, r_cut=5.5, ref=("fcc", (3, 3, 3), 3.6, 0.1), stream=3),
    "gas-l16-s2": dict(level=16, species=2, n_q=8, r_cut=5.0, ref=("gas", 6, 0.085, 1.9), stream=4),
    "bcc-l16-s1": dict(level=16, species=1, n_q=8, r_cut=5.0, ref=("bcc", (4, 4, 4), 3.16, 0.15), stream=5),
}
R_MIN = 2.0
PRUNE_STREAM = 99


def oracle_basis(level: int) -> O.Basis:
    graphs = O.connected_graphs(level)
    m_all = len(O.basis_functions(level, graphs))
    u, f = synth.random_neighbourhoods(3 * m_all, 16, O.n_mu_for_level(level), synth.rng(PRUNE_STREAM, level))
    return O.make_basis(level, u, f)


def reference_structures(spec) -> list:
    ref = spec["ref"]
    if ref[0] in ("bcc", "fcc"):
        kind, cells, a, sigma = ref
        return [synth.crystal(kind, cells, a, sigma, spec["species"], spec["stream"], sub=7)]
    _, count, density, min_sep = ref
    return synth.random_gas_batch(count, 32, 96, density, min_sep, spec["species"], 100 + spec["stream"])


def encode_basis(basis: O.Basis) -> list:
    return [[[list(basis.graphs[k].mu), list(basis.graphs[k].e)] for k in b] for b in basis.bases]


def make(name: str) -> dict:
    spec = SPECS[name]
    level = spec["level"]
    basis = oracle_basis(level)
    n_mu = O.n_mu_for_level(level)
    raw = synth.raw_potential(level, spec["species"], spec["n_q"], R_MIN, spec["r_cut"], n_mu, basis.m,
                              spec["stream"])
    pot = O.Potential(level, spec["species"], spec["n_q"], R_MIN, spec["r_cut"], raw.species_energy,
                      raw.radial, np.ones(basis.m))
    model = O.Model(pot, basis)
    rows = []
    for st in reference_structures(spec):
        nl = O.neighbor_list(st.x, st.cell, st.pbc, spec["r_cut"])
        rows.append(O.basis_matrix(model, st.x, st.z, st.cell, nl))
    b = np.concatenate(rows)
    rms = np.sqrt((b * b).mean(axis=0))
    xi = raw.xi_raw / rms
    return {
        "name": name,
        "level": level,
        "n_species": spec["species"],
        "n_q": spec["n_q"],
        "n_mu": n_mu,
        "r_min": R_MIN,
        "r_cut": spec["r_cut"],
        "m": basis.m,
        "species_energy": [float(v) for v in raw.species_energy],
        "radial_shape": list(raw.radial.shape),
        "radial": [float(v) for v in raw.radial.ravel()],
        "xi": [float(v) for v in xi],
        "basis": encode_basis(basis),
        "note": "xi_alpha = xi_raw_alpha / rms_alpha over a seeded reference structure (oracle, FP64)",
    }


def main(argv):
    names = argv[1:] or list(SPECS)
    os.makedirs(OUT, exist_ok=True)
    for name in names:
        pot = make(name)
        with open(os.path.join(OUT, name + ".json"), "w") as fh:
            json.dump(pot, fh, indent=0)
        print(name, "m =", pot["m"])




# ---------------------------------------------------------------------------
# Active sets for the extrapolation grade (paper Sec. 2.1: configuration and
# neighbourhood mode; MaxVol of Goreinov et al. 2010 as cited in Sec. 1)
# ---------------------------------------------------------------------------

ACTIVE = {
    # neighbourhood mode: pool = every atom of a 20^3-cell BCC box (16,000 atoms, sigma 0.05 A)
    # configuration mode: pool = summed basis rows of 4m 128-atom BCC boxes (sigma 0.05 A,
    # every cell vector scaled by an independent factor in [0.98, 1.02])
    "bcc-l16-s1": dict(pool_cells=(20, 20, 20), a=3.16, sigma=0.05, stream=5),
}


def make_active_set(name: str) -> dict:
    import json as _json
    spec = ACTIVE[name]
    with open(os.path.join(OUT, name + ".json")) as fh:
        pot = _json.load(fh)
    model = O.load_model(pot)
    st = synth.crystal("bcc", spec["pool_cells"], spec["a"], spec["sigma"], pot["n_species"], spec["stream"], sub=8)
    nl = O.neighbor_list(st.x, st.cell, st.pbc, pot["r_cut"])
    pool = O.basis_matrix(model, st.x, st.z, st.cell, nl)
    rows, a_inv, iters = O.maxvol(pool, delta=0.01)
    m = pool.shape[1]
    g = synth.rng(spec["stream"], 60)
    cfg_rows = []
    for k in range(4 * m):
        c = synth.crystal("bcc", (4, 4, 4), spec["a"], spec["sigma"], pot["n_species"], spec["stream"], sub=100 + k)
        scale = g.uniform(0.98, 1.02, size=3)
        cell = c.cell * scale[:, None]
        x = c.x @ np.linalg.inv(c.cell) @ cell
        nlc = O.neighbor_list(x, cell, c.pbc, pot["r_cut"])
        cfg_rows.append(O.basis_matrix(model, x, c.z, cell, nlc).sum(axis=0))
    cfg_pool = np.array(cfg_rows)
    cfg_sel, a_inv_cfg, iters_cfg = O.maxvol(cfg_pool, delta=0.01)
    return {
        "potential": name,
        "m": m,
        "a_inv": [float(v) for v in a_inv.ravel()],
        "active_rows": [int(r) for r in rows],
        "cond": float(np.linalg.cond(pool[rows])),
        "maxvol_iterations": int(iters),
        "a_inv_cfg": [float(v) for v in a_inv_cfg.ravel()],
        "active_cfg": [int(r) for r in cfg_sel],
        "cond_cfg": float(np.linalg.cond(cfg_pool[cfg_sel])),
        "maxvol_iterations_cfg": int(iters_cfg),
        "note": "A^-1 of the MaxVol active sets (delta 0.01), FP64 Gauss-Jordan; row-major m x m",
    }


def main_active(argv):
    for name in argv[1:] or list(ACTIVE):
        d = make_active_set(name)
        with open(os.path.join(OUT, name + "-active.json"), "w") as fh:
            json.dump(d, fh, indent=0)
        print(name, "cond", d["cond"], "cond_cfg", d["cond_cfg"], "iters", d["maxvol_iterations"], d["maxvol_iterations_cfg"])


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "active":
        main_active(sys.argv[1:])
    else:
        main(sys.argv)
