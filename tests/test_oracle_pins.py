"""Pins of the oracle against closed forms, brute force, hand-derived counts,
finite differences and invariances.  CPU only."""
import itertools
import json
import math
import os

import numpy as np
import pytest
import torch

import synth
from oracle import mtp as O

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def pot_file(name):
    with open(os.path.join(ROOT, "potentials", name + ".json")) as fh:
        return json.load(fh)


def random_model(level, n_species, n_q=8, r_min=2.0, r_cut=5.0, stream=77, xi_scale=1.0):
    """Unnormalised random model (fine for identities that hold at any scale)."""
    graphs = O.connected_graphs(level)
    nb = len(O.basis_functions(level, graphs))
    u, f = synth.random_neighbourhoods(3 * nb, 12, O.n_mu_for_level(level), synth.rng(99, level))
    basis = O.make_basis(level, u, f)
    raw = synth.raw_potential(level, n_species, n_q, r_min, r_cut, O.n_mu_for_level(level), basis.m, stream)
    pot = O.Potential(level, n_species, n_q, r_min, r_cut, raw.species_energy, raw.radial, raw.xi_raw * xi_scale)
    return O.Model(pot, basis)


# --------------------------------------------------------------------------- radial basis


def test_chebyshev_matches_trigonometric_and_hyperbolic_forms():
    xi = np.linspace(-1, 1, 41)
    t = O.chebyshev(xi, 12)
    for k in range(12):
        assert np.allclose(t[k], np.cos(k * np.arccos(xi)), atol=1e-13)
    xo = np.array([-2.5, -1.3, 1.01, 1.7, 3.0])
    t = O.chebyshev(xo, 10)
    for k in range(10):
        ref = np.cosh(k * np.arccosh(np.abs(xo))) * np.sign(xo) ** k
        assert np.allclose(t[k], ref, rtol=1e-12)


def test_radial_basis_endpoints():
    # xi(R_min) = -1, xi(R_cut) = 1; Q_k(R_min) = (-1)^k (R_cut - R_min)^2, Q_k(R_cut) = 0
    q = O.radial_basis(np.array([2.0, 5.0]), 2.0, 5.0, 8)
    for k in range(8):
        assert q[k][0] == pytest.approx((-1) ** k * 9.0, rel=1e-15)
        assert q[k][1] == 0.0


# --------------------------------------------------------------------------- basis enumeration


def _parse_golden_basis(path):
    out = set()
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            lev, facs = line.split("|")
            key = []
            for tok in facs.split():
                mu, e = tok.split("/")
                key.append((eval(mu), eval(e)))
            out.add((int(lev), tuple(sorted(key))))
    return out


def test_level8_basis_equals_hand_derivation():
    graphs = O.connected_graphs(8)
    got = set()
    for b in O.basis_functions(8, graphs):
        key = tuple(sorted((graphs[k].mu, graphs[k].e) for k in b))
        got.add((sum(graphs[k].level for k in b), key))
    assert got == _parse_golden_basis(os.path.join(HERE, "golden", "basis_level8.txt"))


@pytest.mark.parametrize("level,count", [(2, 1), (4, 2), (6, 5), (8, 9), (16, 116), (20, 460)])
def test_basis_counts(level, count):
    # 2, 4, 6, 8: by hand (level-8 list in tests/golden/basis_level8.txt; level 4 = {M00,
    # M00^2}; level 6 adds M00^3, M10, M01.M01).  16 and 20: independent enumeration of
    # the same definition done when the hot path was scoped (116 and 460).
    assert len(O.basis_functions(level)) == count


def test_moment_tensor_sets():
    # components (nu+1)(nu+2)/2 summed over the tensors the graphs use
    for level, comps in [(8, 11), (16, 130), (20, 295)]:
        lay = O.moment_layout(O.connected_graphs(level))
        assert sum((n + 1) * (n + 2) // 2 for _, n in lay) == comps


def test_graph_levels_and_canonical_form():
    for g in O.connected_graphs(16):
        assert g.level <= 16
        mat = [[g.mult(v, w) for w in range(g.nv)] for v in range(g.nv)]
        # every relabelling gives back the same canonical graph
        for p in itertools.permutations(range(g.nv)):
            mu = [g.mu[p[a]] for a in range(g.nv)]
            m2 = [[mat[p[a]][p[b]] for b in range(g.nv)] for a in range(g.nv)]
            assert O.canonical_graph(mu, m2) == g


# --------------------------------------------------------------------------- contractions


@pytest.mark.parametrize("level", [16, 20])
def test_tensor_form_equals_graph_bruteforce(level):
    """einsum over Cartesian indices == sum over neighbour tuples of the defining
    product of f values and dot products (tiny neighbourhoods)."""
    graphs = O.connected_graphs(level)
    n_mu = O.n_mu_for_level(level)
    g = synth.rng(5, level)
    for trial in range(2):
        n = 4 + trial
        u = g.normal(size=(n, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        f = g.normal(size=(n, n_mu))
        mom = O.cartesian_moments(O.moment_layout(graphs), torch.zeros(n, dtype=torch.long), 1,
                                  torch.as_tensor(u), torch.as_tensor(f))
        vals = O.graph_values(graphs, mom)[:, 0].numpy()
        for k, gr in enumerate(graphs):
            ref = O.graph_value_bruteforce(gr, u, f)
            assert vals[k] == pytest.approx(ref, rel=1e-11, abs=1e-11 * (1 + abs(ref)))


def _sym_components(u, f, mu, K):
    return sum(f[j, mu] * u[j, 0] ** K[0] * u[j, 1] ** K[1] * u[j, 2] ** K[2] for j in range(u.shape[0]))


@pytest.mark.parametrize("level", [12, 16])
def test_symmetric_polynomial_equals_bruteforce(level):
    """The integer polynomial in symmetric components (the table the library
    must reproduce) evaluates to the brute-force graph value."""
    graphs = O.connected_graphs(level)
    g = synth.rng(6, level)
    n = 5
    u = g.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    f = g.normal(size=(n, O.n_mu_for_level(level)))
    for gr in graphs:
        poly = O.expand_cartesian(gr)
        val = 0.0
        for mono, coef in poly.items():
            term = float(coef)
            for mu, K in mono:
                term *= _sym_components(u, f, mu, K)
            val += term
        ref = O.graph_value_bruteforce(gr, u, f)
        assert val == pytest.approx(ref, rel=1e-11, abs=1e-11)


def _rotation(g):
    q, r = np.linalg.qr(g.normal(size=(3, 3)))
    q *= np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


@pytest.mark.parametrize("level", [16, 20])
def test_every_basis_function_is_rotation_invariant(level):
    graphs = O.connected_graphs(level)
    bases = O.basis_functions(level, graphs)
    g = synth.rng(7, level)
    u = g.normal(size=(2, 9, 3))
    u /= np.linalg.norm(u, axis=-1, keepdims=True)
    f = g.normal(size=(2, 9, O.n_mu_for_level(level)))
    rot = _rotation(g)
    b0 = O.free_basis_rows(graphs, bases, u, f)
    b1 = O.free_basis_rows(graphs, bases, u @ rot.T, f)
    assert np.allclose(b0, b1, rtol=1e-11, atol=1e-11 * np.abs(b0).max())
    # a reflection as well (O(3) invariance of full contractions)
    b2 = O.free_basis_rows(graphs, bases, -u, f)
    assert np.allclose(b0, b2, rtol=1e-11, atol=1e-11 * np.abs(b0).max())


def test_cayley_hamilton_dependency_is_the_one_pruned_at_level16():
    """For unit vectors tr M02 = M00, and Cayley-Hamilton for a symmetric 3x3
    matrix gives tr(M02^4) = p1 p3 - (p1^2 - p2) p2 / 2 + p1 (p1^3 - 3 p1 p2 + 2 p3) / 6
    with p1 = M00, p2 = M02:M02, p3 = tr(M02^3)."""
    g = synth.rng(8, 0)
    for _ in range(5):
        u = g.normal(size=(11, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        f = g.normal(size=11)
        m02 = np.einsum("j,ja,jb->ab", f, u, u)
        p1, p2, p3 = f.sum(), np.sum(m02 * m02), np.trace(m02 @ m02 @ m02)
        lhs = np.trace(np.linalg.matrix_power(m02, 4))
        rhs = p1 * p3 - (p1 ** 2 - p2) * p2 / 2 + p1 * (p1 ** 3 - 3 * p1 * p2 + 2 * p3) / 6
        assert lhs == pytest.approx(rhs, rel=1e-12)
    graphs = O.connected_graphs(16)
    allb = O.basis_functions(16, graphs)
    u, f = synth.random_neighbourhoods(3 * len(allb), 12, 4, synth.rng(99, 16))
    kept = set(O.prune_dependent(O.free_basis_rows(graphs, allb, u, f)))
    dropped = [allb[k] for k in range(len(allb)) if k not in kept]
    assert len(dropped) == 1
    (b,) = dropped
    # Basis order puts lower levels first and, within a level, fewer factors
    # first, so of the five functions in the identity (levels 8, 12, 14, 16, 16)
    # the greedy pass drops the last one: (M02:M02)^2 = p2^2.
    assert len(b) == 2 and b[0] == b[1]
    gr = graphs[b[0]]
    assert gr.mu == (0, 0) and gr.e == (2,)


@pytest.mark.parametrize("level", [16, 20])
def test_pruned_columns_are_dependent_and_kept_ones_independent(level):
    """Checked on a second, independent set of random neighbourhoods."""
    graphs = O.connected_graphs(level)
    allb = O.basis_functions(level, graphs)
    n_mu = O.n_mu_for_level(level)
    u, f = synth.random_neighbourhoods(3 * len(allb), 12, n_mu, synth.rng(99, level))
    kept = O.prune_dependent(O.free_basis_rows(graphs, allb, u, f))
    u2, f2 = synth.random_neighbourhoods(2 * len(allb), 14, n_mu, synth.rng(98, level))
    rows = O.free_basis_rows(graphs, allb, u2, f2)
    rows /= np.linalg.norm(rows, axis=0, keepdims=True)
    a = rows[:, kept]
    s = np.linalg.svd(a, compute_uv=False)
    assert s.min() > 1e-7 * s.max()
    drop = [k for k in range(len(allb)) if k not in set(kept)]
    coef, *_ = np.linalg.lstsq(a, rows[:, drop], rcond=None)
    assert np.abs(a @ coef - rows[:, drop]).max() < 1e-9


def test_potential_files_carry_the_oracle_basis():
    from oracle.make_potentials import oracle_basis, encode_basis
    for name, level in [("bcc-l8-s1", 8), ("bcc-l16-s3", 16)]:
        assert pot_file(name)["basis"] == encode_basis(oracle_basis(level))


# --------------------------------------------------------------------------- neighbour list


def test_lattice_shell_counts():
    st = synth.crystal("bcc", (4, 4, 4), 3.16, 0.0, 1, 1)
    i, _, _ = O.neighbor_list(st.x, st.cell, st.pbc, 5.0)
    assert np.all(np.bincount(i, minlength=st.n) == 26)     # 8 + 6 + 12
    st = synth.crystal("fcc", (3, 3, 3), 3.6, 0.0, 1, 1)
    i, _, _ = O.neighbor_list(st.x, st.cell, st.pbc, 5.5)
    assert np.all(np.bincount(i, minlength=st.n) == 54)     # 12 + 6 + 24 + 12


def test_neighbor_list_matches_explicit_supercell():
    """Small triclinic cell: every (j, n) pair equals a pair in an explicit
    replicated supercell with open boundaries."""
    g = synth.rng(9, 0)
    st = synth.random_gas(6, 0.085, 1.9, 1, g)
    rc = 5.0
    i, j, n = O.neighbor_list(st.x, st.cell, st.pbc, rc)
    pairs = set(zip(i.tolist(), j.tolist(), map(tuple, n.tolist())))
    reach = 4
    ref = set()
    for a in range(st.n):
        for b in range(st.n):
            for nn in itertools.product(range(-reach, reach + 1), repeat=3):
                d = st.x[b] + np.array(nn) @ st.cell - st.x[a]
                r = math.sqrt(d @ d)
                if 0 < r < rc:
                    ref.add((a, b, nn))
    assert pairs == ref


# --------------------------------------------------------------------------- energies


def test_level2_dimer_closed_form():
    """Level 2: one basis function B = M00 = sum_j f_0(r_ij), a pair potential.
    Two atoms at distance d in open space: E = 2 s + 2 xi f0(d) and the force
    on atom 1 along the bond is -2 xi f0'(d), with f0 and f0' written from
    T_k(cos t) = cos(k t) and T_k'(cos t) = k sin(k t) / sin(t)."""
    model = random_model(2, 1, stream=11)
    c = model.pot.radial[0, :, 0, 0]
    s = model.pot.species_energy[0]
    xi = model.pot.xi[0]
    rmin, rc = 2.0, 5.0
    for d in [2.3, 3.1, 4.4]:
        x = np.array([[0.0, 0.0, 0.0], [d, 0.0, 0.0]])
        cell = np.eye(3) * 50.0
        nl = O.neighbor_list(x, cell, (0, 0, 0), rc)
        out = O.evaluate(model, x, np.zeros(2, np.int32), cell, nl)
        t = math.acos((2 * d - rmin - rc) / (rc - rmin))
        f0 = sum(c[k] * math.cos(k * t) for k in range(8)) * (rc - d) ** 2
        dT = [k * math.sin(k * t) / math.sin(t) for k in range(8)]
        df0 = sum(c[k] * (dT[k] * 2 / (rc - rmin) * (rc - d) ** 2 - math.cos(k * t) * 2 * (rc - d)) for k in range(8))
        assert out["e"] == pytest.approx(2 * s + 2 * xi * f0, rel=1e-13)
        assert out["f"][1, 0] == pytest.approx(-2 * xi * df0, rel=1e-11)
        assert out["f"][0, 0] == pytest.approx(2 * xi * df0, rel=1e-11)


def test_level8_trimer_hand_formula():
    """Three atoms; site energy of atom 0 from the nine level-8 basis functions
    written out by hand in terms of f_mu and bond angles."""
    model = random_model(8, 1, stream=12)
    x = np.array([[0.0, 0.0, 0.0], [2.6, 0.3, -0.2], [-0.4, 2.9, 0.5]])
    cell = np.eye(3) * 50
    nl = O.neighbor_list(x, cell, (0, 0, 0), 5.0)
    out = O.evaluate(model, x, np.zeros(3, np.int32), cell, nl, want=("e",))
    c = model.pot.radial[:, :, 0, 0]
    vecs = [x[1] - x[0], x[2] - x[0]]
    rs = [np.linalg.norm(v) for v in vecs]
    us = [v / r for v, r in zip(vecs, rs)]
    f = [[sum(c[mu, k] * q for k, q in enumerate(O.radial_basis(r, 2.0, 5.0, 8))) for r in rs] for mu in range(2)]
    cos = us[0] @ us[1]
    m00 = f[0][0] + f[0][1]
    m10 = f[1][0] + f[1][1]
    m01m01 = f[0][0] ** 2 + f[0][1] ** 2 + 2 * f[0][0] * f[0][1] * cos
    m02m02 = f[0][0] ** 2 + f[0][1] ** 2 + 2 * f[0][0] * f[0][1] * cos ** 2
    vals = {((0,), ()): m00, ((1,), ()): m10, ((0, 0), (1,)): m01m01, ((0, 0), (2,)): m02m02}
    graphs = model.basis.graphs
    e0 = model.pot.species_energy[0]
    for a, b in enumerate(model.basis.bases):
        term = model.pot.xi[a]
        for k in b:
            term *= vals[(graphs[k].mu, graphs[k].e)]
        e0 += term
    assert out["e_atom"][0] == pytest.approx(e0, rel=1e-12)


def _small(name, cells=(2, 2, 2), stream=21):
    pot = pot_file(name)
    model = O.load_model(pot)
    kind = "fcc" if name.startswith("fcc") else "bcc"
    a = 3.6 if kind == "fcc" else 3.16
    st = synth.crystal(kind, cells, a, 0.1, pot["n_species"], stream)
    return model, st, pot["r_cut"]


def test_forces_and_virial_match_central_differences():
    model, st, rc = _small("bcc-l16-s3")
    nl = O.neighbor_list(st.x, st.cell, st.pbc, rc)
    out = O.evaluate(model, st.x, st.z, st.cell, nl)
    h = 1e-5

    def energy(x, cell):
        return O.evaluate(model, x, st.z, cell, O.neighbor_list(x, cell, st.pbc, rc), want=("e",))["e"]

    g = synth.rng(10, 0)
    for _ in range(4):
        a, c = int(g.integers(st.n)), int(g.integers(3))
        xp, xm = st.x.copy(), st.x.copy()
        xp[a, c] += h
        xm[a, c] -= h
        fd = -(energy(xp, st.cell) - energy(xm, st.cell)) / (2 * h)
        assert out["f"][a, c] == pytest.approx(fd, rel=1e-6, abs=1e-6)
    for p, q in [(0, 0), (1, 2), (2, 0)]:
        e = np.zeros((3, 3))
        e[p, q] = h
        fp = energy(st.x @ (np.eye(3) + e).T, st.cell @ (np.eye(3) + e).T)
        fm = energy(st.x @ (np.eye(3) - e).T, st.cell @ (np.eye(3) - e).T)
        assert out["w_full"][p, q] == pytest.approx(-(fp - fm) / (2 * h), rel=1e-6, abs=1e-6)
    assert np.abs(out["f"].sum(axis=0)).max() < 1e-10 * np.abs(out["f"]).max() * st.n
    w = out["w_full"]
    assert np.allclose(w, w.T, rtol=1e-11, atol=1e-11 * np.abs(w).max())


def test_cluster_virial_equals_position_force_sum():
    model, st, rc = _small("bcc-l8-s1")
    cell = st.cell * 4.0          # open boundaries: atoms do not see images
    nl = O.neighbor_list(st.x, cell, (0, 0, 0), rc)
    out = O.evaluate(model, st.x, st.z, cell, nl)
    w = np.einsum("ia,ib->ab", out["f"], st.x)
    assert np.allclose(out["w_full"], w, rtol=1e-11, atol=1e-11 * np.abs(w).max())


def test_translation_permutation_wrap_invariance():
    model, st, rc = _small("bcc-l16-s3", stream=22)
    nl = O.neighbor_list(st.x, st.cell, st.pbc, rc)
    ref = O.evaluate(model, st.x, st.z, st.cell, nl, want=("e",))
    # translation (then wrap back into the cell)
    x2 = synth.wrap(st.x + np.array([0.37, -1.2, 2.9]), st.cell)
    e2 = O.evaluate(model, x2, st.z, st.cell, O.neighbor_list(x2, st.cell, st.pbc, rc), want=("e",))
    assert np.allclose(e2["e_atom"], ref["e_atom"], rtol=1e-11, atol=1e-11)
    # unwrapped positions (one atom moved by a lattice vector)
    x3 = st.x.copy()
    x3[3] += st.cell[1] - st.cell[2]
    e3 = O.evaluate(model, x3, st.z, st.cell, O.neighbor_list(x3, st.cell, st.pbc, rc), want=("e",))
    assert np.allclose(e3["e_atom"], ref["e_atom"], rtol=1e-11, atol=1e-11)
    # permutation of atoms
    p = synth.rng(11, 0).permutation(st.n)
    e4 = O.evaluate(model, st.x[p], st.z[p], st.cell, O.neighbor_list(st.x[p], st.cell, st.pbc, rc), want=("e",))
    assert np.allclose(e4["e_atom"], ref["e_atom"][p], rtol=1e-11, atol=1e-11)


def test_supercell_extensivity():
    """Replicating a small triclinic periodic cell 2x2x2 replicates every site
    energy and multiplies E by 8 (pins multi-image handling)."""
    model = O.load_model(pot_file("gas-l16-s2"))
    st = synth.random_gas(10, 0.085, 1.9, 2, synth.rng(12, 0))
    rc = 5.0
    nl = O.neighbor_list(st.x, st.cell, st.pbc, rc)
    e1 = O.evaluate(model, st.x, st.z, st.cell, nl, want=("e",))
    shifts = np.array(list(itertools.product(range(2), repeat=3)))
    x8 = np.concatenate([st.x + s @ st.cell for s in shifts])
    z8 = np.concatenate([st.z] * 8)
    cell8 = st.cell * 2
    e8 = O.evaluate(model, x8, z8, cell8, O.neighbor_list(x8, cell8, st.pbc, rc), want=("e",))
    assert np.allclose(e8["e_atom"], np.tile(e1["e_atom"], 8), rtol=1e-10, atol=1e-10)
    assert e8["e"] == pytest.approx(8 * e1["e"], rel=1e-11)


def test_parameter_gradient_identities():
    """dE/ds_z = N_z; dE/dxi_alpha = sum_i B_alpha(i); Euler homogeneity:
    sum c dE/dc = sum_alpha deg_alpha xi_alpha sum_i B_alpha(i)."""
    model, st, rc = _small("bcc-l16-s3", stream=23)
    nl = O.neighbor_list(st.x, st.cell, st.pbc, rc)
    out = O.evaluate(model, st.x, st.z, st.cell, nl, want=("e", "dtheta"))
    assert np.array_equal(out["dE_ds"], np.bincount(st.z, minlength=3).astype(float))
    b = O.basis_matrix(model, st.x, st.z, st.cell, nl)
    assert np.allclose(out["dE_dxi"], b.sum(0), rtol=1e-12, atol=1e-12)
    deg = np.array([sum(model.basis.graphs[k].nv for k in bb) for bb in model.basis.bases])
    lhs = np.sum(model.pot.radial * out["dE_dc"])
    rhs = np.sum(deg * model.pot.xi * b.sum(0))
    assert lhs == pytest.approx(rhs, rel=1e-10)


def test_parameter_gradient_matches_finite_differences():
    model, st, rc = _small("bcc-l8-s1", stream=24)
    nl = O.neighbor_list(st.x, st.cell, st.pbc, rc)
    out = O.evaluate(model, st.x, st.z, st.cell, nl, want=("e", "dtheta"))
    h = 1e-5
    for idx in [(0, 0, 0, 0), (1, 3, 0, 0), (0, 7, 0, 0)]:
        c0 = model.pot.radial.copy()
        vals = []
        for sgn in (1, -1):
            c = c0.copy()
            c[idx] += sgn * h
            model.c = torch.as_tensor(c)
            vals.append(O.evaluate(model, st.x, st.z, st.cell, nl, want=("e",))["e"])
        model.c = torch.as_tensor(c0)
        assert out["dE_dc"][idx] == pytest.approx((vals[0] - vals[1]) / (2 * h), rel=1e-6, abs=1e-7)


def test_force_matching_double_backward_matches_finite_differences():
    """Loss l = (1/3N) sum |F - F_t|^2; dl/dtheta from the double backward
    against central differences of l in theta (h = 1e-5)."""
    pot = pot_file("fcc-l20-s4")
    model = O.load_model(pot)
    st = synth.crystal("fcc", (1, 1, 2), 3.6, 0.1, 4, 3)
    rc = pot["r_cut"]
    nl = O.neighbor_list(st.x, st.cell, st.pbc, rc)
    ft = synth.target_forces(st.n, 3)
    loss, grads = O.force_matching_grad(model, st.x, st.z, st.cell, nl, ft)
    h = 1e-5

    def loss_at():
        f = O.evaluate(model, st.x, st.z, st.cell, nl, want=("f",))["f"]
        return float(((f - ft) ** 2).sum() / (3 * st.n))

    assert loss == pytest.approx(loss_at(), rel=1e-13)
    assert np.all(grads[0] == 0.0)      # species energies do not enter forces
    checks = [("xi", 0), ("xi", 57), ("xi", 301), ("c", (0, 1, 2, 3)), ("c", (4, 9, 1, 1)), ("c", (2, 0, 3, 0))]
    for which, idx in checks:
        p = model.xi if which == "xi" else model.c
        g = grads[2] if which == "xi" else grads[1]
        base = p.clone()
        vals = []
        for sgn in (1, -1):
            q = base.clone()
            q[idx] += sgn * h
            if which == "xi":
                model.xi = q
            else:
                model.c = q
            vals.append(loss_at())
        if which == "xi":
            model.xi = base
        else:
            model.c = base
        assert g[idx] == pytest.approx((vals[0] - vals[1]) / (2 * h), rel=2e-5, abs=1e-7)


@pytest.mark.slow
def test_nve_energy_error_scales_with_dt_squared():
    """Velocity Verlet on a 16-atom box with oracle forces: the total-energy
    fluctuation shrinks about 4x when dt halves, and shows no drift."""
    model = O.load_model(pot_file("bcc-l8-s1"))
    st = synth.crystal("bcc", (2, 2, 2), 3.16, 0.02, 1, 31)
    rc = 5.0
    mass = 183.84 * 1.0364269e-4          # amu -> eV ps^2 / A^2
    kb = 8.617333e-5
    v0 = synth.rng(31, 5).normal(0, math.sqrt(kb * 10.0 / mass), size=(st.n, 3))
    v0 -= v0.mean(0)

    def run(dt, steps):
        x, v = st.x.copy(), v0.copy()
        out = O.evaluate(model, x, st.z, st.cell, O.neighbor_list(x, st.cell, st.pbc, rc), want=("e", "f"))
        f = out["f"]
        etot = []
        for _ in range(steps):
            v = v + 0.5 * dt * f / mass
            x = x + dt * v
            out = O.evaluate(model, x, st.z, st.cell, O.neighbor_list(x, st.cell, st.pbc, rc), want=("e", "f"))
            f = out["f"]
            v = v + 0.5 * dt * f / mass
            etot.append(out["e"] + 0.5 * mass * (v * v).sum())
        return np.array(etot)

    e1 = run(2e-3, 100)
    e2 = run(1e-3, 200)
    fl1 = e1.max() - e1.min()
    fl2 = e2.max() - e2.min()
    assert 2.8 < fl1 / fl2 < 5.5
    # no secular drift: the change of the mean energy between the first and the
    # last quarter of the run stays well inside the bounded oscillation
    q = len(e2) // 4
    drift = abs(e2[-q:].mean() - e2[:q].mean())
    assert drift < 0.5 * fl2


def test_metal_unit_constant_from_si_values():
    """1 amu (A/ps)^2 in eV from the SI definitions (CODATA 2018 atomic mass
    constant, exact elementary charge): the oracle's kinetic-energy constant."""
    amu_kg = 1.66053906660e-27
    j = amu_kg * (1e-10 / 1e-12) ** 2
    assert O.AMU_A2_PS2_IN_EV == pytest.approx(j / 1.602176634e-19, rel=1e-7)


def _md_start(seed, temperature=300.0, cells=(2, 2, 2)):
    st = synth.crystal("bcc", cells, 3.16, 0.03, 1, seed)
    mass = 183.84
    kt = 8.617333e-5 * temperature
    v = synth.rng(seed, 5).normal(0, math.sqrt(kt / (mass * O.AMU_A2_PS2_IN_EV)), size=(st.n, 3))
    v -= v.mean(0)
    return st, v, [mass]


def test_velocity_verlet_free_flight_is_exact():
    """With every xi = 0 the forces vanish: x_n = x_0 + n dt v_0, v and the
    energies stay constant (the potential energy is sum_i s[z_i])."""
    model = O.load_model(pot_file("bcc-l8-s1"))
    model.xi = torch.zeros_like(model.xi)
    st, v0, masses = _md_start(41)
    dt, n = 1e-3, 4
    x, v, f, e_pot, e_kin = O.velocity_verlet(model, st.x, v0, st.z, st.cell, st.pbc, masses, dt, n)
    assert np.abs(f).max() == 0.0
    assert np.allclose(x, st.x + n * dt * v0, rtol=0, atol=1e-12)
    assert np.array_equal(v, v0)
    s = float(model.s[0]) * st.n
    assert np.allclose(e_pot, s, rtol=1e-14)
    ke = 0.5 * masses[0] * O.AMU_A2_PS2_IN_EV * (v0 * v0).sum()
    assert np.allclose(e_kin, ke, rtol=1e-14)


def test_velocity_verlet_is_time_reversible_and_conserves_momentum():
    """Velocity Verlet is symmetric: n steps, reversed velocities, n steps
    return to the start; the total momentum stays constant (sum F = 0)."""
    model = O.load_model(pot_file("bcc-l8-s1"))
    st, v0, masses = _md_start(42)
    dt, n = 1e-3, 6
    x1, v1, f1, _, _ = O.velocity_verlet(model, st.x, v0, st.z, st.cell, st.pbc, masses, dt, n)
    assert np.abs(x1 - st.x).max() > 1e-3           # it moved
    assert np.abs(v1.sum(0) - v0.sum(0)).max() < 1e-10
    x2, v2, _, _, _ = O.velocity_verlet(model, x1, -v1, st.z, st.cell, st.pbc, masses, dt, n, f=f1)
    assert np.abs(x2 - st.x).max() < 1e-10
    assert np.abs(v2 + v0).max() < 1e-8


@pytest.mark.slow
def test_velocity_verlet_energy_error_scales_with_dt_squared():
    """The oracle integrator's total-energy fluctuation shrinks about 4x when
    dt halves (second order), with no secular drift."""
    model = O.load_model(pot_file("bcc-l8-s1"))
    st, v0, masses = _md_start(43, temperature=50.0)

    def etot(dt, n):
        _, _, _, e_pot, e_kin = O.velocity_verlet(model, st.x, v0, st.z, st.cell, st.pbc, masses, dt, n)
        return e_pot + e_kin

    e1 = etot(2e-3, 40)
    e2 = etot(1e-3, 80)
    ratio = (e1.max() - e1.min()) / (e2.max() - e2.min())
    assert 2.8 < ratio < 5.5


# --------------------------------------------------------------------------- grade and MaxVol


def test_maxvol_dominance_and_active_rows_have_unit_grade():
    g = synth.rng(13, 0)
    pool = g.normal(size=(300, 12)) * np.exp(g.normal(size=12))
    rows, a_inv, _ = O.maxvol(pool, delta=0.01)
    gam = O.grade(pool, a_inv)
    assert gam.max() <= 1.01 + 1e-12
    assert np.allclose(gam[rows], 1.0, atol=1e-12)
    assert np.allclose(O.invert(pool[rows]), np.linalg.inv(pool[rows]), rtol=1e-9, atol=1e-9)
    # column scaling invariance: B -> B D, A -> A D
    d = np.exp(g.normal(size=12))
    gam2 = O.grade(pool * d, O.invert(pool[rows] * d))
    assert np.allclose(gam, gam2, rtol=1e-10)


def test_maxvol_reaches_a_dominant_set_found_by_brute_force():
    """Tiny pool: the set MaxVol returns with delta = 0 is dominant, i.e. no
    single-row swap increases |det A| (checked by trying every swap)."""
    g = synth.rng(14, 0)
    pool = g.normal(size=(9, 3))
    rows, _, _ = O.maxvol(pool, delta=0.0)
    vol = abs(np.linalg.det(pool[rows]))
    for k in range(3):
        for i in range(9):
            r2 = rows.copy()
            r2[k] = i
            assert abs(np.linalg.det(pool[r2])) <= vol * (1 + 1e-12)
    best = max(abs(np.linalg.det(pool[list(c)])) for c in itertools.combinations(range(9), 3))
    assert vol >= best / 3 ** 1.5 - 1e-12   # dominant submatrix bound (Goreinov et al. 2010)


def test_invert_pivots_and_matches_closed_forms():
    """Gauss-Jordan with partial pivoting: a permutation (zero diagonal, so
    pivoting is required) is its own transpose inverse, exactly; a 2 x 2
    matrix against the adjugate formula; a singular matrix is refused."""
    perm = np.array([[0.0, 1.0, 0.0], [0.0, 0.0, 1.0], [1.0, 0.0, 0.0]])
    assert np.array_equal(O.invert(perm), perm.T)
    a = np.array([[3.0, -2.0], [5.0, 7.0]])
    adj = np.array([[7.0, 2.0], [-5.0, 3.0]]) / (3.0 * 7.0 + 2.0 * 5.0)
    assert np.allclose(O.invert(a), adj, rtol=1e-15, atol=1e-16)
    with pytest.raises(np.linalg.LinAlgError):
        O.invert(np.array([[1.0, 2.0], [0.0, 0.0]]))


def test_initial_rows_greedy_order_on_orthogonal_rows():
    """On rows that are orthogonal with distinct norms the greedy start takes
    them by decreasing norm; rows in the span of those already taken (here a
    scaled copy) are never taken while independent rows remain."""
    q, _ = np.linalg.qr(synth.rng(15, 0).normal(size=(5, 5)))
    norms = np.array([3.0, 7.0, 1.0, 5.0, 2.0])
    pool = np.vstack([q * norms[:, None], 10.0 * q[2]])   # row 5: a longer copy of row 2's direction
    rows = O.initial_rows(pool)
    assert rows.tolist() == [5, 1, 3, 0, 4]
    assert abs(np.linalg.det(pool[rows])) > 0


def test_maxvol_ties_go_to_the_lowest_row():
    """Two identical pool rows dominate: the swap takes the lower index."""
    pool = np.array([[1.0, 0.0], [0.0, 1.0], [5.0, 0.5], [5.0, 0.5], [0.2, 0.1]])
    rows, _, it = O.maxvol(pool, rows=np.array([0, 1]), delta=0.0)
    assert it >= 1 and 2 in rows.tolist() and 3 not in rows.tolist()


def test_grade_flags():
    gam = np.array([0.5, 2.0, 2.0000001, 9.99, 10.0, 10.5])
    assert O.grade_flags(gam, 2.0, 10.0).tolist() == [0, 0, 1, 1, 1, 3]


def test_berendsen_with_infinite_tau_is_velocity_verlet():
    """With tau_p so long that the scale factor rounds to 1, the NPT
    integrator is the NVE one bit for bit and the cell does not move."""
    model = O.load_model(pot_file("bcc-l8-s1"))
    st, v0, masses = _md_start(43)
    dt, n = 1e-3, 3
    x1, v1, f1, _, _ = O.velocity_verlet(model, st.x, v0, st.z, st.cell, st.pbc, masses, dt, n)
    x2, v2, f2, cell2, _ = O.berendsen_npt(model, st.x, v0, st.z, st.cell, st.pbc, masses, dt, n, 1.0, 1e300)
    assert np.array_equal(x1, x2) and np.array_equal(v1, v2) and np.array_equal(f1, f2)
    assert np.array_equal(cell2, st.cell)


def test_pressure_virial_term_is_minus_dE_dV():
    """For a static configuration the pressure is -dE/dV under isotropic
    scaling of the cell and positions (central differences in the volume)."""
    model = O.load_model(pot_file("bcc-l8-s1"))
    st = synth.crystal("bcc", (3, 3, 3), 3.16, 0.08, 1, 44)
    r_cut = model.pot.r_cut
    out = O.evaluate(model, st.x, st.z, st.cell, O.neighbor_list(st.x, st.cell, st.pbc, r_cut), want=("e", "w"))
    p = O.pressure_bar(0.0, out["w"], st.cell) / O.EV_PER_A3_IN_BAR
    h = 1e-5
    ev = []
    for s in (1 + h, 1 - h):
        x, c = st.x * s, st.cell * s
        e = O.evaluate(model, x, st.z, c, O.neighbor_list(x, c, st.pbc, r_cut), want=("e",))["e"]
        ev.append((e, abs(np.linalg.det(c))))
    p_fd = -(ev[0][0] - ev[1][0]) / (ev[0][1] - ev[1][1])
    assert p == pytest.approx(p_fd, rel=1e-6, abs=1e-9)


def test_berendsen_ideal_gas_relaxes_to_the_ideal_gas_volume():
    """With every xi = 0 (no forces, zero virial) the atoms fly freely and the
    pressure is the kinetic 2 E_kin / (3 V); the barostat drives the volume to
    V* = 2 E_kin / (3 p_target), the ideal-gas law written in SI units."""
    model = O.load_model(pot_file("bcc-l8-s1"))
    model.xi = torch.zeros_like(model.xi)
    st, v0, masses = _md_start(45, temperature=600.0)
    p_target = 2000.0   # bar
    dt, tau = 1e-3, 1e-2
    x, v, f, cell, pr = O.berendsen_npt(model, st.x, v0, st.z, st.cell, st.pbc, masses, dt, 150, p_target, tau,
                                        bulk_modulus=p_target)
    ke_j = 0.5 * masses[0] * 1.66053906660e-27 * ((v0 * 1e2) ** 2).sum()   # A/ps = 100 m/s
    v_star = 2.0 * ke_j / (3.0 * p_target * 1e5) * 1e30                    # A^3
    assert np.array_equal(v, v0)
    assert abs(np.linalg.det(cell)) == pytest.approx(v_star, rel=1e-6)
    assert pr[-1] == pytest.approx(p_target, rel=1e-6)


def test_independent_columns_on_known_rank():
    """A 12 x 6 matrix whose columns 4 and 5 are combinations of columns 0-2:
    four columns are independent, and every dropped column is reproduced by
    the kept ones to rounding."""
    g = np.random.default_rng(5)
    a = g.normal(size=(12, 6))
    a[:, 4] = 2.0 * a[:, 0] - a[:, 2]
    a[:, 5] = 0.5 * a[:, 1] + 3.0 * a[:, 0]
    cols = O.independent_columns(a)
    assert len(cols) == 4
    for k in set(range(6)) - set(cols):
        coef, *_ = np.linalg.lstsq(a[:, cols], a[:, k], rcond=None)
        assert np.abs(a[:, cols] @ coef - a[:, k]).max() <= 1e-12 * np.abs(a[:, k]).max()


def test_parameter_gradient_has_the_radial_mixing_relations():
    """dE/dtheta of any set of configurations satisfies n_mu (n_mu + 1) / 2
    exact linear relations: E is unchanged to first order when f_mu gains a
    multiple of f_nu (nu <= mu; nu = mu is a scaling) and xi compensates.
    At level 8 (n_mu = 2) the independent columns of a pool of 40 strained
    16-atom BCC cells number n_params - 3."""
    model = O.load_model(pot_file("bcc-l8-s1"))
    rows = []
    g = synth.rng(31, 61)
    for k in range(40):
        st = synth.crystal("bcc", (2, 2, 2), 3.16, 0.05, 1, 31, sub=100 + k)
        d = np.diag(1.0 + g.uniform(-0.02, 0.02, size=3))
        x, cell = st.x @ d, st.cell @ d
        out = O.evaluate(model, x, st.z, cell, O.neighbor_list(x, cell, st.pbc, model.pot.r_cut),
                         want=("e", "dtheta"))
        rows.append(np.concatenate([out["dE_ds"], out["dE_dc"].ravel(), out["dE_dxi"]]))
    rows = np.array(rows)
    n_mu = model.pot.radial.shape[0]
    assert len(O.independent_columns(rows)) == rows.shape[1] - n_mu * (n_mu + 1) // 2
