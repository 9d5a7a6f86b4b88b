"""Oracle: a plain, slow, FP64 CPU reference of Moment Tensor Potential evaluation.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls or
executes this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library.

What it computes.  The paper (Sec. 1 and Sec. 2.2) evaluates the Moment Tensor
Potential of Shapeev 2016 as extended in MLIP-2/MLIP-3 (the works it cites for
the model) and reports energies, forces and stresses plus an extrapolation grade
(Sec. 2.1).  The paper prints no equation; this file restates the published
definition, written for readability rather than speed:

* neighbours: every (j, n) with r_ij = x_j + n.H - x_i and 0 < |r_ij| < R_cut,
  n an integer image vector on periodic axes (a full list, self images kept);
* radial basis: Q_k(r) = T_k(xi(r)) (R_cut - r)^2, xi = (2r - R_min - R_cut) /
  (R_cut - R_min), T_k Chebyshev polynomials of the first kind by the
  three-term recurrence (also used below R_min: no clamping);
* radial functions: f_mu(r) = sum_k c[mu, k, z_i, z_j] Q_k(r);
* moment tensors: M_{mu,nu}(i) = sum_j f_mu(|r_ij|) rhat_ij^{(x) nu}, with
  level 2 + 4 mu + nu;
* basis functions B_alpha: products of connected contraction graphs of moment
  tensors (each edge contracts one index pair, no self loops), total level <= L;
* site energy E_i = s[z_i] + sum_alpha xi_alpha B_alpha(i), E = sum_i E_i;
* forces F = -dE/dx, virial W = -dE/d(strain) (6 components xx yy zz xy xz yz);
* extrapolation grade gamma_i = max_k |(b_i A^-1)_k| with b_i the basis row
  of atom i and A the active set, selected by MaxVol (Goreinov et al. 2010).

Forms used: a tensor form (explicit 3^nu Cartesian arrays, contracted with
einsum over Cartesian indices), a graph form (brute-force sum over neighbour
tuples, tiny neighbourhoods only) and torch.autograd for every derivative.
Every function is pinned by tests against something other than itself: closed
forms, finite differences, invariances, brute force and hand-derived counts.
"""
from __future__ import annotations

import dataclasses
import itertools
import math
from collections import Counter

import numpy as np
import torch

DT = torch.float64

# ---------------------------------------------------------------------------
# Radial basis (Shapeev 2016 Sec. 2 / MLIP-2: Chebyshev basis times (R_c - r)^2)
# ---------------------------------------------------------------------------


def chebyshev(xi, n: int):
    """T_0..T_{n-1} at xi by T_0 = 1, T_1 = xi, T_{k+1} = 2 xi T_k - T_{k-1}."""
    t = [xi * 0 + 1, xi]
    for k in range(2, n):
        t.append(2 * xi * t[k - 1] - t[k - 2])
    return t[:n]


def radial_basis(r, r_min: float, r_cut: float, n_q: int):
    """Q_k(r) = T_k(xi) (R_cut - r)^2 for k < n_q; returns a list of n_q arrays."""
    xi = (2 * r - (r_min + r_cut)) / (r_cut - r_min)
    cut = (r_cut - r) ** 2
    return [tk * cut for tk in chebyshev(xi, n_q)]


# ---------------------------------------------------------------------------
# Basis enumeration: connected contraction graphs and their products
# ---------------------------------------------------------------------------


def moment_level(mu: int, nu: int) -> int:
    """Level of M_{mu,nu} (MLIP convention): 2 + 4 mu + nu."""
    return 2 + 4 * mu + nu


def n_mu_for_level(level: int) -> int:
    """Radial functions admitted by the level: every mu with 2 + 4 mu <= L."""
    return (level - 2) // 4 + 1


@dataclasses.dataclass(frozen=True)
class Graph:
    """Connected contraction graph.  ``mu[v]`` labels vertex v; ``e`` is the
    upper triangle (row-major, v<w) of the edge multiplicity matrix.  Vertex
    v stands for the moment tensor M_{mu[v], nu[v]} with nu[v] = sum_w e_vw."""
    mu: tuple
    e: tuple

    @property
    def nv(self) -> int:
        return len(self.mu)

    def mult(self, v: int, w: int) -> int:
        if v == w:
            return 0
        a, b = min(v, w), max(v, w)
        k = a * self.nv - a * (a + 1) // 2 + (b - a - 1)
        return self.e[k]

    @property
    def nu(self) -> tuple:
        return tuple(sum(self.mult(v, w) for w in range(self.nv)) for v in range(self.nv))

    @property
    def level(self) -> int:
        return sum(moment_level(m, n) for m, n in zip(self.mu, self.nu))

    @property
    def sort_key(self) -> tuple:
        return (self.level, self.mu, self.e)


def _upper(mat) -> tuple:
    n = len(mat)
    return tuple(mat[v][w] for v in range(n) for w in range(v + 1, n))


def _is_connected(mat) -> bool:
    n = len(mat)
    seen, stack = {0}, [0]
    while stack:
        v = stack.pop()
        for w in range(n):
            if mat[v][w] and w not in seen:
                seen.add(w)
                stack.append(w)
    return len(seen) == n


def canonical_graph(mu, mat) -> Graph:
    """Smallest (mu tuple, upper-triangle tuple) over all vertex orderings."""
    n = len(mu)
    best = None
    for p in itertools.permutations(range(n)):
        key = (tuple(mu[p[a]] for a in range(n)),
               tuple(mat[p[a]][p[b]] for a in range(n) for b in range(a + 1, n)))
        if best is None or key < best:
            best = key
    return Graph(*best)


def connected_graphs(level: int) -> list:
    """All connected, loopless, vertex-labelled multigraphs with total level <= L,
    up to isomorphism, sorted by (level, mu tuple, e tuple)."""
    n_mu = n_mu_for_level(level)
    found = set()
    # level = 2V + 4 sum(mu) + 2|E| and |E| >= V - 1 for a connected graph
    for nv in range(1, (level + 2) // 4 + 1):
        pairs = [(v, w) for v in range(nv) for w in range(v + 1, nv)]
        max_edges = (level - 2 * nv) // 2
        for mults in itertools.product(range(max_edges + 1), repeat=len(pairs)):
            n_edges = sum(mults)
            if n_edges > max_edges:
                continue
            mat = [[0] * nv for _ in range(nv)]
            for (v, w), k in zip(pairs, mults):
                mat[v][w] = mat[w][v] = k
            if nv > 1 and not _is_connected(mat):
                continue
            spare = level - 2 * nv - 2 * n_edges
            for mu in itertools.product(range(n_mu), repeat=nv):
                if 4 * sum(mu) <= spare:
                    found.add(canonical_graph(mu, mat))
    return sorted(found, key=lambda g: g.sort_key)


def basis_functions(level: int, graphs=None) -> list:
    """Every multiset of connected graphs with total level <= L, as sorted
    tuples of graph indices, in order (level, factor count, factor sort keys)."""
    graphs = graphs if graphs is not None else connected_graphs(level)
    out = []

    def grow(start, chosen, lev):
        if chosen:
            out.append(tuple(chosen))
        for k in range(start, len(graphs)):
            if lev + graphs[k].level <= level:
                chosen.append(k)
                grow(k, chosen, lev + graphs[k].level)
                chosen.pop()

    grow(0, [], 0)

    def key(b):
        return (sum(graphs[k].level for k in b), len(b), tuple(graphs[k].sort_key for k in b))

    return sorted(out, key=key)


def moment_layout(graphs) -> list:
    """Sorted list of the (mu, nu) moment tensors that the graphs use."""
    return sorted({(m, n) for g in graphs for m, n in zip(g.mu, g.nu)})


# ---------------------------------------------------------------------------
# Symmetric-component polynomial of a graph, by brute force over Cartesian indices
# ---------------------------------------------------------------------------


def expand_cartesian(g: Graph) -> dict:
    """Integer polynomial of a connected graph in the symmetric components
    M_mu[a, b, c] (a, b, c = powers of x, y, z).  Every assignment of a
    Cartesian index to every edge slot is enumerated; each vertex collects the
    indices of its incident slots.  Keys: sorted tuple of (mu, (a, b, c)) per
    vertex; values: how many assignments give that monomial."""
    slots = []
    for v in range(g.nv):
        for w in range(v + 1, g.nv):
            slots += [(v, w)] * g.mult(v, w)
    poly = Counter()
    for assign in itertools.product(range(3), repeat=len(slots)):
        cnt = [[0, 0, 0] for _ in range(g.nv)]
        for (v, w), a in zip(slots, assign):
            cnt[v][a] += 1
            cnt[w][a] += 1
        poly[tuple(sorted((g.mu[v], tuple(cnt[v])) for v in range(g.nv)))] += 1
    return dict(poly)


# ---------------------------------------------------------------------------
# Tensor form: moments as explicit Cartesian arrays, graphs contracted by einsum
# ---------------------------------------------------------------------------

_LETTERS = "abcdefghijklmopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"  # 'n' is the atom axis


def graph_einsum(g: Graph) -> str:
    """einsum spec contracting one edge slot per shared Cartesian index."""
    idx = [[] for _ in range(g.nv)]
    k = 0
    for v in range(g.nv):
        for w in range(v + 1, g.nv):
            for _ in range(g.mult(v, w)):
                idx[v].append(_LETTERS[k])
                idx[w].append(_LETTERS[k])
                k += 1
    return ",".join("n" + "".join(s) for s in idx) + "->n"


def cartesian_moments(layout, owner, n_atoms: int, u, f):
    """M_{mu,nu}[i] = sum over pairs p owned by i of f[p, mu] u_p^{(x) nu}.

    owner [P] long: centre atom of each pair; u [P, 3]; f [P, n_mu]."""
    out = {}
    max_nu = max(n for _, n in layout)
    power = [u.new_ones(u.shape[0])]
    for nu in range(1, max_nu + 1):
        power.append(power[-1].unsqueeze(-1) * u.reshape((u.shape[0],) + (1,) * (nu - 1) + (3,)))
    for mu, nu in layout:
        contrib = f[:, mu].reshape((-1,) + (1,) * nu) * power[nu]
        acc = u.new_zeros((n_atoms,) + (3,) * nu)
        out[(mu, nu)] = acc.index_add(0, owner, contrib)
    return out


def graph_values(graphs, moments):
    """Value of every connected graph for every atom: [G, n_atoms]."""
    vals = []
    for g in graphs:
        ops = [moments[(m, n)] for m, n in zip(g.mu, g.nu)]
        vals.append(torch.einsum(graph_einsum(g), *ops))
    return torch.stack(vals)


def basis_from_graphs(bases, gvals):
    """B[n_atoms, m]: each basis function is the product of its graph values."""
    cols = []
    for b in bases:
        v = gvals[b[0]]
        for k in b[1:]:
            v = v * gvals[k]
        cols.append(v)
    return torch.stack(cols, dim=1)


# ---------------------------------------------------------------------------
# Graph form: brute force over neighbour tuples (definition written out)
# ---------------------------------------------------------------------------


def graph_value_bruteforce(g: Graph, u: np.ndarray, f: np.ndarray) -> float:
    """sum over (j_1..j_V) of prod_v f[j_v, mu_v] prod_{v<w} (u_{j_v}.u_{j_w})^{e_vw},
    one neighbourhood, looping over every tuple of neighbours."""
    n = u.shape[0]
    dots = u @ u.T
    total = 0.0
    for js in itertools.product(range(n), repeat=g.nv):
        term = 1.0
        for v in range(g.nv):
            term *= f[js[v], g.mu[v]]
        for v in range(g.nv):
            for w in range(v + 1, g.nv):
                term *= dots[js[v], js[w]] ** g.mult(v, w)
        total += term
    return total


# ---------------------------------------------------------------------------
# Pruning of linearly dependent basis functions (FP64, greedy in basis order)
# ---------------------------------------------------------------------------


def free_basis_rows(graphs, bases, u: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Basis rows for neighbourhoods given directly by unit vectors u [H, n, 3]
    and free radial values f [H, n, n_mu] (no radial basis involved)."""
    h, n, _ = u.shape
    owner = torch.arange(h).repeat_interleave(n)
    tu = torch.as_tensor(u.reshape(-1, 3), dtype=DT)
    tf = torch.as_tensor(f.reshape(h * n, -1), dtype=DT)
    mom = cartesian_moments(moment_layout(graphs), owner, h, tu, tf)
    return basis_from_graphs(bases, graph_values(graphs, mom)).numpy()


def prune_dependent(rows: np.ndarray, rel_tol: float = 1e-9) -> list:
    """Indices of the columns kept by a greedy pass in column order: a column
    is kept when, after scaling every column to unit norm and projecting out
    the span of the kept ones (Gram-Schmidt, applied twice), the residual norm
    exceeds rel_tol."""
    a = rows / np.linalg.norm(rows, axis=0, keepdims=True)
    basis = []
    kept = []
    for k in range(a.shape[1]):
        v = a[:, k].copy()
        for _ in range(2):
            for q in basis:
                v -= (q @ v) * q
        nrm = np.linalg.norm(v)
        if nrm > rel_tol:
            basis.append(v / nrm)
            kept.append(k)
    return kept


@dataclasses.dataclass
class Basis:
    level: int
    graphs: list
    bases: list          # after pruning
    layout: list         # (mu, nu) tensors used by the kept bases

    @property
    def m(self) -> int:
        return len(self.bases)

    @property
    def n_mu(self) -> int:
        return n_mu_for_level(self.level)


def make_basis(level: int, u: np.ndarray, f: np.ndarray) -> Basis:
    """Enumerate, then drop every basis function that is linearly dependent on
    earlier ones, judged on the given random neighbourhoods."""
    graphs = connected_graphs(level)
    allb = basis_functions(level, graphs)
    rows = free_basis_rows(graphs, allb, u, f)
    kept = [allb[k] for k in prune_dependent(rows)]
    used = sorted({k for b in kept for k in b})
    gsub = [graphs[k] for k in used]
    remap = {k: i for i, k in enumerate(used)}
    kept = [tuple(remap[k] for k in b) for b in kept]
    return Basis(level, gsub, kept, moment_layout(gsub))


# ---------------------------------------------------------------------------
# Neighbour list (brute force over all atoms and images)
# ---------------------------------------------------------------------------


def neighbor_list(x: np.ndarray, cell: np.ndarray, pbc, r_cut: float, query=None, candidates=None):
    """All (i, j, n) with 0 < |x_j + n.H - x_i|^2 < R_cut^2, i in ``query``.

    The squared distance is evaluated as (dx*dx + dy*dy) + dz*dz with
    d = (x_j + s) - x_i and s = (n1 a + n2 b) + n3 c, each a separately
    rounded FP64 operation.  Rows are sorted by (i, j, n1, n2, n3).
    Returns int64 arrays i, j and n [P, 3]."""
    x = np.asarray(x, dtype=np.float64)
    cell = np.asarray(cell, dtype=np.float64)
    n_atoms = x.shape[0]
    query = np.arange(n_atoms) if query is None else np.asarray(query)
    cand = np.arange(n_atoms) if candidates is None else np.asarray(candidates)
    inv = np.linalg.inv(cell)
    frac = x @ inv
    rng = []
    for k in range(3):
        if pbc[k]:
            h = 1.0 / np.linalg.norm(inv[:, k])
            span = frac[:, k].max() - frac[:, k].min()
            reach = int(math.ceil(span + r_cut / h)) + 1
            rng.append(range(-reach, reach + 1))
        else:
            rng.append(range(0, 1))
    rc2 = r_cut * r_cut
    out_i, out_j, out_n = [], [], []
    xc = x[cand]
    for i in query:
        for n1 in rng[0]:
            for n2 in rng[1]:
                for n3 in rng[2]:
                    s = (n1 * cell[0] + n2 * cell[1]) + n3 * cell[2]
                    d = (xc + s) - x[i]
                    r2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
                    hit = np.nonzero((r2 < rc2) & (r2 > 0.0))[0]
                    if hit.size:
                        out_i.append(np.full(hit.size, i))
                        out_j.append(cand[hit])
                        out_n.append(np.tile([n1, n2, n3], (hit.size, 1)))
    if not out_i:
        return (np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros((0, 3), np.int64))
    i = np.concatenate(out_i).astype(np.int64)
    j = np.concatenate(out_j).astype(np.int64)
    n = np.concatenate(out_n).astype(np.int64)
    order = np.lexsort((n[:, 2], n[:, 1], n[:, 0], j, i))
    return i[order], j[order], n[order]


# ---------------------------------------------------------------------------
# Potential and site energies
# ---------------------------------------------------------------------------


@dataclasses.dataclass
class Potential:
    level: int
    n_species: int
    n_q: int
    r_min: float
    r_cut: float
    species_energy: np.ndarray   # [S]
    radial: np.ndarray           # [n_mu, n_q, S, S]: c[mu, k, z_i, z_j]
    xi: np.ndarray               # [m]


def _t(a, requires_grad=False):
    t = torch.as_tensor(np.asarray(a), dtype=DT).clone()
    return t.requires_grad_(requires_grad)


def pair_vectors(x, cell, strain, i, j, n):
    """r_ij = x_j + n.H - x_i after the affine map (I + strain) applied to
    positions and cell rows."""
    defo = torch.eye(3, dtype=DT) + strain
    xs = x @ defo.T
    hs = cell @ defo.T
    return xs[j] + n.to(DT) @ hs - xs[i]


def basis_rows(pot: Potential, basis: Basis, c_radial, x, z, cell, strain, nl, atoms):
    """B [len(atoms), m] for the listed centre atoms (torch fp64, differentiable
    in x, strain and the radial coefficients c_radial [n_mu, n_q, S, S])."""
    i, j, n = nl
    atoms = torch.as_tensor(np.asarray(atoms), dtype=torch.long)
    pos = torch.full((x.shape[0],), -1, dtype=torch.long)
    pos[atoms] = torch.arange(atoms.numel())
    sel = pos[i] >= 0
    ii, jj, nn = i[sel], j[sel], n[sel]
    d = pair_vectors(x, cell, strain, ii, jj, nn)
    r = torch.sqrt((d * d).sum(-1))
    u = d / r.unsqueeze(-1)
    q = torch.stack(radial_basis(r, pot.r_min, pot.r_cut, pot.n_q), dim=1)       # [P, n_q]
    c = c_radial[:, :, z[ii], z[jj]]                                              # [n_mu, n_q, P]
    f = torch.einsum("mkp,pk->pm", c, q)
    mom = cartesian_moments(basis.layout, pos[ii], atoms.numel(), u, f)
    return basis_from_graphs(basis.bases, graph_values(basis.graphs, mom))


class Model:
    """Potential + basis with torch leaves for every parameter."""

    def __init__(self, pot: Potential, basis: Basis):
        self.pot = pot
        self.basis = basis
        self.s = _t(pot.species_energy)
        self.c = _t(pot.radial)
        self.xi = _t(pot.xi)

    def params(self):
        return [self.s, self.c, self.xi]

    def requires_grad_(self, flag=True):
        for p in self.params():
            p.requires_grad_(flag)
        return self

    def site_energies(self, x, z, cell, strain, nl, atoms):
        b = basis_rows(self.pot, self.basis, self.c, x, z, cell, strain, nl, atoms)
        atoms_t = torch.as_tensor(np.asarray(atoms), dtype=torch.long)
        return self.s[z[atoms_t]] + b @ self.xi


def _nl_tensors(nl):
    i, j, n = nl
    return (torch.as_tensor(i, dtype=torch.long), torch.as_tensor(j, dtype=torch.long),
            torch.as_tensor(n, dtype=torch.long))


def _chunks(n_atoms: int, pairs_per_atom: float, budget: int):
    step = max(1, int(budget // max(1.0, pairs_per_atom)))
    return [np.arange(a, min(n_atoms, a + step)) for a in range(0, n_atoms, step)]


def evaluate(model: Model, x, z, cell, nl, want=("e", "f", "w"), chunk_pairs=4096, atoms=None):
    """Site energies, total energy, forces, virial and parameter gradients.

    Forces and the virial come from torch.autograd of the tensor-form energy:
    F = -dE/dx, W = -dE/dstrain at zero strain.  ``atoms`` restricts the sum
    to those centre atoms (E_sub = sum of their site energies); derivatives are
    then those of E_sub.  Work is split into chunks of centre atoms only to
    bound memory; the result is the plain sum over chunks."""
    nlt = _nl_tensors(nl)
    n_atoms = x.shape[0]
    centres = np.arange(n_atoms) if atoms is None else np.asarray(atoms)
    xt = _t(x)
    zt = torch.as_tensor(np.asarray(z), dtype=torch.long)
    ct = _t(cell)
    need_x = "f" in want
    need_w = "w" in want
    need_p = "dtheta" in want
    ppa = max(1.0, len(nl[0]) / max(1, n_atoms))
    e_site = torch.zeros(len(centres), dtype=DT)
    grad_x = torch.zeros((n_atoms, 3), dtype=DT)
    grad_w = torch.zeros((3, 3), dtype=DT)
    grad_p = [torch.zeros_like(p) for p in model.params()]
    model.requires_grad_(need_p)
    done = 0
    for chunk in _chunks(len(centres), ppa, chunk_pairs):
        idx = centres[chunk]
        xr = xt.clone().requires_grad_(need_x)
        strain = torch.zeros((3, 3), dtype=DT, requires_grad=need_w)
        e = model.site_energies(xr, zt, ct, strain, nlt, idx)
        e_site[done:done + len(idx)] = e.detach()
        done += len(idx)
        leaves = ([xr] if need_x else []) + ([strain] if need_w else []) + (model.params() if need_p else [])
        if leaves:
            g = torch.autograd.grad(e.sum(), leaves, allow_unused=True)
            k = 0
            if need_x:
                grad_x += g[k] if g[k] is not None else 0
                k += 1
            if need_w:
                grad_w += g[k] if g[k] is not None else 0
                k += 1
            if need_p:
                for a in range(3):
                    if g[k + a] is not None:
                        grad_p[a] += g[k + a]
    model.requires_grad_(False)
    out = {"e_atom": e_site.numpy(), "e": float(e_site.sum())}
    if need_x:
        out["f"] = (-grad_x).numpy()
    if need_w:
        w = -grad_w.numpy()
        out["w_full"] = w
        out["w"] = np.array([w[0, 0], w[1, 1], w[2, 2], w[0, 1], w[0, 2], w[1, 2]])
    if need_p:
        out["dE_ds"] = grad_p[0].numpy()
        out["dE_dc"] = grad_p[1].numpy()
        out["dE_dxi"] = grad_p[2].numpy()
    return out


def force_matching_grad(model: Model, x, z, cell, nl, f_target, chunk_pairs=2048):
    """Loss l = (1/3N) sum_i |F_i - F_t,i|^2 and dl/dtheta by double backward:
    with v = F - F_t held fixed, dl/dtheta = -(2/3N) d/dtheta [sum_i v_i . dE/dx_i]."""
    base = evaluate(model, x, z, cell, nl, want=("e", "f"), chunk_pairs=chunk_pairs)
    n_atoms = x.shape[0]
    v = torch.as_tensor(base["f"] - np.asarray(f_target), dtype=DT)
    loss = float((v * v).sum() / (3 * n_atoms))
    nlt = _nl_tensors(nl)
    xt = _t(x)
    zt = torch.as_tensor(np.asarray(z), dtype=torch.long)
    ct = _t(cell)
    model.requires_grad_(True)
    acc = [torch.zeros_like(p) for p in model.params()]
    ppa = max(1.0, len(nl[0]) / max(1, n_atoms))
    for chunk in _chunks(n_atoms, ppa, chunk_pairs):
        xr = xt.clone().requires_grad_(True)
        strain = torch.zeros((3, 3), dtype=DT)
        e = model.site_energies(xr, zt, ct, strain, nlt, chunk).sum()
        (gx,) = torch.autograd.grad(e, [xr], create_graph=True)
        phi = (v * gx).sum()
        g = torch.autograd.grad(phi, model.params(), allow_unused=True)
        for a in range(3):
            if g[a] is not None:
                acc[a] += g[a].detach()
    model.requires_grad_(False)
    scale = -2.0 / (3 * n_atoms)
    return loss, [scale * a.numpy() for a in acc]


def basis_matrix(model: Model, x, z, cell, nl, atoms=None, chunk_pairs=4096) -> np.ndarray:
    """B rows [len(atoms), m] (no gradients)."""
    nlt = _nl_tensors(nl)
    n_atoms = x.shape[0]
    centres = np.arange(n_atoms) if atoms is None else np.asarray(atoms)
    ppa = max(1.0, len(nl[0]) / max(1, n_atoms))
    rows = []
    with torch.no_grad():
        for chunk in _chunks(len(centres), ppa, chunk_pairs):
            rows.append(basis_rows(model.pot, model.basis, model.c, _t(x), torch.as_tensor(np.asarray(z), dtype=torch.long),
                                   _t(cell), torch.zeros((3, 3), dtype=DT), nlt, centres[chunk]))
    return torch.cat(rows).numpy()


# ---------------------------------------------------------------------------
# Extrapolation grade and MaxVol (paper Sec. 2.1, Sec. 2.3; Goreinov et al. 2010)
# ---------------------------------------------------------------------------


def grade(b: np.ndarray, a_inv: np.ndarray) -> np.ndarray:
    """gamma_i = max_k |(b_i A^-1)_k| for every row b_i of b."""
    return np.abs(np.asarray(b) @ np.asarray(a_inv)).max(axis=1)


def grade_flags(gamma: np.ndarray, tau_sel: float, tau_brk: float) -> np.ndarray:
    """bit 0: gamma > tau_sel (select); bit 1: gamma > tau_brk (break)."""
    return ((gamma > tau_sel).astype(np.uint8) | ((gamma > tau_brk).astype(np.uint8) << 1))


def invert(a: np.ndarray) -> np.ndarray:
    """A^-1 by Gauss-Jordan elimination with partial pivoting, FP64."""
    a = np.array(a, dtype=np.float64)
    m = a.shape[0]
    aug = np.hstack([a, np.eye(m)])
    for col in range(m):
        piv = col + int(np.argmax(np.abs(aug[col:, col])))
        if aug[piv, col] == 0.0:
            raise np.linalg.LinAlgError("singular active set")
        if piv != col:
            aug[[col, piv]] = aug[[piv, col]]
        aug[col] /= aug[col, col]
        for r in range(m):
            if r != col and aug[r, col] != 0.0:
                aug[r] -= aug[r, col] * aug[col]
    return aug[:, m:]


def initial_rows(pool: np.ndarray) -> np.ndarray:
    """Greedy start for MaxVol: repeatedly take the row with the largest
    residual after projecting out the rows already taken (Gram-Schmidt)."""
    p = np.array(pool, dtype=np.float64)
    m = p.shape[1]
    res = p.copy()
    chosen = []
    for _ in range(m):
        norms = np.einsum("ij,ij->i", res, res)
        norms[chosen] = -1.0
        k = int(np.argmax(norms))
        chosen.append(k)
        q = res[k] / np.sqrt(norms[k])
        res -= np.outer(res @ q, q)
    return np.array(chosen)


def independent_columns(pool: np.ndarray, rel_tol: float = 1e-9) -> np.ndarray:
    """A maximal set of linearly independent columns of the pool (greedy
    column-pivoted Gram-Schmidt on the columns scaled to unit norm, two
    projection passes per step; stop when no residual exceeds rel_tol).
    Returns the chosen column indices, sorted."""
    p = np.array(pool, dtype=np.float64)
    norms = np.linalg.norm(p, axis=0)
    res = p / np.where(norms > 0, norms, 1.0)
    basis, chosen = [], []
    for _ in range(min(p.shape)):
        r = np.linalg.norm(res, axis=0)
        r[chosen] = -1.0
        k = int(np.argmax(r))
        if r[k] <= rel_tol:
            break
        chosen.append(k)
        q = res[:, k] / r[k]
        for _ in range(2):
            res -= np.outer(q, q @ res)
        basis.append(q)
    return np.array(sorted(chosen), dtype=np.int64)


def maxvol(pool: np.ndarray, rows=None, delta: float = 0.01, max_iter: int = 10000):
    """MaxVol: swap a pool row into the active set while some |(P A^-1)_ik|
    exceeds 1 + delta; ties go to the lowest i, then the lowest k.
    Returns (active row indices, A^-1, iterations)."""
    p = np.asarray(pool, dtype=np.float64)
    rows = initial_rows(p) if rows is None else np.array(rows)
    it = 0
    while True:
        a_inv = invert(p[rows])
        c = np.abs(p @ a_inv)
        flat = int(np.argmax(c))             # first maximum in row-major order
        i, k = divmod(flat, c.shape[1])
        if c[i, k] <= 1.0 + delta or it >= max_iter:
            return rows, a_inv, it
        rows[k] = i
        it += 1


# ---------------------------------------------------------------------------
# Molecular dynamics (the paper's throughput runs are LAMMPS MD: 100 steps of
# 1 fs, Sec. 2.2 and Fig. 3; its examples run 1 fs MD, Sec. 3)
# ---------------------------------------------------------------------------

# LAMMPS metal units: kinetic energy of 1 amu moving at 1 A/ps, in eV.
AMU_A2_PS2_IN_EV = 1.0364269e-4


def velocity_verlet(model: Model, x, v, z, cell, pbc, masses, dt: float, n_steps: int, f=None):
    """Velocity-Verlet (NVE) trajectory with the MTP forces, metal units
    (x in A, v in A/ps, masses per species in amu, dt in ps).  Each step:
    v += (dt/2) F/m; x += dt v; F = F(x) on a fresh neighbour list; v += (dt/2) F/m.
    f: forces at the initial x (computed when None).  Positions are not wrapped.
    Returns (x, v, f, e_pot [n_steps], e_kin [n_steps]) after each step."""
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    z = np.asarray(z)
    m = np.asarray(masses, dtype=np.float64)[z][:, None] * AMU_A2_PS2_IN_EV   # eV ps^2 / A^2
    r_cut = model.pot.r_cut
    if f is None:
        f = evaluate(model, x, z, cell, neighbor_list(x, cell, pbc, r_cut), want=("e", "f"))["f"]
    f = np.array(f, dtype=np.float64)
    e_pot, e_kin = [], []
    for _ in range(n_steps):
        v = v + 0.5 * dt * f / m
        x = x + dt * v
        out = evaluate(model, x, z, cell, neighbor_list(x, cell, pbc, r_cut), want=("e", "f"))
        f = out["f"]
        v = v + 0.5 * dt * f / m
        e_pot.append(out["e"])
        e_kin.append(float(0.5 * (m * v * v).sum()))
    return x, v, f, np.array(e_pot), np.array(e_kin)


EV_PER_A3_IN_BAR = 1.602176634e-19 / 1e-30 / 1e5   # 1 eV/A^3 in bar (SI definitions)


def pressure_bar(e_kin: float, virial, cell) -> float:
    """Instantaneous pressure of a periodic system in bar:
    P = (2 E_kin + W_xx + W_yy + W_zz) / (3 V), with W = -dE/d(strain) the
    pressure virial and V = |det H|."""
    vol = abs(float(np.linalg.det(np.asarray(cell, dtype=np.float64))))
    return (2.0 * e_kin + float(virial[0] + virial[1] + virial[2])) / (3.0 * vol) * EV_PER_A3_IN_BAR


def berendsen_npt(model: Model, x, v, z, cell, pbc, masses, dt: float, n_steps: int, p_target: float,
                  tau_p: float, bulk_modulus: float = 10.0, f=None, w=None):
    """Velocity Verlet with the Berendsen barostat (isotropic coupling; Berendsen
    et al. 1984): each step is the velocity-Verlet step of velocity_verlet, then
    the pressure P of the new velocities and of the virial of the new forces,
    and the positions and the cell rows are multiplied by
    mu = (1 - (dt / tau_p) (p_target - P) / bulk_modulus)^(1/3).
    Pressures and the modulus in bar, tau_p in ps.  f, w: forces and virial at
    the initial x (computed when None).  Returns (x, v, f, cell, pressures [n_steps])."""
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    cell = np.array(cell, dtype=np.float64)
    z = np.asarray(z)
    m = np.asarray(masses, dtype=np.float64)[z][:, None] * AMU_A2_PS2_IN_EV
    r_cut = model.pot.r_cut
    if f is None:
        f = evaluate(model, x, z, cell, neighbor_list(x, cell, pbc, r_cut), want=("e", "f"))["f"]
    f = np.array(f, dtype=np.float64)
    pressures = []
    for _ in range(n_steps):
        v = v + 0.5 * dt * f / m
        x = x + dt * v
        out = evaluate(model, x, z, cell, neighbor_list(x, cell, pbc, r_cut), want=("e", "f", "w"))
        f = out["f"]
        v = v + 0.5 * dt * f / m
        p = pressure_bar(float(0.5 * (m * v * v).sum()), out["w"], cell)
        pressures.append(p)
        mu = (1.0 - dt / tau_p * (p_target - p) / bulk_modulus) ** (1.0 / 3.0)
        x = x * mu
        cell = cell * mu
    return x, v, f, cell, np.array(pressures)


# ---------------------------------------------------------------------------
# Potential files (written by oracle/make_potentials.py)
# ---------------------------------------------------------------------------


def basis_from_encoding(level: int, enc) -> Basis:
    """Rebuild a Basis from its canonical encoding [[[mu...], [e...]], ...] per basis."""
    graphs = sorted({Graph(tuple(mu), tuple(e)) for b in enc for mu, e in b}, key=lambda g: g.sort_key)
    index = {g: k for k, g in enumerate(graphs)}
    bases = [tuple(index[Graph(tuple(mu), tuple(e))] for mu, e in b) for b in enc]
    return Basis(level, graphs, bases, moment_layout(graphs))


def load_model(pot: dict) -> Model:
    """Model from a potential dictionary (JSON file contents)."""
    p = Potential(pot["level"], pot["n_species"], pot["n_q"], pot["r_min"], pot["r_cut"],
                  np.array(pot["species_energy"]), np.array(pot["radial"]).reshape(pot["radial_shape"]),
                  np.array(pot["xi"]))
    return Model(p, basis_from_encoding(pot["level"], pot["basis"]))
