"""Build-time generator of the MTP basis and its straight-line CUDA code.

For a level L this module
  1. enumerates the connected contraction graphs of moment tensors with total
     level <= L and all their products (the basis functions B_alpha of the
     Moment Tensor Potential, Shapeev 2016, the model the paper accelerates;
     paper Sec. 2.2 on the level),
  2. removes basis functions that are linear combinations of earlier ones, by
     exact rank computations over the prime field GF(2^31 - 1) at random points
     of the unit sphere (a rational parametrisation, so |u| = 1 holds exactly),
  3. expands each graph into an integer polynomial of symmetric moment
     components with the multinomial theorem (exported for table checks),
  4. factors every graph into a DAG of symmetric contractions with shared
     subexpressions, and
  5. writes a C++/CUDA header with the moment layout, straight-line device
     code for the per-pair moment update, the per-atom contraction with its
     reverse pass, the per-pair adjoint, and host tables of the basis.

Canonical forms and the order of basis functions (shared by every consumer of
the table):
  * a graph is the lexicographically smallest (mu tuple, upper-triangle edge
    multiplicity tuple) over vertex orderings; its sort key is
    (level, mu tuple, edge tuple);
  * a basis function is a multiset of graphs sorted by that key; basis
    functions are ordered by (level, number of factors, factor keys);
  * moment components are ordered by (mu, nu) and, within a tensor, by
    (a, b, c) with a descending, then b descending (powers of x, y, z).
"""
from __future__ import annotations

import itertools
import math
import os
import sys
from collections import defaultdict

import numpy as np

# levels from which the contraction runs as an interpreted program
INTERPRET_FROM_LEVEL = 18
# levels whose neighbour sweeps work on the components with a z-exponent of at
# most 1 (the others follow from |rhat| = 1 in the contraction, or in the
# first records of an interpreted contraction program)
SPHERE_MAX_LEVEL = 20

# ---------------------------------------------------------------------------
# graphs and basis functions
# ---------------------------------------------------------------------------


def level_of_moment(mu, nu):
    return 2 + 4 * mu + nu


def radial_count(level):
    return (level - 2) // 4 + 1


def multi_indices(n):
    """(a, b, c) with a + b + c = n, a descending, then b descending."""
    return [(a, b, n - a - b) for a in range(n, -1, -1) for b in range(n - a, -1, -1)]


def n_sym(n):
    return (n + 1) * (n + 2) // 2


class G:
    """A canonical connected graph."""
    __slots__ = ("mu", "e", "nv", "nu", "level", "edges")

    def __init__(self, mu, e):
        self.mu = tuple(mu)
        self.e = tuple(e)
        self.nv = len(mu)
        pairs = [(v, w) for v in range(self.nv) for w in range(v + 1, self.nv)]
        self.edges = {p: k for p, k in zip(pairs, e) if k}
        nu = [0] * self.nv
        for (v, w), k in self.edges.items():
            nu[v] += k
            nu[w] += k
        self.nu = tuple(nu)
        self.level = sum(level_of_moment(m, n) for m, n in zip(self.mu, self.nu))

    @property
    def key(self):
        return (self.level, self.mu, self.e)


def _block_perms(mu_sorted):
    """Permutations of vertex positions that keep the sorted labels sorted."""
    blocks = []
    start = 0
    for k in range(1, len(mu_sorted) + 1):
        if k == len(mu_sorted) or mu_sorted[k] != mu_sorted[start]:
            blocks.append(list(range(start, k)))
            start = k
    for parts in itertools.product(*[itertools.permutations(b) for b in blocks]):
        yield [v for part in parts for v in part]


def _canonical(mu_sorted, mat):
    n = len(mu_sorted)
    best = None
    for p in _block_perms(mu_sorted):
        e = tuple(mat[p[a]][p[b]] for a in range(n) for b in range(a + 1, n))
        if best is None or e < best:
            best = e
    return tuple(mu_sorted), best


def _connected(n, mat):
    reach = {0}
    frontier = [0]
    while frontier:
        nxt = []
        for v in frontier:
            for w in range(n):
                if mat[v][w] and w not in reach:
                    reach.add(w)
                    nxt.append(w)
        frontier = nxt
    return len(reach) == n


def graphs_for_level(level):
    """Canonical connected graphs, sorted by key.  Labels are generated as
    non-decreasing tuples, so only permutations inside blocks of equal labels
    are needed to canonicalise."""
    nmu = radial_count(level)
    seen = set()
    nv = 1
    while 2 * nv + 2 * (nv - 1) <= level:
        pairs = [(v, w) for v in range(nv) for w in range(v + 1, nv)]
        budget = (level - 2 * nv) // 2          # edges allowed
        for labels in itertools.combinations_with_replacement(range(nmu), nv):
            spare = (level - 2 * nv - 4 * sum(labels)) // 2
            if spare < (nv - 1):
                continue
            cap = min(budget, spare)

            def fill(k, left, mult):
                if k == len(pairs):
                    yield list(mult)
                    return
                for x in range(left + 1):
                    mult.append(x)
                    yield from fill(k + 1, left - x, mult)
                    mult.pop()

            for mult in fill(0, cap, []):
                mat = [[0] * nv for _ in range(nv)]
                for (v, w), x in zip(pairs, mult):
                    mat[v][w] = mat[w][v] = x
                if nv > 1 and not _connected(nv, mat):
                    continue
                seen.add(_canonical(labels, mat))
        nv += 1
    out = [G(mu, e) for mu, e in seen]
    out.sort(key=lambda g: g.key)
    return out


def products_for_level(level, graphs):
    """All multisets of graphs with total level <= L, in canonical order."""
    res = []
    levels = [g.level for g in graphs]

    def walk(first, acc, lev):
        for k in range(first, len(graphs)):
            if lev + levels[k] > level:
                continue
            acc.append(k)
            res.append(tuple(acc))
            walk(k, acc, lev + levels[k])
            acc.pop()

    walk(0, [], 0)
    res.sort(key=lambda b: (sum(levels[k] for k in b), len(b), tuple(graphs[k].key for k in b)))
    return res


# ---------------------------------------------------------------------------
# multinomial expansion into symmetric components
# ---------------------------------------------------------------------------


def multinomial_weight(k):
    n = sum(k)
    return math.factorial(n) // (math.factorial(k[0]) * math.factorial(k[1]) * math.factorial(k[2]))


def expand_graph(g: G):
    """{monomial: integer coefficient}; a monomial is a sorted tuple of
    (mu, (a, b, c)) per vertex.  Each edge of multiplicity e expands
    (u_v . u_w)^e = sum_{|k|=e} e!/k! u_v^k u_w^k."""
    edges = sorted(g.edges.items())
    poly = defaultdict(int)
    for choice in itertools.product(*[multi_indices(e) for _, e in edges]):
        weight = 1
        acc = [[0, 0, 0] for _ in range(g.nv)]
        for ((v, w), _), k in zip(edges, choice):
            weight *= multinomial_weight(k)
            for d in range(3):
                acc[v][d] += k[d]
                acc[w][d] += k[d]
        mono = tuple(sorted((g.mu[v], tuple(acc[v])) for v in range(g.nv)))
        poly[mono] += weight
    return dict(poly)


# ---------------------------------------------------------------------------
# exact pruning over GF(p)
# ---------------------------------------------------------------------------

PRIME = 2147483647  # 2^31 - 1


def _inv(a):
    return pow(int(a), PRIME - 2, PRIME)


def _sphere_points(rng, count):
    """Points (x, y, z) of GF(p)^3 with x^2 + y^2 + z^2 = 1 (inverse
    stereographic projection of random (s, t))."""
    pts = []
    while len(pts) < count:
        s, t = (int(v) for v in rng.integers(0, PRIME, size=2))
        q = (s * s + t * t + 1) % PRIME
        if q == 0:
            continue
        qi = _inv(q)
        pts.append(((2 * s * qi) % PRIME, (2 * t * qi) % PRIME, ((s * s + t * t - 1) * qi) % PRIME))
    return np.array(pts, dtype=np.int64)


def _mod_rank_greedy(cols):
    """Indices of columns independent of all earlier kept columns (GF(p))."""
    n_rows = cols.shape[0]
    piv_rows = []       # pivot row of each kept column's reduced vector
    reduced = []        # reduced kept vectors
    kept = []
    for k in range(cols.shape[1]):
        v = cols[:, k].copy() % PRIME
        for pr, rv in zip(piv_rows, reduced):
            if v[pr]:
                v = (v - (int(v[pr]) * rv) % PRIME) % PRIME
        nz = np.nonzero(v)[0]
        if nz.size:
            pr = int(nz[0])
            v = (v * _inv(v[pr])) % PRIME
            piv_rows.append(pr)
            reduced.append(v)
            kept.append(k)
    del n_rows
    return kept


def prune(level, graphs, products, seed=20251017):
    """Keep the basis functions that are linearly independent of earlier ones
    as polynomials in (u_j, f_mu(j)) with |u_j| = 1."""
    rng = np.random.default_rng(seed)
    nmu = radial_count(level)
    n_hood = 2 * len(products) + 8
    n_nb = 12
    layout = sorted({(m, n) for g in graphs for m, n in zip(g.mu, g.nu)})
    maxnu = max(n for _, n in layout)
    pts = _sphere_points(rng, n_hood * n_nb).reshape(n_hood, n_nb, 3)
    f = rng.integers(0, PRIME, size=(n_hood, n_nb, nmu), dtype=np.int64)
    # powers of each coordinate
    pw = np.ones((maxnu + 1, n_hood, n_nb, 3), dtype=np.int64)
    for k in range(1, maxnu + 1):
        pw[k] = (pw[k - 1] * pts) % PRIME
    comp = {}
    for mu, nu in layout:
        for K in multi_indices(nu):
            mono = (pw[K[0], :, :, 0] * pw[K[1], :, :, 1]) % PRIME
            mono = (mono * pw[K[2], :, :, 2]) % PRIME
            comp[(mu, K)] = ((mono * f[:, :, mu]) % PRIME).sum(axis=1) % PRIME
    gval = []
    for g in graphs:
        acc = np.zeros(n_hood, dtype=np.int64)
        for mono, coef in expand_graph(g).items():
            t = np.full(n_hood, coef % PRIME, dtype=np.int64)
            for key in mono:
                t = (t * comp[key]) % PRIME
            acc = (acc + t) % PRIME
        gval.append(acc)
    cols = np.zeros((n_hood, len(products)), dtype=np.int64)
    for a, b in enumerate(products):
        v = np.ones(n_hood, dtype=np.int64)
        for k in b:
            v = (v * gval[k]) % PRIME
        cols[:, a] = v
    return _mod_rank_greedy(cols)


# ---------------------------------------------------------------------------
# contraction DAG
# ---------------------------------------------------------------------------


class Dag:
    """Nodes are symmetric tensors stored by multi_indices(rank) components.

    ('M', mu, nu, off): slice of M_{mu,nu}: component K -> M_mu[off + K],
                        rank nu - |off|.
    ('C', A, B):        B (rank p) fully contracted into A (rank >= p):
                        C[K] = sum_{|P| = p} p!/P! A[K + P] B[P].
    """

    def __init__(self):
        self.nodes = []      # list of (kind, ...), rank
        self.index = {}

    def _add(self, key, rank):
        if key not in self.index:
            self.index[key] = len(self.nodes)
            self.nodes.append((key, rank))
        return self.index[key]

    def rank(self, n):
        return self.nodes[n][1]

    def leaf(self, mu, nu, off):
        return self._add(("M", mu, nu, tuple(off)), nu - sum(off))

    def contract(self, a, b):
        ra, rb = self.rank(a), self.rank(b)
        if ra < rb:
            a, b, ra, rb = b, a, rb, ra
        key = ("C",) + ((min(a, b), max(a, b)) if ra == rb else (a, b))
        return self._add(key, ra - rb)

    def graph(self, g: G):
        """[(weight, scalar node)] whose weighted sum is the graph value."""
        if g.nv == 1:
            return [(1, self.leaf(g.mu[0], 0, (0, 0, 0)))]
        # spanning tree by breadth-first search from vertex 0, lowest index first
        tree = set()
        seen = {0}
        queue = [0]
        while queue:
            v = queue.pop(0)
            for (a, b) in sorted(g.edges):
                if v in (a, b):
                    w = b if a == v else a
                    if w not in seen:
                        seen.add(w)
                        tree.add((a, b))
                        queue.append(w)
        cut = sorted(p for p in g.edges if p not in tree)
        out = []
        for choice in itertools.product(*[multi_indices(g.edges[p]) for p in cut]):
            weight = 1
            off = [[0, 0, 0] for _ in range(g.nv)]
            for p, k in zip(cut, choice):
                weight *= multinomial_weight(k)
                for v in p:
                    for d in range(3):
                        off[v][d] += k[d]
            cur = {v: self.leaf(g.mu[v], g.nu[v], off[v]) for v in range(g.nv)}
            nbrs = {v: set() for v in range(g.nv)}
            for (a, b) in tree:
                nbrs[a].add(b)
                nbrs[b].add(a)
            alive = set(range(g.nv))
            while len(alive) > 1:
                leaves = [v for v in alive if len(nbrs[v]) == 1]
                v = min(leaves, key=lambda t: (self.rank(cur[t]), t))
                (w,) = nbrs[v]
                cur[w] = self.contract(cur[w], cur[v])
                nbrs[w].discard(v)
                nbrs.pop(v)
                alive.discard(v)
            out.append((weight, cur[alive.pop()]))
        return out


# ---------------------------------------------------------------------------
# the level description
# ---------------------------------------------------------------------------


class Level:
    def __init__(self, level):
        self.level = level
        self.nmu = radial_count(level)
        all_graphs = graphs_for_level(level)
        all_products = products_for_level(level, all_graphs)
        kept = prune(level, all_graphs, all_products)
        self.n_enumerated = len(all_products)
        used = sorted({k for a in kept for k in all_products[a]})
        remap = {k: i for i, k in enumerate(used)}
        self.graphs = [all_graphs[k] for k in used]
        self.bases = [tuple(remap[k] for k in all_products[a]) for a in kept]
        self.layout = sorted({(m, n) for g in self.graphs for m, n in zip(g.mu, g.nu)})
        self.nu_max = [max([n for m, n in self.layout if m == mu], default=-1) for mu in range(self.nmu)]
        self.comps = [(mu, K) for mu, nu in self.layout for K in multi_indices(nu)]
        self.comp_index = {c: i for i, c in enumerate(self.comps)}
        # components the neighbour sweeps accumulate.  Because rhat is a unit
        # vector, u^(a,b,c) = u^(a,b,c-2) - u^(a+2,b,c-2) - u^(a,b+2,c-2) for
        # c >= 2, so with every degree 0..nu_max present for each mu the
        # components with a z-exponent of at most 1 determine all others
        # (SPHERE_MAX_LEVEL: levels that use this; above it all are swept)
        self.expand = {}
        if level <= SPHERE_MAX_LEVEL:
            for c, (mu, K) in enumerate(self.comps):
                a, b, z = K
                if z >= 2:
                    src = [(mu, (a, b, z - 2)), (mu, (a + 2, b, z - 2)), (mu, (a, b + 2, z - 2))]
                    assert all(t in self.comp_index for t in src), (level, mu, K)
                    self.expand[c] = tuple(self.comp_index[t] for t in src)
        self.swept = [c for c in range(len(self.comps)) if c not in self.expand]
        self.dag = Dag()
        self.roots = [self.dag.graph(g) for g in self.graphs]
        # levels with an interpreted contraction sweep the neighbours once per
        # component group (mu = 0 / mu >= 1), so that a group's moments or
        # adjoints fit in registers
        if level >= INTERPRET_FROM_LEVEL and self.nmu > 1:
            self.groups = [[c for c, (mu, K) in enumerate(self.comps) if mu == 0],
                           [c for c, (mu, K) in enumerate(self.comps) if mu >= 1]]
        else:
            self.groups = [list(range(len(self.comps)))]

    @property
    def m(self):
        return len(self.bases)


# ---------------------------------------------------------------------------
# code emission
# ---------------------------------------------------------------------------


def tree_sum(terms):
    """Balanced sum expression (short dependency chains)."""
    terms = list(terms)
    if not terms:
        return "R(0)"
    while len(terms) > 1:
        nxt = []
        for k in range(0, len(terms) - 1, 2):
            nxt.append("(%s + %s)" % (terms[k], terms[k + 1]))
        if len(terms) % 2:
            nxt.append(terms[-1])
        terms = nxt
    return terms[0]


def emit_dot(lines, ind, name, pairs, declare=True, max_chain=6):
    """name = sum_k x_k * y_k as interleaved FMA chains of length <= max_chain,
    combined by a balanced sum."""
    nacc = max(1, min(4, (len(pairs) + max_chain - 1) // max_chain))
    accs = []
    for a in range(nacc):
        sub = pairs[a::nacc]
        if not sub:
            continue
        acc = name if nacc == 1 else "%s_p%d" % (name, a)
        x0, y0 = sub[0]
        lines.append(ind + "%s%s = %s * %s;" % ("R " if (declare or nacc > 1) else "", acc, x0, y0))
        for x, y in sub[1:]:
            lines.append(ind + "%s = fmadd(%s, %s, %s);" % (acc, x, y, acc))
        accs.append(acc)
    if nacc > 1:
        lines.append(ind + "%s%s = %s;" % ("R " if declare else "", name, tree_sum(accs)))


def _mono_name(K):
    return "u%d%d%d" % K


def _emit_monomials(lines, maxnu, ind, need=None):
    """u^K for all |K| <= maxnu, each from a lower one times one coordinate."""
    lines.append(ind + "const R u000 = R(1);")
    for nu in range(1, maxnu + 1):
        for K in multi_indices(nu):
            if need is not None and K not in need:
                continue
            if K[0] > 0:
                src, c = (K[0] - 1, K[1], K[2]), "ux"
            elif K[1] > 0:
                src, c = (K[0], K[1] - 1, K[2]), "uy"
            else:
                src, c = (K[0], K[1], K[2] - 1), "uz"
            lines.append(ind + "const R %s = %s * %s;" % (_mono_name(K), _mono_name(src), c))


def _closure(keys):
    """All monomials needed to build ``keys`` by the rule in _emit_monomials."""
    need = set()
    for K in keys:
        k = tuple(K)
        while sum(k) > 0:
            need.add(k)
            if k[0] > 0:
                k = (k[0] - 1, k[1], k[2])
            elif k[1] > 0:
                k = (k[0], k[1] - 1, k[2])
            else:
                k = (k[0], k[1], k[2] - 1)
    return need


def _monomial_source(K):
    """The lower monomial and coordinate that u^K is formed from."""
    if K[0] > 0:
        return (K[0] - 1, K[1], K[2]), "ux"
    if K[1] > 0:
        return (K[0], K[1] - 1, K[2]), "uy"
    return (K[0], K[1], K[2] - 1), "uz"


def _monomial_order(maxnu):
    return [K for nu in range(0, maxnu + 1) for K in multi_indices(nu)]


def emit_moments(lv: Level, subset=None, fname="moments"):
    """M[c] += f[mu] * u^K for every component (mu, K) (of ``subset`` if
    given).  Each monomial is formed and consumed at once, so few monomials
    are live at a time."""
    L = []
    ind = "    "
    L.append("  template <class R>")
    L.append("  __device__ __forceinline__ static void %s(R* __restrict__ M, const R* __restrict__ f, R ux, R uy, R uz) {"
             % fname)
    L.append(ind + "const R u000 = R(1);")
    by_k = defaultdict(list)
    for c, (mu, K) in enumerate(lv.comps):
        if (subset is None or c in subset) and c not in lv.expand:
            by_k[K].append((c, mu))
    need = _closure(by_k)
    for K in _monomial_order(max(sum(K) for K in by_k)):
        if sum(K) > 0 and K not in need:
            continue
        if sum(K) > 0:
            src, co = _monomial_source(K)
            L.append(ind + "const R %s = %s * %s;" % (_mono_name(K), _mono_name(src), co))
        for c, mu in by_k.get(K, []):
            if sum(K) == 0:
                L.append(ind + "M[%d] += f[%d];" % (c, mu))
            else:
                L.append(ind + "M[%d] = fmadd(f[%d], %s, M[%d]);" % (c, mu, _mono_name(K), c))
    L.append("  }")
    return L


# Adjoint code shape options.  ADJ_FOLD_BY_DEGREE folds the per-degree sums
# s_{mu,d} into S_mu and T_mu as soon as the last monomial of degree d is done
# (fewer live accumulators); ADJ_MAX_CHAIN > 0 splits accumulation chains
# longer than that over interleaved partial sums.  On the level-16 energy/force
# kernel both measured slower than the plain form (1.69 and 1.70 ms against
# 1.60 ms on 1,024,000 atoms), so both are off.
ADJ_FOLD_BY_DEGREE = False
ADJ_MAX_CHAIN = 0


def emit_pair_adjoint(lv: Level, subset=None, fname="pair_adjoint"):
    """Gradient of sum_c D[c] M_c(r) with respect to the pair vector r, where
    M_c(r) = f_mu(|r|) rhat^K:

        S_mu = sum_K D u^K,  T_mu = sum_K |K| D u^K,  G_mu = sum_K D grad_u(u^K)
        g = u * sum_mu (df_mu S_mu - f_mu T_mu / r) + (1/r) sum_mu f_mu G_mu

    (grad of u^K along the sphere is (grad_u u^K - |K| u^K u) / r).  S_mu is
    also returned: it is the chain-rule factor of d E / d c[mu, k, zi, zj].
    The code visits monomials u^J in generation order and adds every term that
    uses u^J right away: D[mu,J] u^J into S_{mu,|J|}, and D[mu,K] u^J into
    G_{mu,d,K_d} for K = J + e_d (grad u^K has component K_d u^{K - e_d})."""
    L = []
    ind = "    "
    L.append("  template <class R>")
    L.append("  __device__ __forceinline__ static void %s(const R* __restrict__ D, const R* __restrict__ f, "
             "const R* __restrict__ df, R ux, R uy, R uz, R rinv, R& gx, R& gy, R& gz, R* __restrict__ S) {" % fname)
    L.append(ind + "const R u000 = R(1);")
    comp = {key: c for key, c in lv.comp_index.items() if (subset is None or c in subset) and c not in lv.expand}
    comps = [key for c, key in enumerate(lv.comps) if (subset is None or c in subset) and c not in lv.expand]
    terms = defaultdict(int)     # accumulator name -> number of terms so far
    parts = defaultdict(list)    # accumulator name -> partial-sum names declared

    def total(name):
        """Expression for the full sum of accumulator `name`."""
        return tree_sum(parts[name])

    # number of terms of every accumulator (for the chain splitting)
    count = defaultdict(int)
    for J in _monomial_order(max(sum(K) for _, K in comps)):
        for mu in range(lv.nmu):
            if (mu, J) in comp:
                count["s%d_%d" % (mu, sum(J))] += 1
            for d, dn in enumerate("xyz"):
                K = list(J)
                K[d] += 1
                if (mu, tuple(K)) in comp:
                    count["g%d%s%d" % (mu, dn, K[d])] += 1

    def acc(name, x, y):
        n = terms[name]
        terms[name] += 1
        nparts = 1
        if ADJ_MAX_CHAIN:
            nparts = min(4, (count[name] + ADJ_MAX_CHAIN - 1) // ADJ_MAX_CHAIN)
        k = n % nparts
        part = name if k == 0 else "%s_q%d" % (name, k)
        if part in parts[name]:
            L.append(ind + "%s = fmadd(%s, %s, %s);" % (part, x, y, part))
        else:
            parts[name].append(part)
            L.append(ind + "R %s = %s * %s;" % (part, x, y))

    maxnu = max(sum(K) for _, K in comps)
    folded = set()   # mu with S_mu / T_mu declared

    def fold(deg):
        for mu in range(lv.nmu):
            name = "s%d_%d" % (mu, deg)
            if name not in parts:
                continue
            v = total(name)
            if mu not in folded:
                folded.add(mu)
                L.append(ind + "R S%d = %s;" % (mu, v))
                L.append(ind + "R T%d = %s;" % (mu, "R(0)" if deg == 0 else ("%s" % v if deg == 1 else
                                                                             "R(%d) * (%s)" % (deg, v))))
            else:
                L.append(ind + "S%d += %s;" % (mu, v))
                if deg == 1:
                    L.append(ind + "T%d += %s;" % (mu, v))
                elif deg > 1:
                    L.append(ind + "T%d = fmadd(R(%d), %s, T%d);" % (mu, deg, v, mu))

    used = set()
    for mu, K in comps:
        used.add(K)
        for d in range(3):
            if K[d] > 0:
                used.add(tuple(K[t] - (t == d) for t in range(3)))
    need = _closure(used)
    order = [J for J in _monomial_order(maxnu) if sum(J) == 0 or J in need]
    for idx, J in enumerate(order):
        if sum(J) > 0:
            src, co = _monomial_source(J)
            L.append(ind + "const R %s = %s * %s;" % (_mono_name(J), _mono_name(src), co))
        mj = _mono_name(J)
        for mu in range(lv.nmu):
            c = comp.get((mu, J))
            if c is not None:
                acc("s%d_%d" % (mu, sum(J)), "D[%d]" % c, mj)
            for d, dn in enumerate("xyz"):
                K = list(J)
                K[d] += 1
                c2 = comp.get((mu, tuple(K)))
                if c2 is not None:
                    acc("g%d%s%d" % (mu, dn, K[d]), "D[%d]" % c2, mj)
        if ADJ_FOLD_BY_DEGREE and (idx + 1 == len(order) or sum(order[idx + 1]) != sum(J)):
            fold(sum(J))
    L.append(ind + "R ax = R(0), ay = R(0), az = R(0), radial = R(0);")
    for mu in range(lv.nmu):
        nus = sorted({sum(K) for (m, K) in comps if m == mu})
        if not nus:
            L.append(ind + "S[%d] = R(0);" % mu)
            continue
        if not ADJ_FOLD_BY_DEGREE:
            L.append(ind + "const R S%d = %s;" % (mu, tree_sum(total("s%d_%d" % (mu, n)) for n in nus)))
            tnus = [n for n in nus if n > 0]
            L.append(ind + "const R T%d = %s;" % (mu, tree_sum((total("s%d_%d" % (mu, n))) if n == 1 else
                                                                ("R(%d) * %s" % (n, total("s%d_%d" % (mu, n))))
                                                                for n in tnus)))
        L.append(ind + "S[%d] = S%d;" % (mu, mu))
        for dn in "xyz":
            gp = []
            for a in range(1, maxnu + 1):
                name = "g%d%s%d" % (mu, dn, a)
                if name in parts:
                    gp.append(total(name) if a == 1 else "R(%d) * %s" % (a, total(name)))
            if gp:
                L.append(ind + "a%s = fmadd(f[%d], %s, a%s);" % (dn, mu, tree_sum(gp), dn))
        L.append(ind + "radial = fmadd(df[%d], S%d, radial);" % (mu, mu))
        L.append(ind + "radial = fmadd(-f[%d] * rinv, T%d, radial);" % (mu, mu))
    L.append(ind + "gx = fmadd(ux, radial, ax * rinv);")
    L.append(ind + "gy = fmadd(uy, radial, ay * rinv);")
    L.append(ind + "gz = fmadd(uz, radial, az * rinv);")
    L.append("  }")
    return L


def emit_contract(lv: Level, fname="contract"):
    """Per atom: graph values from the DAG, basis products, E = sum xi B, and the
    reverse pass D = dE/dM.  ``WANT_B`` stores the basis values."""
    dag = lv.dag
    L = []
    ind = "    "
    # M: the moment components, indexed M[c] (an array, or a strided view of them in shared memory)
    # B: where the basis values go when WANT_B: an array (B[a] = value) or a sink called as B(a, value)
    L.append("  template <class R, bool WANT_B, class MV = const R*, class BV = R*>")
    L.append("  __device__ __forceinline__ static R %s(MV M, "
             "const typename ScalarOf<R>::T* __restrict__ xi, R* __restrict__ D, BV B) {" % fname)
    L.append(ind + "(void)B;")
    # forward.  Components with a z-exponent >= 2 (when the sweeps leave them
    # out) are formed from the swept ones first, in increasing z-exponent.
    for c in sorted(lv.expand, key=lambda t: (lv.comps[t][1][2], t)):
        s0, s1, s2 = (("M[%d]" % t) if t not in lv.expand else ("mx%d" % t) for t in lv.expand[c])
        L.append(ind + "const R mx%d = (%s - %s) - %s;" % (c, s0, s1, s2))

    def mref(c):
        return ("mx%d" % c) if c in lv.expand else ("M[%d]" % c)

    def comp_ref(n, K):
        key, rank = dag.nodes[n]
        if key[0] == "M":
            _, mu, nu, off = key
            full = (off[0] + K[0], off[1] + K[1], off[2] + K[2])
            return mref(lv.comp_index[(mu, full)])
        return "v%d_%d" % (n, multi_indices(rank).index(K))

    wname = {}
    for n, (key, rank) in enumerate(dag.nodes):
        if key[0] != "C":
            continue
        _, a, b = key
        p = dag.rank(b)
        Ps = multi_indices(p)
        # weighted copy of B's components (weights p!/P!)
        wn = []
        for P in Ps:
            w = multinomial_weight(P)
            if w == 1:
                wn.append(comp_ref(b, P))
            else:
                nm = "w%d_%d" % (n, Ps.index(P))
                L.append(ind + "const R %s = R(%d) * %s;" % (nm, w, comp_ref(b, P)))
                wn.append(nm)
        wname[n] = wn
        for ki, K in enumerate(multi_indices(rank)):
            terms = [(comp_ref(a, (K[0] + P[0], K[1] + P[1], K[2] + P[2])), wn[j]) for j, P in enumerate(Ps)]
            emit_dot(L, ind, "v%d_%d" % (n, ki), terms)
    # graph values
    for gi, roots in enumerate(lv.roots):
        parts = []
        for w, node in roots:
            ref = comp_ref(node, (0, 0, 0))
            parts.append(ref if w == 1 else "R(%d) * %s" % (w, ref))
        L.append(ind + "const R G%d = %s;" % (gi, tree_sum(parts)))
    # basis values, energy
    L.append(ind + "R E = R(0);")
    for a, b in enumerate(lv.bases):
        L.append(ind + "const R B%d = %s;" % (a, " * ".join("G%d" % k for k in b)))
        L.append(ind + "if (WANT_B) store_basis(B, %d, B%d);" % (a, a))
        L.append(ind + "E = fmadd(R(xi[%d]), B%d, E);" % (a, a))
    # reverse: dE/dG
    gbar = defaultdict(list)
    for a, b in enumerate(lv.bases):
        for j in range(len(b)):
            others = [b[t] for t in range(len(b)) if t != j]
            gbar[b[j]].append((a, others))
    for gi in range(len(lv.graphs)):
        terms = []
        for a, others in gbar[gi]:
            prod = " * ".join("G%d" % k for k in others)
            terms.append("R(xi[%d])" % a + (" * " + prod if prod else ""))
        L.append(ind + "const R Gb%d = %s;" % (gi, tree_sum(terms)))
    # node adjoints
    adj = defaultdict(list)          # (node, comp index) -> list of expressions
    for gi, roots in enumerate(lv.roots):
        for w, node in roots:
            adj[(node, 0)].append("Gb%d" % gi if w == 1 else "R(%d) * Gb%d" % (w, gi))
    dcontrib = defaultdict(list)     # M component -> expressions

    def flush(n):
        """Emit the adjoint of node n; return variable names per component."""
        key, rank = dag.nodes[n]
        names = []
        for ki in range(n_sym(rank)):
            ex = adj.get((n, ki))
            if not ex:
                names.append(None)
                continue
            nm = "b%d_%d" % (n, ki)
            L.append(ind + "const R %s = %s;" % (nm, tree_sum(ex)))
            names.append(nm)
        return names

    for n in range(len(dag.nodes) - 1, -1, -1):
        key, rank = dag.nodes[n]
        names = flush(n)
        if all(x is None for x in names):
            continue
        if key[0] == "M":
            _, mu, nu, off = key
            for ki, K in enumerate(multi_indices(rank)):
                if names[ki] is None:
                    continue
                full = (off[0] + K[0], off[1] + K[1], off[2] + K[2])
                dcontrib[lv.comp_index[(mu, full)]].append(names[ki])
            continue
        _, a, b = key
        p = dag.rank(b)
        Ps = multi_indices(p)
        ra = dag.rank(a)
        # A-adjoint: Abar[K+P] += Cbar[K] * Bw[P]
        # B-adjoint: Bbar[P] += w_P * sum_K Cbar[K] A[K+P]
        bacc = defaultdict(list)
        for ki, K in enumerate(multi_indices(rank)):
            if names[ki] is None:
                continue
            for j, P in enumerate(Ps):
                full = (K[0] + P[0], K[1] + P[1], K[2] + P[2])
                if dag.nodes[a][0][0] == "M" or True:
                    aidx = multi_indices(ra).index(full)
                    adj[(a, aidx)].append("%s * %s" % (names[ki], wname[n][j]))
                bacc[j].append((names[ki], comp_ref(a, full)))
        for j, lst in bacc.items():
            P = Ps[j]
            w = multinomial_weight(P)
            nm = "c%d_%d" % (n, j)
            emit_dot(L, ind, nm, lst)
            bidx = j
            adj[(b, bidx)].append(nm if w == 1 else "R(%d) * %s" % (w, nm))
    # adjoints of the formed components go to the swept ones they came from
    # (reverse of the expansion, in decreasing z-exponent)
    dneg = defaultdict(list)
    for c in sorted(lv.expand, key=lambda t: (-lv.comps[t][1][2], -t)):
        if not dcontrib.get(c) and not dneg.get(c):
            continue
        nm = "dx%d" % c
        pos = tree_sum(dcontrib.get(c, [])) if dcontrib.get(c) else "R(0)"
        L.append(ind + "const R %s = %s;" % (nm, pos if not dneg.get(c) else "%s - %s" % (pos, tree_sum(dneg[c]))))
        s0, s1, s2 = lv.expand[c]
        dcontrib[s0].append(nm)
        dneg[s1].append(nm)
        dneg[s2].append(nm)
    for c in range(len(lv.comps)):
        if c in lv.expand:
            L.append(ind + "D[%d] = R(0);" % c)
            continue
        ex = dcontrib.get(c)
        neg = dneg.get(c)
        if neg:
            L.append(ind + "D[%d] = %s - %s;" % (c, tree_sum(ex) if ex else "R(0)", tree_sum(neg)))
        else:
            L.append(ind + "D[%d] = %s;" % (c, tree_sum(ex)))
    L.append(ind + "return E;")
    L.append("  }")
    return L




def _node_closure(dag, roots):
    """C nodes and M leaves reachable from the (weight, node) roots."""
    seen = set()
    stack = [node for _, node in roots]
    while stack:
        n = stack.pop()
        if n in seen:
            continue
        seen.add(n)
        key = dag.nodes[n][0]
        if key[0] == "C":
            stack += [key[1], key[2]]
    return seen


def emit_contract_by_graph(lv: Level, fname="contract"):
    """Same results as emit_contract (up to rounding order), with the reverse
    pass run graph by graph: each graph's DAG nodes are formed again from the
    moments (read through an optimisation barrier, so that the compiler forms
    them anew instead of keeping the forward pass's values) and their adjoints
    are added into the D accumulators at once.  Across the reverse pass only
    the moments, the D accumulators and the graph adjoints stay live, instead
    of every node value of the DAG."""
    dag = lv.dag
    L = []
    ind = "    "
    L.append("  template <class R, bool WANT_B, class MV = const R*, class BV = R*>")
    L.append("  __device__ __forceinline__ static R %s(MV M, "
             "const typename ScalarOf<R>::T* __restrict__ xi, R* __restrict__ D, BV B) {" % fname)
    L.append(ind + "(void)B;")
    exp_order = sorted(lv.expand, key=lambda t: (lv.comps[t][1][2], t))

    def emit_nodes(nodes, mname, sfx):
        """Forward values of the C nodes in `nodes`; M component c is mname(c)."""
        wname = {}

        def comp_ref(n, K):
            key, rank = dag.nodes[n]
            if key[0] == "M":
                _, mu, nu, off = key
                return mname(lv.comp_index[(mu, (off[0] + K[0], off[1] + K[1], off[2] + K[2]))])
            return "v%d_%d%s" % (n, multi_indices(rank).index(K), sfx)

        for n in sorted(nodes):
            key, rank = dag.nodes[n]
            if key[0] != "C":
                continue
            _, a, b = key
            Ps = multi_indices(dag.rank(b))
            wn = []
            for j, P in enumerate(Ps):
                w = multinomial_weight(P)
                if w == 1:
                    wn.append(comp_ref(b, P))
                else:
                    nm = "w%d_%d%s" % (n, j, sfx)
                    L.append(ind + "const R %s = R(%d) * %s;" % (nm, w, comp_ref(b, P)))
                    wn.append(nm)
            wname[n] = wn
            for ki, K in enumerate(multi_indices(rank)):
                terms = [(comp_ref(a, (K[0] + P[0], K[1] + P[1], K[2] + P[2])), wn[j]) for j, P in enumerate(Ps)]
                emit_dot(L, ind, "v%d_%d%s" % (n, ki, sfx), terms)
        return comp_ref, wname

    # forward pass: formed moment components, every node, graphs, basis, E
    for c in exp_order:
        s0, s1, s2 = (("M[%d]" % t) if t not in lv.expand else ("mx%d" % t) for t in lv.expand[c])
        L.append(ind + "const R mx%d = (%s - %s) - %s;" % (c, s0, s1, s2))
    comp_ref, _ = emit_nodes(range(len(dag.nodes)), lambda c: ("mx%d" % c) if c in lv.expand else ("M[%d]" % c), "")
    for gi, roots in enumerate(lv.roots):
        parts = []
        for w, node in roots:
            ref = comp_ref(node, (0, 0, 0))
            parts.append(ref if w == 1 else "R(%d) * %s" % (w, ref))
        L.append(ind + "const R G%d = %s;" % (gi, tree_sum(parts)))
    L.append(ind + "R E = R(0);")
    for a, b in enumerate(lv.bases):
        L.append(ind + "const R B%d = %s;" % (a, " * ".join("G%d" % k for k in b)))
        L.append(ind + "if (WANT_B) store_basis(B, %d, B%d);" % (a, a))
        L.append(ind + "E = fmadd(R(xi[%d]), B%d, E);" % (a, a))
    gbar = defaultdict(list)
    for a, b in enumerate(lv.bases):
        for j in range(len(b)):
            others = [b[t] for t in range(len(b)) if t != j]
            gbar[b[j]].append((a, others))
    for gi in range(len(lv.graphs)):
        terms = []
        for a, others in gbar[gi]:
            prod = " * ".join("G%d" % k for k in others)
            terms.append("R(xi[%d])" % a + (" * " + prod if prod else ""))
        L.append(ind + "const R Gb%d = %s;" % (gi, tree_sum(terms)))
    # reverse pass, graph by graph
    for c in range(len(lv.comps)):
        L.append(ind + "D[%d] = R(0);" % c)
    for gi, roots in enumerate(lv.roots):
        sfx = "_g%d" % gi
        nodes = _node_closure(dag, roots)
        # moment components the graph reads (and the swept ones they are formed from)
        used = set()
        for n in nodes:
            key, rank = dag.nodes[n]
            if key[0] == "M":
                _, mu, nu, off = key
                for K in multi_indices(rank):
                    used.add(lv.comp_index[(mu, (off[0] + K[0], off[1] + K[1], off[2] + K[2]))])
        stack = list(used)
        while stack:
            c = stack.pop()
            for t in lv.expand.get(c, ()):
                if t not in used:
                    used.add(t)
                    stack.append(t)

        def mname(c, sfx=sfx):
            return ("mx%d%s" % (c, sfx)) if c in lv.expand else ("m%d%s" % (c, sfx))

        for c in sorted(t for t in used if t not in lv.expand):
            L.append(ind + "R %s = M[%d];" % (mname(c), c))
            L.append(ind + "opaque(%s);" % mname(c))
        for c in exp_order:
            if c in used:
                s0, s1, s2 = (mname(t) for t in lv.expand[c])
                L.append(ind + "const R %s = (%s - %s) - %s;" % (mname(c), s0, s1, s2))
        cref, wname = emit_nodes(nodes, mname, sfx)
        adj = defaultdict(list)
        for w, node in roots:
            adj[(node, 0)].append("Gb%d" % gi if w == 1 else "R(%d) * Gb%d" % (w, gi))
        dpos, dneg = defaultdict(list), defaultdict(list)
        for n in sorted(nodes, reverse=True):
            key, rank = dag.nodes[n]
            names = []
            for ki in range(n_sym(rank)):
                ex = adj.get((n, ki))
                if not ex:
                    names.append(None)
                    continue
                nm = "b%d_%d%s" % (n, ki, sfx)
                L.append(ind + "const R %s = %s;" % (nm, tree_sum(ex)))
                names.append(nm)
            if key[0] == "M":
                _, mu, nu, off = key
                for ki, K in enumerate(multi_indices(rank)):
                    if names[ki] is not None:
                        dpos[lv.comp_index[(mu, (off[0] + K[0], off[1] + K[1], off[2] + K[2]))]].append(names[ki])
                continue
            _, a, b = key
            Ps = multi_indices(dag.rank(b))
            ra = dag.rank(a)
            bacc = defaultdict(list)
            for ki, K in enumerate(multi_indices(rank)):
                if names[ki] is None:
                    continue
                for j, P in enumerate(Ps):
                    full = (K[0] + P[0], K[1] + P[1], K[2] + P[2])
                    adj[(a, multi_indices(ra).index(full))].append("%s * %s" % (names[ki], wname[n][j]))
                    bacc[j].append((names[ki], cref(a, full)))
            for j, lst in bacc.items():
                w = multinomial_weight(Ps[j])
                nm = "c%d_%d%s" % (n, j, sfx)
                emit_dot(L, ind, nm, lst)
                adj[(b, j)].append(nm if w == 1 else "R(%d) * %s" % (w, nm))
        # this graph's adjoints of formed components go to the swept ones
        for c in sorted(lv.expand, key=lambda t: (-lv.comps[t][1][2], -t)):
            if not dpos.get(c) and not dneg.get(c):
                continue
            nm = "dx%d%s" % (c, sfx)
            pos = tree_sum(dpos[c]) if dpos.get(c) else "R(0)"
            L.append(ind + "const R %s = %s;" % (nm, pos if not dneg.get(c) else "%s - %s" % (pos, tree_sum(dneg[c]))))
            s0, s1, s2 = lv.expand[c]
            dpos[s0].append(nm)
            dneg[s1].append(nm)
            dneg[s2].append(nm)
        for c in sorted(set(dpos) | set(dneg)):
            if c in lv.expand:
                continue
            ex = "D[%d]" % c
            if dpos.get(c):
                ex = "%s + %s" % (ex, tree_sum(dpos[c]))
            if dneg.get(c):
                ex = "(%s) - %s" % (ex, tree_sum(dneg[c]))
            L.append(ind + "D[%d] = %s;" % (c, ex))
    L.append(ind + "return E;")
    L.append("  }")
    return L


# Contraction code shape for the straight-line levels in FP32: the reverse
# pass graph by graph with recomputed nodes (True) or over the whole DAG
# (False).  FP64 and dual-number code always take the whole-DAG form (the
# recomputation costs FP64-pipe time: 46.5 against 44.4 ms for the
# 1,024,000-atom FP64 evaluation).
CONTRACT_BY_GRAPH = True


def emit_contract_dispatch():
    """contract(): the per-graph form for FP32, the whole-DAG form otherwise."""
    return ["  template <class R, bool WANT_B, class MV = const R*, class BV = R*>",
            "  __device__ __forceinline__ static R contract(MV M, "
            "const typename ScalarOf<R>::T* __restrict__ xi, R* __restrict__ D, BV B) {",
            "    if constexpr (std::is_same<R, float>::value)",
            "      return contract_graph<R, WANT_B, MV, BV>(M, xi, D, B);",
            "    else",
            "      return contract_dag<R, WANT_B, MV, BV>(M, xi, D, B);",
            "  }"]


def emit_contract_program(lv: Level):
    """Contraction as a program for a per-thread interpreter (levels whose
    straight-line code would be too large).  Values V: [0, C) moment
    components, then every DAG node component, a constant 1, the graph values
    and the basis values.  Records (int32): DOT = [0, dst, n, (a, b, w) * n]
    meaning V[dst] = sum w V[a] V[b]; PROD = [1, dst, n, g * n] meaning
    V[dst] = prod V[g].  Forward runs the records in order, the reverse pass
    in reverse order."""
    dag = lv.dag
    C = len(lv.comps)
    base = {}
    nv = C
    for n, (key, rank) in enumerate(dag.nodes):
        if key[0] == "C":
            base[n] = nv
            nv += n_sym(rank)
    one = nv
    nv += 1
    goff = nv
    nv += len(lv.graphs)
    boff = nv
    nv += lv.m

    def ref(n, K):
        key, rank = dag.nodes[n]
        if key[0] == "M":
            _, mu, nu, off = key
            return lv.comp_index[(mu, (off[0] + K[0], off[1] + K[1], off[2] + K[2]))]
        return base[n] + multi_indices(rank).index(K)

    prog, starts = [], []
    # moment components the sweeps leave out (z-exponent >= 2), formed first
    # from the swept ones: V[c] = V[s0] - V[s1] - V[s2] (the reverse pass then
    # adds their adjoints into the swept components)
    for c in sorted(lv.expand, key=lambda t: (lv.comps[t][1][2], t)):
        s0, s1, s2 = lv.expand[c]
        starts.append(len(prog))
        prog += [0, c, 3, s0, one, 1, s1, one, -1, s2, one, -1]
    for n, (key, rank) in enumerate(dag.nodes):
        if key[0] != "C":
            continue
        _, a, b = key
        Ps = multi_indices(dag.rank(b))
        for ki, K in enumerate(multi_indices(rank)):
            starts.append(len(prog))
            prog += [0, base[n] + ki, len(Ps)]
            for P in Ps:
                prog += [ref(a, (K[0] + P[0], K[1] + P[1], K[2] + P[2])), ref(b, P), multinomial_weight(P)]
    for gi, roots in enumerate(lv.roots):
        starts.append(len(prog))
        prog += [0, goff + gi, len(roots)]
        for w, node in roots:
            prog += [ref(node, (0, 0, 0)), one, w]
    for a_, bas in enumerate(lv.bases):
        starts.append(len(prog))
        prog += [1, boff + a_, len(bas)] + [goff + k for k in bas]
    # dependency levels of the records (for the warp-parallel interpreter):
    # a record's level is one more than the highest level among the records
    # that produce its inputs (moments and the constant 1 are level 0)
    vlevel = {}
    rlevel = []
    for st in starts:
        typ, dst, cnt = prog[st], prog[st + 1], prog[st + 2]
        if typ == 0:
            ins = [prog[st + 3 + 3 * t] for t in range(cnt)] + [prog[st + 4 + 3 * t] for t in range(cnt)]
        else:
            ins = [prog[st + 3 + t] for t in range(cnt)]
        lev = 1 + max(vlevel.get(v, 0) for v in ins)
        vlevel[dst] = lev
        rlevel.append(lev)
    nlev = max(rlevel)
    order = sorted(range(len(starts)), key=lambda r: (rlevel[r], r))
    level_off = [0] * (nlev + 1)
    for r in order:
        level_off[rlevel[r]] += 1
    for k in range(1, nlev + 1):
        level_off[k] += level_off[k - 1]
    L = []
    nm = "L%d" % lv.level
    L.append("  static constexpr int NVALUES = %d, ONE = %d, BOFF = %d, NRECORDS = %d;" % (nv, one, boff, len(starts)))
    L.append("  static constexpr int NLEVELS = %d;   // dependency levels of the records" % nlev)
    L.append("  template <class R, bool WANT_B>")
    L.append("  __device__ static R contract(const R* __restrict__ M, const typename ScalarOf<R>::T* __restrict__ xi, "
             "R* __restrict__ D, R* __restrict__ B) {")
    L.append("    return interpret_contract<R, WANT_B, NCOMP, NVALUES, ONE, BOFF, NBASIS, NRECORDS>("
             "kProg%s, kStarts%s, M, xi, D, B);" % (nm, nm))
    L.append("  }")
    L.append("  // one warp: V, A shared arrays of NVALUES (V[0, NCOMP) = moments on entry, A[0, NCOMP) = dE/dM on")
    L.append("  // return); the records of each dependency level are spread over the lanes")
    L.append("  template <class R, bool WANT_B, class BV>")
    L.append("  __device__ static R contract_warp(R* V, R* A, const typename ScalarOf<R>::T* __restrict__ xi, BV B, "
             "int lane) {")
    L.append("    return interpret_values_warp<R, WANT_B, NCOMP, NVALUES, ONE, BOFF, NBASIS, NLEVELS>("
             "kProg%s, kStarts%s, kLevelOrder%s, kLevelOff%s, V, A, xi, B, lane);" % (nm, nm, nm, nm))
    L.append("  }")
    L.append("  // V[0, NCOMP) = moments on entry, A[0, NCOMP) = dE/dM on return (arrays of NVALUES)")
    L.append("  template <class R, bool WANT_B>")
    L.append("  __device__ static R contract_values(R* V, R* A, const typename ScalarOf<R>::T* __restrict__ xi, "
             "R* B) {")
    L.append("    return interpret_values<R, WANT_B, NCOMP, NVALUES, ONE, BOFF, NBASIS, NRECORDS>("
             "kProg%s, kStarts%s, V, A, xi, B);" % (nm, nm))
    L.append("  }")
    tables = ["__device__ const int32_t kProg%s[] = {%s};" % (nm, ",".join(str(v) for v in prog)),
              "__device__ const int32_t kStarts%s[] = {%s};" % (nm, ",".join(str(v) for v in starts)),
              "__device__ const int32_t kLevelOrder%s[] = {%s};" % (nm, ",".join(str(v) for v in order)),
              "__device__ const int32_t kLevelOff%s[] = {0,%s};" % (nm, ",".join(str(v) for v in level_off[1:]))]
    return L, tables


def emit_groups(lv: Level):
    """Per component group G: moments_group<G>, pair_adjoint_group<G> (the
    group's terms only; S[mu] of other groups set to zero), store_group<G>
    (group components of a register array into a full vector with stride
    ld) and load_group<G>, plus the radial-function range [MU_LO, MU_HI)."""
    L = []
    ng = len(lv.groups)
    for g, grp in enumerate(lv.groups):
        sub = set(grp)
        L += emit_moments(lv, sub, "moments_g%d" % g)
        L += emit_pair_adjoint(lv, sub, "pair_adjoint_g%d" % g)
        L.append("  template <class R>")
        L.append("  __device__ __forceinline__ static void store_g%d(const R* __restrict__ Mg, R* __restrict__ M, "
                 "int64_t ld) {" % g)
        # only swept components travel (the others are formed in the contraction)
        L += ["    M[%d * ld] = Mg[%d];" % (c, c) for c in grp if c not in lv.expand]
        L.append("  }")
        L.append("  template <class R>")
        L.append("  __device__ __forceinline__ static void load_g%d(const R* __restrict__ D, int64_t ld, "
                 "R* __restrict__ Dg) {" % g)
        L += ["    Dg[%d] = D[%d * ld];" % (c, c) for c in grp if c not in lv.expand]
        L.append("  }")
    for grp in lv.groups:
        assert sorted(grp) == list(range(min(grp), max(grp) + 1)), "component groups are contiguous ranges"
    L.append("  static constexpr int GROUP_C_LO[%d] = {%s};" % (ng, ", ".join(str(min(g)) for g in lv.groups)))
    L.append("  static constexpr int GROUP_C_HI[%d] = {%s};" % (ng, ", ".join(str(max(g) + 1) for g in lv.groups)))
    mus = [sorted({lv.comps[c][0] for c in grp}) for grp in lv.groups]
    L.append("  static constexpr int GROUP_MU_LO[%d] = {%s};" % (ng, ", ".join(str(m[0]) for m in mus)))
    L.append("  static constexpr int GROUP_MU_HI[%d] = {%s};" % (ng, ", ".join(str(m[-1] + 1) for m in mus)))
    for fn, args, call in (
            ("moments_group", "R* __restrict__ M, const R* __restrict__ f, R ux, R uy, R uz", "(M, f, ux, uy, uz)"),
            ("pair_adjoint_group", "const R* __restrict__ D, const R* __restrict__ f, const R* __restrict__ df, "
             "R ux, R uy, R uz, R rinv, R& gx, R& gy, R& gz, R* __restrict__ S",
             "(D, f, df, ux, uy, uz, rinv, gx, gy, gz, S)"),
            ("store_group", "const R* __restrict__ Mg, R* __restrict__ M, int64_t ld", "(Mg, M, ld)"),
            ("load_group", "const R* __restrict__ D, int64_t ld, R* __restrict__ Dg", "(D, ld, Dg)")):
        base = {"moments_group": "moments_g", "pair_adjoint_group": "pair_adjoint_g",
                "store_group": "store_g", "load_group": "load_g"}[fn]
        L.append("  template <int G, class R>")
        L.append("  __device__ __forceinline__ static void %s(%s) {" % (fn, args))
        for g in range(ng):
            kw = "if" if g == 0 else "else if"
            L.append("    %s constexpr (G == %d) %s%d<R>%s;" % (kw, g, base, g, call))
        L.append("  }")
    return L


def emit_header(lv: Level):
    name = "MtpLevel%d" % lv.level
    out = []
    out.append("// Generated by paper_2510_00193_gb300/basisgen.py for MTP level %d. Do not edit." % lv.level)
    out.append("#pragma once")
    out.append("#include \"mtp_math.cuh\"")
    out.append("#include \"mtp_interp.cuh\"")
    out.append("namespace mtp {")
    out.append("struct %s {" % name)
    out.append("  static constexpr int LEVEL = %d;" % lv.level)
    out.append("  static constexpr int NMU = %d;" % lv.nmu)
    out.append("  static constexpr int NCOMP = %d;" % len(lv.comps))
    out.append("  static constexpr int NBASIS = %d;" % lv.m)
    out.append("  static constexpr int NGRAPH = %d;" % len(lv.graphs))
    out.append("  static constexpr int NUMAX = %d;" % max(lv.nu_max))
    out.append("  static constexpr int NGROUPS = %d;" % len(lv.groups))
    out += emit_moments(lv)
    out += emit_pair_adjoint(lv)
    if len(lv.groups) > 1:
        out += emit_groups(lv)
    if lv.level >= INTERPRET_FROM_LEVEL:
        body, tables = emit_contract_program(lv)
        out = out[:out.index("struct %s {" % name)] + tables + out[out.index("struct %s {" % name):]
        out += body
    else:
        out += emit_contract(lv, "contract_dag")
        out += (emit_contract_by_graph(lv, "contract_graph") if CONTRACT_BY_GRAPH
                else emit_contract(lv, "contract_graph"))
        out += emit_contract_dispatch()
    out.append("};")
    out.append("}  // namespace mtp")
    return "\n".join(out) + "\n"


def emit_tables(levels):
    """Host tables: per level the basis functions as factor lists of graphs,
    graphs as (nv, mu[], e[]), and each graph's expanded polynomial."""
    out = ["// Generated by paper_2510_00193_gb300/basisgen.py. Do not edit.", "#pragma once",
           "#include <cstdint>", "namespace mtp { namespace tables {"]
    entries = []
    for lv in levels:
        L = lv.level
        gdata = []
        for g in lv.graphs:
            gdata += [g.nv] + list(g.mu) + list(g.e)
        bdata = []
        for b in lv.bases:
            bdata += [len(b)] + list(b)
        pdata = []
        nterms = 0
        for g in lv.graphs:
            poly = sorted(expand_graph(g).items())
            pdata.append(len(poly))
            for mono, coef in poly:
                pdata.append(coef)
                for mu, K in mono:
                    pdata += [mu, K[0], K[1], K[2]]
                nterms += 1
        cdata = []
        for mu, K in lv.comps:
            cdata += [mu, K[0], K[1], K[2]]
        for nm, arr in (("graphs", gdata), ("bases", bdata), ("poly", pdata), ("comps", cdata)):
            out.append("static const int64_t L%d_%s[] = {%s};" % (L, nm, ",".join(str(v) for v in arr) or "0"))
        entries.append("  {%d, %d, %d, %d, %d, L%d_graphs, %d, L%d_bases, %d, L%d_poly, %d, L%d_comps, %d, %d}" % (
            L, lv.nmu, lv.m, len(lv.graphs), len(lv.comps), L, len(gdata), L, len(bdata), L, len(pdata), L,
            len(cdata), lv.n_enumerated))
    out.append("struct LevelTable { int level, nmu, m, ngraph, ncomp; const int64_t* graphs; int64_t ngraphs_len;"
               " const int64_t* bases; int64_t nbases_len; const int64_t* poly; int64_t npoly_len;"
               " const int64_t* comps; int64_t ncomps_len; int n_enumerated; };")
    out.append("static const LevelTable kLevels[] = {")
    out.append(",\n".join(entries))
    out.append("};")
    out.append("static const int kNumLevels = %d;" % len(levels))
    out.append("}}  // namespace mtp::tables")
    return "\n".join(out) + "\n"


LEVELS = (2, 4, 6, 8, 10, 12, 14, 16, 18, 20)


def generate(outdir, levels=LEVELS):
    os.makedirs(outdir, exist_ok=True)
    lvs = [Level(L) for L in levels]
    written = []
    for lv in lvs:
        path = os.path.join(outdir, "mtp_level%d.cuh" % lv.level)
        _write_if_changed(path, emit_header(lv))
        written.append(path)
    path = os.path.join(outdir, "mtp_tables.h")
    _write_if_changed(path, emit_tables(lvs))
    written.append(path)
    return written


def _write_if_changed(path, text):
    if os.path.exists(path):
        with open(path) as fh:
            if fh.read() == text:
                return
    with open(path, "w") as fh:
        fh.write(text)


if __name__ == "__main__":
    lv = [int(a) for a in sys.argv[2:]] or list(LEVELS)
    generate(sys.argv[1], lv)


# ---------------------------------------------------------------------------
# floating-point operation counts of the generated code (for roofline figures)
# ---------------------------------------------------------------------------


def _flops_of(lines):
    """fmadd = 2 flops, every other binary * + - = 1 flop (integer constants
    folded into R(k) * x count as one multiply)."""
    import re
    total = 0
    for ln in lines:
        code = ln.split("//")[0]
        if "=" not in code or code.strip().startswith(("template", "__device__", "}", "(void)", "if (WANT_B)")):
            continue
        rhs = code.split("=", 1)[1]
        total += 2 * rhs.count("fmadd(")
        total += len(re.findall(r"[^\s(,]\s*[\*\+\-]\s*[^\s)]", rhs.replace("fmadd(", "(")))
    return total


def flop_counts(lv, sweep_all=False):
    """Per-pair and per-atom flop counts of the generated functions.  With
    sweep_all, of the code that sweeps every Cartesian component (the
    method's operation count as written, without the reduction on the unit
    sphere)."""
    saved = lv.expand, lv.swept
    if sweep_all:
        lv.expand, lv.swept = {}, list(range(len(lv.comps)))
    try:
        keys = {K for c, (mu, K) in enumerate(lv.comps) if c not in lv.expand}
        n_mono = len(_closure(keys))
        mom = emit_moments(lv)
        adj = emit_pair_adjoint(lv)
        # algorithmic count: the whole-DAG contraction; executed (FP32): the
        # form the FP32 kernels run
        con = []
        if lv.level < INTERPRET_FROM_LEVEL:
            con = (emit_contract_by_graph(lv) if (CONTRACT_BY_GRAPH and not sweep_all) else emit_contract(lv))
    finally:
        lv.expand, lv.swept = saved
    return {
        "monomials": n_mono,
        "moments": _flops_of(mom) - n_mono,
        "pair_adjoint": _flops_of(adj) - n_mono,
        "contract": _flops_of(con),
        "ncomp": len(lv.comps),
        "nswept": len(lv.comps) if sweep_all else len(lv.swept),
    }
