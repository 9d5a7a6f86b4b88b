"""The C-ABI library loads, exports every declared symbol, and its basis tables
equal the oracle's bit for bit.  Host-only calls; no GPU needed."""
import ctypes
import os
import re

import pytest

import synth
from oracle import mtp as O

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def lib():
    from paper_2510_00193_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    import paper_2510_00193_gb300 as P
    return P


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "mtp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(mtp_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2510_00193_gb300 import _lib
    so = _lib.load()
    names = _declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(so, name), name
        assert name in _lib.SIGNATURES, name


@pytest.mark.parametrize("level", [2, 8, 12, 16])
def test_basis_table_matches_oracle_bit_exactly(lib, level):
    graphs, bases = lib.decode_basis(level)
    u, f = synth.random_neighbourhoods(3 * len(O.basis_functions(level)), 16, O.n_mu_for_level(level),
                                       synth.rng(99, level))
    ob = O.make_basis(level, u, f)
    assert graphs == [(g.mu, g.e) for g in ob.graphs]
    assert bases == ob.bases
    info = lib.mtp_basis_info(level)
    assert info["m"] == ob.m and info["n_mu"] == ob.n_mu


@pytest.mark.parametrize("level", [8, 12, 16])
def test_graph_polynomials_match_cartesian_expansion(lib, level):
    """Multinomial expansion (library) == brute force over Cartesian indices (oracle)."""
    graphs, _ = lib.decode_basis(level)
    poly = lib.mtp_basis_table(level, 2).tolist()
    k = 0
    for mu, e in graphs:
        g = O.Graph(mu, e)
        nterms = poly[k]
        k += 1
        mine = {}
        for _ in range(nterms):
            coef = poly[k]
            k += 1
            mono = []
            for _v in range(g.nv):
                m_, a, b, c = poly[k:k + 4]
                k += 4
                mono.append((m_, (a, b, c)))
            mine[tuple(sorted(mono))] = coef
        assert mine == O.expand_cartesian(g)
    assert k == len(poly)


def test_component_layout_covers_moment_tensors(lib):
    comps = lib.mtp_basis_table(16, 3).reshape(-1, 4).tolist()
    assert len(comps) == lib.mtp_basis_info(16)["n_comp"] == 130
    lay = O.moment_layout(O.connected_graphs(16))
    want = sorted((mu, a, b, nu - a - b) for mu, nu in lay for a in range(nu + 1) for b in range(nu - a + 1))
    assert sorted(map(tuple, comps)) == want


def test_errors_are_reported_not_raised_as_crashes(lib):
    from paper_2510_00193_gb300 import _lib
    so = _lib.load()
    m = ctypes.c_int32()
    assert so.mtp_basis_info(7, ctypes.byref(m), None, None, None) == -7
    assert b"level 7" in so.mtp_last_error()
    n = ctypes.c_int64()
    assert so.mtp_basis_table(16, 9, None, ctypes.byref(n)) == -1
    assert so.mtp_load_params(None, None) == -1


def test_new_entry_points_refuse_bad_arguments_on_the_host(lib):
    """Argument checks of the MD, MaxVol and basis-row entry points run on the
    host before any device work (no GPU needed): each returns MTP_ERR_ARG with
    a message."""
    from paper_2510_00193_gb300 import _lib
    so = _lib.load()
    fake = ctypes.c_void_p(0x1000)   # never dereferenced: the checks fail first
    rows = (ctypes.c_int32 * 3)(0, 1, 1)
    it = ctypes.c_int32()
    # duplicate initial rows
    assert so.mtp_maxvol(fake, 10, 3, rows, 0.01, 100, fake, ctypes.byref(it), None) == -1
    assert b"distinct" in so.mtp_last_error()
    # row out of range, m > n_pool, negative delta, m beyond the limit
    rows2 = (ctypes.c_int32 * 3)(0, 1, 10)
    assert so.mtp_maxvol(fake, 10, 3, rows2, 0.01, 100, fake, None, None) == -1
    assert so.mtp_maxvol(fake, 2, 3, rows, 0.01, 100, fake, None, None) == -1
    assert so.mtp_maxvol(fake, 10, 3, rows, -1.0, 100, fake, None, None) == -1
    assert so.mtp_maxvol(fake, 10 ** 6, 5000, rows, 0.01, 100, fake, None, None) == -1
    # MD and basis rows without a handle
    cell = (ctypes.c_double * 9)(10, 0, 0, 0, 10, 0, 0, 0, 10)
    pbc = (ctypes.c_int32 * 3)(1, 1, 1)
    out = ctypes.c_void_p()
    assert so.mtp_md_create(None, fake, 4, cell, pbc, 0.3, ctypes.byref(out), None) == -1
    assert so.mtp_md_run(None, None, fake, fake, fake, None, 1e-3, 1, 0, 1, fake, None, None, None) == -1
    assert so.mtp_md_status(None, None, None, None) == -1
    assert so.mtp_compute_basis_rows(None, None, fake, fake, 4, cell, fake, None) == -1
    so.mtp_md_free(None)
