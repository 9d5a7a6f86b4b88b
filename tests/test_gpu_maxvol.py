"""MaxVol active-set selection (mtp_maxvol) and FP64 basis rows
(mtp_compute_basis_rows) against the oracle, through the C-ABI.

Tolerances: selected rows and swap counts bit-exact against oracle.mtp.maxvol
on well-conditioned random pools (same initial rows, same tie rule); the final
A^-1 within 1e-12 of the largest entry (the same Gauss-Jordan steps; the pools
differ only in the order of the products' sums, which can move an entry by a
few units in the last place); basis rows within 1e-10 relative to the row's
largest entry (FP64, other summation order).  On the 16,000-atom lattice pool,
whose rows are nearly degenerate, the result is checked by what MaxVol
guarantees: every pool row has grade <= 1 + delta (+1e-5 for FP64 rounding
times the cancellation of these rows) and the active rows have grade 1.
"""
import numpy as np
import pytest

import synth
from oracle import mtp as O
from tests.helpers import min_image_candidates, oracle_model, pot_dict

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_00193_gb300 import build as B
    B.build()
    import paper_2510_00193_gb300 as P
    return P


def random_pool(n, m, seed):
    g = synth.rng(seed, 0)
    return g.normal(size=(n, m)) * np.exp(g.normal(size=m))


@pytest.mark.parametrize("n,m,seed", [(3000, 24, 1), (517, 9, 2), (64, 1, 4), (2000, 128, 4)])
def test_maxvol_matches_oracle(P, n, m, seed):
    pool = random_pool(n, m, seed)
    init = synth.rng(seed, 1).permutation(n)[:m]    # a poor start, so that rows get swapped
    rows_o, a_inv_o, it_o = O.maxvol(pool, rows=init.copy(), delta=0.01)
    rows_g, a_inv_g, it_g = P.mtp_maxvol(torch.tensor(pool, device="cuda"), init, delta=0.01)
    assert it_o > 0
    assert np.array_equal(rows_g, rows_o)
    assert it_g == it_o
    a = a_inv_g.cpu().numpy()
    assert np.abs(a - a_inv_o).max() <= 1e-12 * np.abs(a_inv_o).max()
    gam = O.grade(pool, a)
    assert gam.max() <= 1.01 + 1e-9


def test_maxvol_edge_cases(P):
    pool = random_pool(300, 12, 5)
    dev = torch.tensor(pool, device="cuda")
    init = O.initial_rows(pool)
    # no swap allowed: the initial rows and their inverse
    rows, a_inv, it = P.mtp_maxvol(dev, init, max_iter=0)
    assert it == 0 and np.array_equal(rows, init)
    assert np.abs(a_inv.cpu().numpy() - O.invert(pool[init])).max() <= 1e-12 * np.abs(O.invert(pool[init])).max()
    # a converged set stays
    rows1, _, _ = P.mtp_maxvol(dev, init)
    rows2, _, it2 = P.mtp_maxvol(dev, rows1)
    assert it2 == 0 and np.array_equal(rows1, rows2)
    # a pool of exactly m rows: nothing to swap
    sq = torch.tensor(pool[:12], device="cuda")
    rows, _, it = P.mtp_maxvol(sq, np.arange(12))
    assert it == 0 and np.array_equal(rows, np.arange(12))
    # invalid input is refused on the host or reported, nothing runs wild
    for bad in (np.r_[init[:-1], init[0]], np.r_[init[:-1], 300], np.r_[init[:-1], -1]):
        with pytest.raises(P.MtpError) as err:
            P.mtp_maxvol(dev, bad)
        assert err.value.code == -1
    # a zero row in the active set: zero pivot, reported as MTP_ERR_ARG
    zero = pool.copy()
    zero[0] = 0.0
    with pytest.raises(P.MtpError) as err:
        P.mtp_maxvol(torch.tensor(zero, device="cuda"), np.arange(12))
    assert err.value.code == -1


def test_basis_rows_and_maxvol_on_the_lattice_pool(P):
    """The neighbourhood-mode pool of the grade workload: every atom of a
    20^3-cell BCC box (16,000 atoms, sigma 0.05 A), level 16, one species."""
    st = synth.crystal("bcc", (20, 20, 20), 3.16, 0.05, 1, 5, sub=8)
    pot = P.Potential.from_dict(pot_dict("bcc-l16-s1"))
    x = torch.tensor(st.x, device="cuda")
    z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    rows_dev = P.mtp_compute_basis_rows(pot, nl, x, z, st.cell)
    pool = rows_dev.cpu().numpy()
    # sampled rows against the oracle
    model = oracle_model("bcc-l16-s1")
    centres = np.array([0, 7777, 15999])
    cand = min_image_candidates(st, centres, 5.5)
    nlo = O.neighbor_list(st.x, st.cell, st.pbc, 5.0, query=centres, candidates=cand)
    ref = O.basis_matrix(model, st.x, st.z, st.cell, nlo, atoms=centres)
    for k, c in enumerate(centres):
        assert np.abs(pool[c] - ref[k]).max() <= 1e-10 * np.abs(ref[k]).max()
    init = O.initial_rows(pool)
    rows, a_inv, it = P.mtp_maxvol(rows_dev, init, delta=0.01)
    assert it > 0 and len(set(rows.tolist())) == pool.shape[1]
    gam = O.grade(pool, O.invert(pool[rows]))
    assert gam.max() <= 1.01 + 1e-5
    assert np.all(np.abs(gam[rows] - 1.0) <= 1e-5)
