"""Extrapolation grade (neighbourhood and configuration mode) against the
oracle: flags bit-exact, grades within 1e-7 relative, for both products: the
tensor-core method (error-free BF16 slicing, FP64 re-check near the
thresholds) and the FP64 method.  The products cancel by ~5e7 on these
active sets, so FP64 rounding alone reaches ~1e-8 relative; 1e-7 leaves a
margin."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import mtp as O
from tests.helpers import ROOT, min_image_candidates, oracle_model, pot_dict

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TAU_SEL, TAU_BRK = 2.0, 10.0


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_00193_gb300 import build as B
    B.build()
    import paper_2510_00193_gb300 as P
    return P


@pytest.fixture(scope="module")
def active():
    with open(os.path.join(ROOT, "potentials", "bcc-l16-s1-active.json")) as fh:
        d = json.load(fh)
    m = d["m"]
    return np.array(d["a_inv"]).reshape(m, m), np.array(d["a_inv_cfg"]).reshape(m, m), d


def run(P, st, a_inv, a_cfg, method=None, chunk_atoms=100):
    pot = P.Potential.from_dict(pot_dict("bcc-l16-s1"))
    x = torch.tensor(st.x, dtype=torch.float64, device="cuda")
    z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    out = P.mtp_compute_grade(pot, nl, x, z, st.cell,
                              a_inv=torch.tensor(a_inv, device="cuda") if a_inv is not None else None,
                              a_inv_cfg=torch.tensor(a_cfg, device="cuda") if a_cfg is not None else None,
                              tau_sel=TAU_SEL, tau_brk=TAU_BRK, chunk_atoms=chunk_atoms, method=method)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("method,chunk", [("tensor", 100), ("tensor", 129), ("tensor", 0), ("fp64", 100)])
def test_grade_matches_oracle_flags_bit_exact(P, active, method, chunk):
    """300 atoms in chunks of 100 (one ragged tile each), 129 (a full tile and
    a one-row tile) or one chunk."""
    a_inv, a_cfg, _ = active
    st = synth.crystal("bcc", (6, 5, 5), 3.16, 0.15, 1, 5)
    meth = P.MTP_GRADE_TENSOR if method == "tensor" else P.MTP_GRADE_FP64
    out = run(P, st, a_inv, a_cfg, method=meth, chunk_atoms=chunk)
    model = oracle_model("bcc-l16-s1")
    b = O.basis_matrix(model, st.x, st.z, st.cell, O.neighbor_list(st.x, st.cell, st.pbc, 5.0))
    gam = O.grade(b, a_inv)
    got = out["gamma"].cpu().numpy()
    assert np.all(np.abs(got - gam) <= 1e-7 * gam)
    assert np.array_equal(out["flags"].cpu().numpy(), O.grade_flags(gam, TAU_SEL, TAU_BRK))
    assert out["gamma_max"] == pytest.approx(gam.max(), rel=1e-7)
    g_cfg = np.abs(b.sum(0) @ a_cfg).max()
    assert out["gamma_cfg"] == pytest.approx(g_cfg, rel=1e-7)
    assert out["status"] == (1 if max(gam.max(), g_cfg) > TAU_BRK else 0)
    assert out["n_ambiguous"] == 0
    # the tensor-core method re-checks exactly the rows within 5% of a threshold
    near = (np.abs(gam - TAU_SEL) <= 0.05 * TAU_SEL) | (np.abs(gam - TAU_BRK) <= 0.05 * TAU_BRK)
    if method == "tensor":
        assert out["n_rechecked"] == int(near.sum())
    else:
        assert out["n_rechecked"] == 0


def test_tensor_and_fp64_methods_agree(P, active):
    """Both products on a 1,024-atom sigma = 0.15 A box: identical flags, grades
    within 1e-7 relative of each other."""
    a_inv, _, _ = active
    st = synth.crystal("bcc", (8, 8, 8), 3.16, 0.15, 1, 5, sub=3)
    t = run(P, st, a_inv, None, method=P.MTP_GRADE_TENSOR, chunk_atoms=0)
    f = run(P, st, a_inv, None, method=P.MTP_GRADE_FP64, chunk_atoms=0)
    gt, gf = t["gamma"].cpu().numpy(), f["gamma"].cpu().numpy()
    assert np.all(np.abs(gt - gf) <= 1e-7 * gf)
    assert np.array_equal(t["flags"].cpu().numpy(), f["flags"].cpu().numpy())
    assert t["gamma_max"] == pytest.approx(f["gamma_max"], rel=1e-7)


def test_grade_is_one_on_the_active_set_and_bounded_on_its_pool(P, active):
    """The pool the active set was selected from (MaxVol, delta 0.01): every
    grade <= 1.01 and the active rows have grade 1.  Tolerance 1e-5: FP64
    rounding (~2e-16 relative in the basis rows, computed in another order
    than the oracle's) times the cancellation factor sum |b||A^-1| / gamma,
    which reaches ~4e8 on these near-degenerate lattice rows."""
    a_inv, _, d = active
    st = synth.crystal("bcc", (20, 20, 20), 3.16, 0.05, 1, 5, sub=8)
    out = run(P, st, a_inv, None)
    got = out["gamma"].cpu().numpy()
    rows = np.array(d["active_rows"])
    assert np.all(np.abs(got[rows] - 1.0) <= 1e-5)
    assert got.max() <= 1.01 + 1e-5
    assert np.all(out["flags"].cpu().numpy() == 0)


@pytest.mark.slow
def test_full_size_config5_sampled(P, active):
    """500,000-atom BCC (50 x 50 x 100 cells, sigma 0.15 A): sampled grades and
    flags against the oracle."""
    a_inv, a_cfg, _ = active
    st = synth.crystal("bcc", (50, 50, 100), 3.16, 0.15, 1, 5)
    out = run(P, st, a_inv, a_cfg)
    got = out["gamma"].cpu().numpy()
    flags = out["flags"].cpu().numpy()
    model = oracle_model("bcc-l16-s1")
    centres = np.sort(synth.rng(5, 77).choice(st.n, 32, replace=False))
    cand = min_image_candidates(st, centres, 5.5)
    nl = O.neighbor_list(st.x, st.cell, st.pbc, 5.0, query=centres, candidates=cand)
    b = O.basis_matrix(model, st.x, st.z, st.cell, nl, atoms=centres)
    gam = O.grade(b, a_inv)
    assert np.all(np.abs(got[centres] - gam) <= 1e-7 * gam)
    assert np.array_equal(flags[centres], O.grade_flags(gam, TAU_SEL, TAU_BRK))
    # rows whose FP64 grade lies within its own error bound of a threshold
    assert out["n_ambiguous"] <= 1e-3 * st.n


def test_level8_grade_padding_and_one_row_chunks(P):
    """Level-8 potential (m = 9: the tensor-core operands are mostly padding)
    with an active set chosen by the oracle's MaxVol on a 128-atom sigma =
    0.05 A box, evaluated on a 250-atom sigma = 0.15 A box in one chunk and in
    chunks of one row; flags bit-exact, grades within 1e-7 relative."""
    model = oracle_model("bcc-l8-s1")
    pool_st = synth.crystal("bcc", (4, 4, 4), 3.16, 0.05, 1, 11)
    pool = O.basis_matrix(model, pool_st.x, pool_st.z, pool_st.cell,
                          O.neighbor_list(pool_st.x, pool_st.cell, pool_st.pbc, 5.0))
    rows, a_inv, _ = O.maxvol(pool, delta=0.01)
    st = synth.crystal("bcc", (5, 5, 5), 3.16, 0.15, 1, 12)
    b = O.basis_matrix(model, st.x, st.z, st.cell, O.neighbor_list(st.x, st.cell, st.pbc, 5.0))
    gam = O.grade(b, a_inv)
    pot = P.Potential.from_dict(pot_dict("bcc-l8-s1"))
    x = torch.tensor(st.x, dtype=torch.float64, device="cuda")
    z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    for method in (P.MTP_GRADE_TENSOR, P.MTP_GRADE_FP64):
        for chunk in (0, 1):
            out = P.mtp_compute_grade(pot, nl, x, z, st.cell, a_inv=torch.tensor(a_inv, device="cuda"),
                                      tau_sel=TAU_SEL, tau_brk=TAU_BRK, chunk_atoms=chunk, method=method)
            torch.cuda.synchronize()
            got = out["gamma"].cpu().numpy()
            assert np.all(np.abs(got - gam) <= 1e-7 * gam), (method, chunk)
            assert np.array_equal(out["flags"].cpu().numpy(), O.grade_flags(gam, TAU_SEL, TAU_BRK))
