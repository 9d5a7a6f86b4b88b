"""Configuration-mode grade over the full parameter gradient (paper Sec. 2.1,
configuration mode, as MLIP defines it: a configuration is represented by the
derivatives of its energy with respect to every parameter,
b_cfg = dE/dtheta = [dE/ds | dE/dc | dE/dxi]).

Active set: MaxVol (delta 0.01) over the oracle's dE/dtheta rows of a pool of
4 n_params seeded small configurations (2 x 2 x 2 BCC cells, sigma 0.05 A,
cell strains U[-2%, 2%] per axis), restricted to a maximal set of linearly
independent columns (the oracle's independent_columns: the full gradient has
n_mu (n_mu + 1) / 2 = 3 exact relations at level 8), inverted by the oracle's
Gauss-Jordan.
Graded: 24 configurations with sigma 0.15 A and strains of up to 4%.
The device computes dE/dtheta of all of them in one batch launch (FP64) and
grades the rows with mtp_grade_rows; against the oracle's
gamma = max_k |(dE/dtheta A^-1)_k|:
  grades within 1e-6 relative (entries of dE/dtheta agree to 1e-10 relative,
  amplified by the cancellation in b A^-1);
  flags bit-exact, with both thresholds placed in gaps between the oracle's
  grades wider than that tolerance;
  gamma = 1 (within 1e-6) on the active configurations themselves;
  MaxVol on the device rows selects the oracle's rows from the same start.
"""
import numpy as np
import pytest

import synth
from oracle import mtp as O
from tests.helpers import oracle_model, pot_dict

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NAME = "bcc-l8-s1"


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_00193_gb300 import build as B
    B.build()
    import paper_2510_00193_gb300 as P
    return P


def _configs(n, sigma, strain, stream):
    g = synth.rng(stream, 61)
    out = []
    for k in range(n):
        st = synth.crystal("bcc", (2, 2, 2), 3.16, sigma, 1, stream, sub=100 + k)
        d = np.diag(1.0 + g.uniform(-strain, strain, size=3))
        out.append(synth.Structure(st.x @ d, st.z, st.cell @ d, st.pbc))
    return out


def _oracle_rows(model, structs):
    rows = []
    for st in structs:
        nl = O.neighbor_list(st.x, st.cell, st.pbc, model.pot.r_cut)
        out = O.evaluate(model, st.x, st.z, st.cell, nl, want=("e", "dtheta"))
        rows.append(np.concatenate([out["dE_ds"], out["dE_dc"].ravel(), out["dE_dxi"]]))
    return np.array(rows)


def _device_rows(P, pot, structs):
    off = np.concatenate([[0], np.cumsum([s.n for s in structs])]).astype(np.int64)
    x = torch.tensor(np.concatenate([s.x for s in structs]), device="cuda")
    z = torch.tensor(np.concatenate([s.z for s in structs]).astype(np.int32), device="cuda")
    b = P.Batch(pot, off, np.stack([s.cell for s in structs]), x)
    out = P.mtp_compute_batch(pot, b, x, z, precision=P.MTP_FP64, dtheta=True)
    torch.cuda.synchronize()
    return out["dtheta"]


def _gap_threshold(sorted_vals, target, tol):
    """A threshold near `target` in a gap of the sorted values wider than tol."""
    best = None
    for lo, hi in zip(sorted_vals[:-1], sorted_vals[1:]):
        if hi - lo > 2 * tol * hi:
            mid = 0.5 * (lo + hi)
            if best is None or abs(mid - target) < abs(best - target):
                best = mid
    assert best is not None
    return best


def test_full_parameter_configuration_grade(P):
    model = oracle_model(NAME)
    pot = P.Potential.from_dict(pot_dict(NAME))
    n_params = pot.n_params
    pool = _configs(4 * n_params, 0.05, 0.02, 21)
    test = _configs(24, 0.15, 0.04, 22)
    rows_pool = _oracle_rows(model, pool)
    assert rows_pool.shape == (4 * n_params, n_params)
    cols = O.independent_columns(rows_pool)
    start = O.initial_rows(rows_pool[:, cols])
    active, a_inv, _ = O.maxvol(rows_pool[:, cols], start.copy(), delta=0.01)
    rows_test = _oracle_rows(model, test)
    gam_ref = O.grade(rows_test[:, cols], a_inv)
    srt = np.sort(gam_ref)
    tau_sel = _gap_threshold(srt, np.median(srt), 1e-6)
    tau_brk = max(tau_sel, _gap_threshold(srt, srt[-3], 1e-6))
    flags_ref = O.grade_flags(gam_ref, tau_sel, tau_brk)
    assert flags_ref.any() and not flags_ref.all()

    a_inv_d = torch.tensor(a_inv, device="cuda")
    cols_d = torch.tensor(cols, dtype=torch.int32, device="cuda")
    dev_test = _device_rows(P, pot, test)
    assert np.allclose(dev_test.cpu().numpy(), rows_test, rtol=1e-10, atol=1e-10 * np.abs(rows_test).max())
    got = P.mtp_grade_rows(dev_test, a_inv_d, tau_sel, tau_brk, cols=cols_d)
    gam = got["gamma"].cpu().numpy()
    assert np.all(np.abs(gam - gam_ref) <= 1e-6 * gam_ref)
    assert np.array_equal(got["flags"].cpu().numpy(), flags_ref)
    assert got["status"] == (P.MTP_STATUS_BREAK if gam_ref.max() > tau_brk else 0)
    # the active configurations grade 1
    dev_pool = _device_rows(P, pot, pool)
    act = P.mtp_grade_rows(dev_pool[torch.tensor(active, device="cuda")].contiguous(), a_inv_d, 2.0, 10.0,
                           cols=cols_d)
    assert np.allclose(act["gamma"].cpu().numpy(), 1.0, rtol=0, atol=1e-6)
    # MaxVol on the device rows (the same columns) from the same start selects the same rows
    sel, _, _ = P.mtp_maxvol(dev_pool[:, torch.tensor(cols, device="cuda")].contiguous(), start.copy(), delta=0.01)
    assert np.array_equal(np.asarray(sel), np.asarray(active))
