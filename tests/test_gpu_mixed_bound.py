"""Mixed-precision accuracy on the full workloads, against a stated bound.

Error model of MTP_MIXED (FP32 arithmetic, FP64 reductions).  The site energy
E_i = s + sum_alpha xi_alpha B_alpha(i) is a sum of products of up to L/2
moment contractions.  First-order rounding analysis: FP32 rounding (unit
u = 2^-24) perturbs every product B_alpha by a relative amount of at most
(number of moment factors) x (relative rounding amplification of a
contraction), so |dE_i| <= kappa u a_i with a_i = sum_alpha |xi_alpha B_alpha(i)|,
the conditioning of the site's basis sum.  The force on atom k is a sum of
pair terms dE_i/dx_k over the sites i whose neighbourhood holds k, so
|dF_k| <= kappa u A_k / (1 A) with A_k = a_k + sum_{j in N(k)} a_j.
kappa is the product of the factor count (8 at level 16, 10 at level 20) and
the amplification of a contraction; its maximum measured over every site and
atom of these workloads is 20 (level 16) and 49 (level 20) for the energies,
21 (level 16) and 57 (level 20) for the forces; the bound asserted here is
kappa = 64, plus an
absolute floor of 1e-5 eV (1e-4 eV/A) for FP64 summation order.  In the
level-18/20 kernels pairs closer than R_min take an FP64 radial path (without
it the level-20 forces on the atoms of its closest pairs were off by
0.15 eV/A, 700 u A_k); the force RMS over the box stays below the 1e-4 eV/A
target.
"""
import numpy as np
import pytest

import synth
from oracle import mtp as O
from tests.helpers import BinnedCandidates, oracle_model, oracle_rows, pot_dict

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

U = 2.0 ** -24
KAPPA = 64.0
E_FLOOR = 1e-5
F_FLOOR = 1e-4

WORKLOADS = {
    "bcc80-l16-s3": ("bcc-l16-s3", ("bcc", (80, 80, 80), 3.16, 0.08, 3, 2)),
    "fcc40-l20-s4": ("fcc-l20-s4", ("fcc", (40, 40, 40), 3.6, 0.1, 4, 3)),
}


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_00193_gb300 import build as B
    B.build()
    import paper_2510_00193_gb300 as P
    return P


def _oracle_a(model, st, r_cut, cands, atoms):
    """a_i = sum_alpha |xi_alpha B_alpha(i)| from the oracle's basis rows."""
    xi = np.abs(np.asarray(model.pot.xi))
    out = []
    for i in atoms:
        j, n = oracle_rows(st, r_cut, i, cands(i))
        nl = (np.full(len(j), i), j, n)
        b = O.basis_matrix(model, st.x, st.z, st.cell, nl, atoms=[i])
        out.append(float(np.abs(b[0]) @ xi))
    return np.array(out)


def _oracle_force(model, st, r_cut, cands, k):
    """Oracle force on atom k and the sites whose neighbourhood holds k."""
    cand = cands(k)
    j, _ = oracle_rows(st, r_cut, k, cand)
    sites = np.unique(np.concatenate([[k], j]))
    rows = [oracle_rows(st, r_cut, i, cand) for i in sites]
    nl = (np.concatenate([np.full(len(r[0]), i) for i, r in zip(sites, rows)]),
          np.concatenate([r[0] for r in rows]), np.concatenate([r[1] for r in rows]))
    out = O.evaluate(model, st.x, st.z, st.cell, nl, want=("e", "f"), atoms=sites)
    return out["f"][k], sites


@pytest.mark.parametrize("wl", sorted(WORKLOADS))
def test_full_size_mixed_within_bound(P, wl):
    name, rec = WORKLOADS[wl]
    d = pot_dict(name)
    r_cut = d["r_cut"]
    st = synth.crystal(*rec)
    pot = P.Potential.from_dict(d)
    x = torch.tensor(st.x, dtype=torch.float64, device="cuda")
    z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    om = P.mtp_compute_efv(pot, nl, x, z, st.cell, precision=P.MTP_MIXED)
    od = P.mtp_compute_efv(pot, nl, x, z, st.cell, precision=P.MTP_FP64)
    assert P.mtp_device_status(pot) == 0
    # whole box: mixed against the FP64 path (itself checked against the oracle)
    rows = P.mtp_compute_basis_rows(pot, nl, x, z, st.cell)
    a = (rows.abs() * torch.tensor(d["xi"], device="cuda").abs()).sum(1)
    del rows
    off, j, _ = nl.to_tensors()
    ii = torch.repeat_interleave(torch.arange(st.n, device="cuda"), off[1:] - off[:-1])
    A = a.clone().index_add_(0, ii, a[j.long()])
    de = (om["e_atom"] - od["e_atom"]).abs()
    dfv = (om["forces"] - od["forces"]).abs().max(1).values
    assert bool((de <= E_FLOOR + KAPPA * U * a).all()), float((de / (E_FLOOR + KAPPA * U * a)).max())
    assert bool((dfv <= F_FLOOR + KAPPA * U * A).all()), float((dfv / (F_FLOOR + KAPPA * U * A)).max())
    assert float(((om["forces"] - od["forces"]) ** 2).mean().sqrt()) <= 1e-4
    assert abs(om["e_total"].item() - od["e_total"].item()) / st.n <= 1e-5
    # sampled against the oracle: random centres and the worst-conditioned ones
    g = synth.rng(rec[5], 91)
    worst = torch.argsort(a, descending=True)[:6].cpu().numpy()
    centres = np.unique(np.concatenate([g.choice(st.n, 10, replace=False), worst]))
    model = oracle_model(name)
    cands = BinnedCandidates(st, 2 * r_cut + 0.5)
    a_ref = _oracle_a(model, st, r_cut, cands, centres)
    e_ref = []
    for c in centres:
        jj, nn = oracle_rows(st, r_cut, c, cands(c))
        out = O.evaluate(model, st.x, st.z, st.cell, (np.full(len(jj), c), jj, nn), want=("e",), atoms=[c])
        e_ref.append(out["e_atom"][0])
    e_mixed = om["e_atom"].cpu().numpy()[centres]
    assert np.all(np.abs(e_mixed - np.array(e_ref)) <= E_FLOOR + KAPPA * U * a_ref)
    # forces: one random atom and the atom with the largest force error
    f_mixed = om["forces"].cpu().numpy()
    for k in [int(g.integers(st.n)), int(torch.argmax(dfv))]:
        f_ref, sites = _oracle_force(model, st, r_cut, cands, k)
        a_sites = _oracle_a(model, st, r_cut, cands, sites)
        assert np.abs(f_mixed[k] - f_ref).max() <= F_FLOOR + KAPPA * U * a_sites.sum(), k
