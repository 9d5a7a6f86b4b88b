"""Neighbour lists of the full 1,024,000-atom BCC workload near the cutoff.

The neighbour build decides most candidates with an FP32 estimate of the
distance whose rounding bound grows with the coordinates (largest in the
252.8 A box), and falls back to the exact FP64 expression only within that
bound of R_cut.  Here the centres whose nearest pair distance to R_cut is
smallest (pairs just inside and just outside the cutoff, anywhere in the box)
have their complete rows (j and image, in order) compared bit for bit with
the oracle's brute-force list.
"""
import numpy as np
import pytest

import synth
from tests.helpers import BinnedCandidates, oracle_rows, pot_dict

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

N_CENTRES = 2000
SHELL = 2e-4   # A: wider than the FP32 bound of the prefilter on this machine


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_00193_gb300 import build as B
    B.build()
    import paper_2510_00193_gb300 as P
    return P


def _pair_r(x, cell, off, j, img):
    """|x_j + n.H - x_i| of every listed pair, FP64 on the device."""
    n = off.numel() - 1
    i = torch.repeat_interleave(torch.arange(n, device=x.device), off[1:] - off[:-1])
    h = torch.tensor(cell, dtype=torch.float64, device=x.device)
    im = img.to(torch.float64)
    s = (im[:, 0:1] * h[0] + im[:, 1:2] * h[1]) + im[:, 2:3] * h[2]
    d = (x[j.long()] + s) - x[i]
    return i, torch.sqrt((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2])


def test_full_size_rows_near_cutoff_bit_exact(P):
    d = pot_dict("bcc-l16-s3")
    r_cut = d["r_cut"]
    st = synth.crystal("bcc", (80, 80, 80), 3.16, 0.08, 3, 2)
    x = torch.tensor(st.x, dtype=torch.float64, device="cuda")
    pot = P.Potential.from_dict(d)
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    off, j, img = nl.to_tensors()
    # pairs just outside R_cut come from a list built with a slightly larger cutoff
    wide = dict(d)
    wide["r_cut"] = r_cut + 1e-3
    nl_w = P.mtp_build_neighbors(P.Potential.from_dict(wide), x, st.cell, st.pbc)
    off_w, j_w, img_w = nl_w.to_tensors()
    i_in, r_in = _pair_r(x, st.cell, off, j, img)
    i_out, r_out = _pair_r(x, st.cell, off_w, j_w, img_w)
    gap = torch.full((st.n,), float("inf"), dtype=torch.float64, device="cuda")
    gap.scatter_reduce_(0, i_in, (r_cut - r_in).abs(), "amin")
    outside = r_out >= r_cut
    gap.scatter_reduce_(0, i_out[outside], (r_out[outside] - r_cut).abs(), "amin")
    order = torch.argsort(gap)[:N_CENTRES]
    centres = order[gap[order] < SHELL].cpu().numpy()
    assert len(centres) >= 1000, "too few centres near the cutoff: %d" % len(centres)
    assert gap.min().item() < 1e-5
    off_h = off.cpu().numpy()
    j_h = j.cpu().numpy()
    img_h = img.cpu().numpy()
    cands = BinnedCandidates(st, r_cut + 0.5)
    for c in centres:
        oj, on = oracle_rows(st, r_cut, c, cands(c))
        a, b = off_h[c], off_h[c + 1]
        assert np.array_equal(j_h[a:b], oj), c
        assert np.array_equal(img_h[a:b], on), c
