"""Both energy/force kernels against the oracle: one thread per atom (the
thread-parallel variant) and one warp per atom (the block-parallel variant for
small systems, paper Sec. 2.1, Table 1), forced through mtp_set_efv_variant,
with the tolerances of test_gpu_parity.py (at level 20 the mixed bound of
test_gpu_mixed_bound.py); the tuner's choice.
"""
import numpy as np
import pytest

import synth
from tests.helpers import pot_dict, structure
from tests.test_gpu_parity import EFV_CASES, dev, gpu_pot, oracle_efv

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = sorted(EFV_CASES)


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_00193_gb300 import build as B
    B.build()
    import paper_2510_00193_gb300 as P
    return P


def run(P, name, st, precision, variant, dtheta=True, chunk=0):
    pot = P.Potential.from_dict(pot_dict(name))
    P.mtp_set_efv_variant(pot, variant)
    x, z = dev(st)
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    out = P.mtp_compute_efv(pot, nl, x, z, st.cell, precision=precision, dtheta=dtheta, chunk_atoms=chunk)
    torch.cuda.synchronize()
    assert P.mtp_device_status(pot) == 0
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("case", CASES)
def test_kernel_variant_matches_oracle(P, case, variant):
    name = EFV_CASES[case][0]
    st, ref = oracle_efv(case)
    theta_ref = np.concatenate([ref["dE_ds"], ref["dE_dc"].ravel(), ref["dE_dxi"]])
    got = run(P, name, st, P.MTP_FP64, variant)
    assert np.all(np.abs(got["e_atom"] - ref["e_atom"]) <= 1e-12 * np.maximum(1.0, np.abs(ref["e_atom"])))
    assert np.abs(got["forces"] - ref["f"]).max() <= 1e-10
    assert np.abs(got["virial"] - ref["w"]).max() <= max(1e-10, 1e-10 * np.abs(ref["w"]).max())
    assert np.all(np.abs(got["dtheta"] - theta_ref) <= 1e-10 * np.maximum(1.0, np.abs(theta_ref)))
    mixed = run(P, name, st, P.MTP_MIXED, variant)
    tol = 1e-5 + (64 * 2.0 ** -24 * ref["abs_terms"] if pot_dict(name)["level"] > 16 else 0.0)
    assert np.all(np.abs(mixed["e_atom"] - ref["e_atom"]) <= tol)
    assert np.sqrt(np.mean((mixed["forces"] - ref["f"]) ** 2)) <= 1e-4
    assert np.abs(mixed["dtheta"] - theta_ref).max() <= 1e-4 * max(1.0, np.abs(theta_ref).max())


def test_warp_per_atom_in_chunks_and_against_thread_per_atom(P):
    """2,000 atoms (10^3 BCC cells, 3 species, level 16): the warp-per-atom
    kernel in one launch, in chunks of 333 (a ragged last chunk) and the
    thread-per-atom kernel agree to FP64 rounding."""
    name = "bcc-l16-s3"
    st = synth.crystal("bcc", (10, 10, 10), 3.16, 0.08, 3, 2)
    a = run(P, name, st, P.MTP_FP64, 2)
    b = run(P, name, st, P.MTP_FP64, 2, chunk=333)
    c = run(P, name, st, P.MTP_FP64, 1)
    for o in (b, c):
        assert np.abs(o["e_atom"] - a["e_atom"]).max() <= 1e-12 * np.abs(a["e_atom"]).max()
        assert np.abs(o["forces"] - a["forces"]).max() <= 1e-11 * max(1.0, np.abs(a["forces"]).max())
        assert np.abs(o["dtheta"] - a["dtheta"]).max() <= 1e-11 * np.abs(a["dtheta"]).max()


def test_tuner(P):
    name = "bcc-l16-s3"
    st = synth.crystal("bcc", (10, 10, 10), 3.16, 0.08, 3, 2)
    pot = P.Potential.from_dict(pot_dict(name))
    x, z = dev(st)
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    res = P.mtp_efv_tune(pot, nl, x, z, st.cell, precision=P.MTP_MIXED)
    assert res["chosen"] in (1, 2) and min(res["ms"]) > 0
    out = P.mtp_compute_efv(pot, nl, x, z, st.cell, precision=P.MTP_MIXED)
    ref = run(P, name, st, P.MTP_MIXED, res["chosen"], dtheta=False)
    assert np.abs(out["e_atom"].cpu().numpy() - ref["e_atom"]).max() <= 1e-9



def test_level20_warp_per_atom_against_three_kernels(P):
    """Level 20 (interpreted contraction) on a 2,048-atom FCC box (8^3 cells,
    4 species): the warp-per-atom kernel (per-group sweeps, warp-parallel
    interpreter) and the three-kernel thread-per-atom form agree to FP64
    rounding, with dE/dtheta, in one launch and in chunks of 700."""
    name = "fcc-l20-s4"
    st = synth.crystal("fcc", (8, 8, 8), 3.6, 0.1, 4, 3)
    a = run(P, name, st, P.MTP_FP64, 2)
    b = run(P, name, st, P.MTP_FP64, 2, chunk=700)
    c = run(P, name, st, P.MTP_FP64, 1)
    for o in (b, c):
        assert np.abs(o["e_atom"] - a["e_atom"]).max() <= 1e-12 * np.abs(a["e_atom"]).max()
        assert np.abs(o["forces"] - a["forces"]).max() <= 1e-11 * max(1.0, np.abs(a["forces"]).max())
        assert np.abs(o["dtheta"] - a["dtheta"]).max() <= 1e-11 * np.abs(a["dtheta"]).max()
