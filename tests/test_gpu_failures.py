"""Failure handling, injected from the host (no fault is made on the GPU).

Every entry point returns a status and never aborts (paper Sec. 2.3: the run
halts above the break threshold; everything else here is an input error):
  - a non-finite position: mtp_build_neighbors returns MTP_ERR_NONFINITE; on
    a list built before the position went bad, the energy/force call records
    MTP_ERR_NONFINITE in the device status word (both precisions);
  - a species index outside 0..S-1: the device status word reports
    MTP_ERR_ARG and no table lookup leaves its array (the bad atom reads as
    species 0);
  - a cell too thin for the cutoff (an image beyond +-511 cells):
    MTP_ERR_NEIGHBOR_OVERFLOW;
  - a singular cell: MTP_ERR_ARG;
  - a grade above the break threshold: MTP_STATUS_BREAK;
  - a pipeline wait of the tensor-core grade kernel that runs out (limit set
    to 0 ns from the host): MTP_ERR_TIMEOUT, after which the same call with the
    default limit gives the bit-identical result.
After each failure a valid call on the same handle gives the results of a
fresh handle.
"""
import ctypes

import numpy as np
import pytest

import synth
from tests.helpers import pot_dict, structure

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


def _setup(P, name="bcc-l16-s3", rec=("bcc", (4, 4, 3), 3.16, 0.08, 3, 2)):
    st = structure(*rec)
    pot = P.Potential.from_dict(pot_dict(name))
    x = torch.tensor(st.x, dtype=torch.float64, device="cuda")
    z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
    return st, pot, x, z


def _code(excinfo):
    return excinfo.value.code


def _clean_call_matches_fresh(P, st, pot, x, z, precision):
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    got = P.mtp_compute_efv(pot, nl, x, z, st.cell, precision=precision)
    assert P.mtp_device_status(pot) == 0
    fresh = P.Potential.from_dict(pot_dict("bcc-l16-s3"))
    ref = P.mtp_compute_efv(fresh, nl, x, z, st.cell, precision=precision)
    torch.cuda.synchronize()
    assert torch.allclose(got["e_atom"], ref["e_atom"], rtol=0, atol=1e-12)
    assert torch.allclose(got["forces"], ref["forces"], rtol=0, atol=1e-4 if precision == P.MTP_MIXED else 1e-12)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nonfinite_position(P, precision):
    prec = P.MTP_FP64 if precision == "fp64" else P.MTP_MIXED
    st, pot, x, z = _setup(P)
    bad = x.clone()
    bad[5, 1] = float("nan")
    with pytest.raises(P.MtpError) as e:
        P.mtp_build_neighbors(pot, bad, st.cell, st.pbc)
    assert _code(e) == -5
    inf = x.clone()
    inf[7, 0] = float("inf")
    with pytest.raises(P.MtpError) as e:
        P.mtp_build_neighbors(pot, inf, st.cell, st.pbc)
    assert _code(e) == -5
    # a list built while the positions were finite, then a NaN position
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    P.mtp_compute_efv(pot, nl, bad, z, st.cell, precision=prec)
    with pytest.raises(P.MtpError) as e:
        P.mtp_device_status(pot)
    assert _code(e) == -5
    _clean_call_matches_fresh(P, st, pot, x, z, prec)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_species_out_of_range(P, precision):
    prec = P.MTP_FP64 if precision == "fp64" else P.MTP_MIXED
    st, pot, x, z = _setup(P)
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    for bad_value in (3, -1, 1 << 20):
        bad = z.clone()
        bad[2] = bad_value
        out = P.mtp_compute_efv(pot, nl, x, bad, st.cell, precision=prec, dtheta=True)
        with pytest.raises(P.MtpError) as e:
            P.mtp_device_status(pot)
        assert _code(e) == -1
        torch.cuda.synchronize()
        assert bool(torch.isfinite(out["e_atom"]).all())   # read as species 0: a defined value
    _clean_call_matches_fresh(P, st, pot, x, z, prec)


def test_cell_too_thin_for_the_cutoff(P):
    """Two atoms in a cell 0.004 A thin along c: images up to 1250 cells away
    lie within the cutoff, beyond the +-511 the list stores."""
    pot = P.Potential.from_dict(pot_dict("bcc-l8-s1"))
    cell = np.diag([12.0, 12.0, 0.004])
    x = torch.tensor([[1.0, 1.0, 0.001], [4.0, 2.0, 0.003]], dtype=torch.float64, device="cuda")
    with pytest.raises(P.MtpError) as e:
        P.mtp_build_neighbors(pot, x, cell, (1, 1, 1))
    assert _code(e) == -4
    # with c at 0.02 A the images stay within +-511 cells and the build succeeds
    nl = P.mtp_build_neighbors(pot, x, np.diag([12.0, 12.0, 0.02]), (1, 1, 1))
    assert nl.info()[1] > 0


def test_singular_cell(P):
    st, pot, x, z = _setup(P)
    sing = np.array(st.cell, dtype=np.float64)
    sing[2] = sing[0] + sing[1]
    with pytest.raises(P.MtpError) as e:
        P.mtp_build_neighbors(pot, x, sing, st.pbc)
    assert _code(e) == -1
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    for prec in (P.MTP_FP64, P.MTP_MIXED):
        with pytest.raises(P.MtpError) as e:
            P.mtp_compute_efv(pot, nl, x, z, sing, precision=prec)
        assert _code(e) == -1


def test_grade_above_break_threshold(P):
    import json
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "potentials", "bcc-l16-s1-active.json")) as fh:
        act = json.load(fh)
    m = act["m"]
    pot = P.Potential.from_dict(pot_dict("bcc-l16-s1"))
    st = synth.crystal("bcc", (3, 3, 3), 3.16, 0.15, 1, 5)
    x = torch.tensor(st.x, dtype=torch.float64, device="cuda")
    z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    a_inv = torch.tensor(act["a_inv"], dtype=torch.float64, device="cuda").reshape(m, m)
    ok = P.mtp_compute_grade(pot, nl, x, z, st.cell, a_inv=a_inv, tau_sel=1e6, tau_brk=1e7)
    assert ok["status"] == 0
    g = ok["gamma_max"]
    brk = P.mtp_compute_grade(pot, nl, x, z, st.cell, a_inv=a_inv, tau_sel=0.5 * g, tau_brk=0.5 * g)
    assert brk["status"] == P.MTP_STATUS_BREAK
    flags = brk["flags"].cpu().numpy()
    gam = brk["gamma"].cpu().numpy()
    assert np.array_equal(flags & 2, (gam > 0.5 * g).astype(np.uint8) * 2)


def test_tensor_core_wait_timeout(P):
    """The pipeline waits of the tensor-core kernel given a 0 ns limit give up
    (MTP_ERR_TIMEOUT); the kernel drains what it issued and frees its Tensor
    Memory, and the next launch with the default limit is bit-identical to
    one made before the timeout."""
    from paper_2510_00193_gb300 import _lib
    rows = 128 * 24
    g = torch.Generator(device="cuda").manual_seed(7)
    to_bf16 = lambda t: (t.to(torch.float32).view(torch.int32) >> 16).to(torch.int16)  # noqa: E731
    xs = to_bf16(torch.randint(-128, 129, (((rows + 127) // 128) * 7 * 128 * 128,), device="cuda", generator=g,
                               dtype=torch.int32))
    ys = to_bf16(torch.randint(-128, 129, (2 * 7 * 64 * 128,), device="cuda", generator=g, dtype=torch.int32))
    fexp = torch.zeros(128, dtype=torch.int32, device="cuda")
    erow = torch.zeros(rows, dtype=torch.int32, device="cuda")
    before = P.mtp_grade_tc_selftest(xs, ys, fexp, erow, rows)
    torch.cuda.synchronize()
    ref = before["gamma_bits"].clone() if isinstance(before, dict) else before.clone()
    so = _lib.load()
    try:
        so.mtp_set_wait_limit(0)
        with pytest.raises(P.MtpError) as e:
            P.mtp_grade_tc_selftest(xs, ys, fexp, erow, rows)
        assert _code(e) == -6
    finally:
        so.mtp_set_wait_limit(-1)
    after = P.mtp_grade_tc_selftest(xs, ys, fexp, erow, rows)
    torch.cuda.synchronize()
    got = after["gamma_bits"] if isinstance(after, dict) else after
    assert torch.equal(got, ref)
    torch.cuda.synchronize()   # the context is still usable
