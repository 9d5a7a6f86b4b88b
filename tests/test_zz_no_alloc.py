"""mtp_compute_efv_noalloc against mtp_compute_efv (mixed precision).

The no-allocation entry point is for callers that cannot let the library
allocate device memory during a step (a fixed device-memory budget laid out at
start-up, or loops where cudaMalloc's device-wide synchronisation is not
acceptable).  Its results must equal the regular entry point's within the
mixed-precision tolerance used elsewhere in these tests (site energies 1e-5 eV,
forces 1e-4 eV/A), on two calls in a row that reuse the shared scratch array.
This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

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


def _alloc(n):
    dev = "cuda"
    return {"e_atom": torch.full((n,), np.nan, dtype=torch.float64, device=dev),
            "forces": torch.full((n, 3), np.nan, dtype=torch.float64, device=dev),
            "virial": torch.full((6,), np.nan, dtype=torch.float64, device=dev),
            "e_total": torch.full((1,), np.nan, dtype=torch.float64, device=dev)}


def test_noalloc_matches_regular_entry_point_on_two_calls(P):
    pot = P.Potential.from_dict(pot_dict("bcc-l16-s3"))
    # a larger configuration first, then a smaller one: the second call runs on
    # scratch that still holds the first call's positions
    for rec in [("bcc", (6, 5, 5), 3.16, 0.08, 3, 2), ("bcc", (4, 4, 3), 3.16, 0.08, 3, 2, 1)]:
        st = structure(*rec)
        x = torch.tensor(st.x, dtype=torch.float64, device="cuda")
        z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
        nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
        ref = P.mtp_compute_efv(pot, nl, x, z, st.cell, precision=P.MTP_MIXED)
        got = P.mtp_compute_efv_noalloc(pot, nl, x, z, st.cell, _alloc(st.n))
        torch.cuda.synchronize()
        assert P.mtp_device_status(pot) == 0
        r = {k: v.cpu().numpy() for k, v in ref.items() if v is not None}
        g = {k: v.cpu().numpy() for k, v in got.items()}
        assert np.abs(g["e_atom"] - r["e_atom"]).max() <= 1e-5
        assert np.abs(g["forces"] - r["forces"]).max() <= 1e-4
        assert np.abs(g["virial"] - r["virial"]).max() <= 1e-4 * max(1.0, np.abs(r["virial"]).max())
        assert abs(g["e_total"][0] - r["e_total"][0]) <= 1e-5 * st.n


def _compare(P, ref, got, n):
    r = {k: v.cpu().numpy() for k, v in ref.items() if v is not None}
    g = {k: v.cpu().numpy() for k, v in got.items()}
    assert np.abs(g["e_atom"] - r["e_atom"]).max() <= 1e-5
    assert np.abs(g["forces"] - r["forces"]).max() <= 1e-4
    assert np.abs(g["virial"] - r["virial"]).max() <= 1e-4 * max(1.0, np.abs(r["virial"]).max())
    assert abs(g["e_total"][0] - r["e_total"][0]) <= 1e-5 * n


def test_noalloc_call_leaves_device_memory_unchanged(P):
    """On a fresh handle, after one warm-up call (which looks up the scratch
    array's address and loads the kernels), a call on the largest allowed
    configuration (65,536 atoms, in chunks of 20,000 atoms) leaves the free
    device memory unchanged: a regular call would first grow the handle's
    buffers to that size."""
    pot = P.Potential.from_dict(pot_dict("bcc-l16-s3"))
    small = structure("bcc", (4, 4, 3), 3.16, 0.08, 3, 2, 1)
    big = structure("bcc", (32, 32, 32), 3.16, 0.08, 3, 2, 2)
    bufs = []
    for st in (small, big):
        x = torch.tensor(st.x, dtype=torch.float64, device="cuda")
        z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
        nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
        bufs.append((st, x, z, nl, _alloc(st.n)))
    st, x, z, nl, out = bufs[0]
    P.mtp_compute_efv_noalloc(pot, nl, x, z, st.cell, out, chunk_atoms=20000)
    torch.cuda.synchronize()
    st, x, z, nl, out = bufs[1]
    free0, _ = torch.cuda.mem_get_info()
    P.mtp_compute_efv_noalloc(pot, nl, x, z, st.cell, out, chunk_atoms=20000)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert P.mtp_device_status(pot) == 0
    ref = P.mtp_compute_efv(pot, nl, x, z, st.cell, precision=P.MTP_MIXED)
    torch.cuda.synchronize()
    _compare(P, ref, out, st.n)


def test_noalloc_level20_fused_path(P):
    """Level 20 (the interpreted contraction) on a 32-atom FCC box, 4 species:
    the fused kernel of this entry point against mtp_compute_efv's three-kernel
    split, on two calls in a row.  The two are different FP32 evaluations, so
    they agree within twice the mixed-precision bound of the other tests
    (site energies 1e-5 eV + 64 u a_i, forces 1e-4 eV/A + 64 u A_k, with a_i
    the sum of |xi_alpha B_alpha(i)| and A_k the sum of a over k and its
    neighbours)."""
    d = pot_dict("fcc-l20-s4")
    pot = P.Potential.from_dict(d)
    st = structure("fcc", (2, 2, 2), 3.6, 0.1, 4, 3)
    x = torch.tensor(st.x, dtype=torch.float64, device="cuda")
    z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    ref = P.mtp_compute_efv(pot, nl, x, z, st.cell, precision=P.MTP_MIXED)
    rows = P.mtp_compute_basis_rows(pot, nl, x, z, st.cell)
    a = (rows.abs() * torch.tensor(d["xi"], device="cuda").abs()).sum(1)
    off, j, _ = nl.to_tensors()
    ii = torch.repeat_interleave(torch.arange(st.n, device="cuda"), off[1:] - off[:-1])
    A = a.clone().index_add_(0, ii, a[j.long()])
    u = 2.0 ** -24
    tol_e = (2 * (1e-5 + 64 * u * a)).cpu().numpy()
    tol_f = (2 * (1e-4 + 64 * u * A)).cpu().numpy()
    for _ in range(2):
        got = P.mtp_compute_efv_noalloc(pot, nl, x, z, st.cell, _alloc(st.n))
        torch.cuda.synchronize()
        assert P.mtp_device_status(pot) == 0
        r = {k: v.cpu().numpy() for k, v in ref.items() if v is not None}
        g = {k: v.cpu().numpy() for k, v in got.items()}
        assert np.all(np.abs(g["e_atom"] - r["e_atom"]) <= tol_e)
        assert np.all(np.abs(g["forces"] - r["forces"]).max(axis=1) <= tol_f)
        assert abs(g["e_total"][0] - r["e_total"][0]) <= tol_e.sum()
        assert np.abs(g["virial"] - r["virial"]).max() <= 1e-4 * max(1.0, np.abs(r["virial"]).max())


def test_noalloc_rejects_configurations_beyond_its_scratch(P):
    from paper_2510_00193_gb300 import _lib
    pot = P.Potential.from_dict(pot_dict("bcc-l16-s3"))
    st = structure("bcc", (3, 3, 3), 3.16, 0.08, 3, 2)
    x = torch.tensor(st.x, dtype=torch.float64, device="cuda")
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    so = _lib.load()
    cell = np.ascontiguousarray(st.cell.reshape(-1), dtype=np.float64)
    dummy = ctypes.c_void_p(x.data_ptr())
    rc = so.mtp_compute_efv_noalloc(pot.handle, nl.handle, dummy, dummy, 65537,
                                    cell.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0, dummy, dummy, dummy,
                                    dummy, None)
    assert rc == -1
    assert b"at most 65536" in so.mtp_last_error()
